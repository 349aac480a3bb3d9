"""Batched and served solves give what the same solves give alone.

Every kernel of a solve is deterministic (claims are resolved by exact keys,
reductions run in a fixed order), so a solve advanced inside a batch graph,
or among other requests on the server, must match the same solve advanced on
its own bit for bit.
"""
import numpy as np
import pytest

from paper_1705_03750_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1705_03750_gb300 import build as B  # noqa: E402

B.build()
from paper_1705_03750_gb300 import vlamet as V  # noqa: E402
from paper_1705_03750_gb300.serve import GpuBackend, Request, Server  # noqa: E402


def _solver(rc, prec):
    s = V.Solver(V.Config.from_run(rc, prec), stream=torch.cuda.Stream())
    s.set_f(I.initial_f(rc))
    return s


@pytest.mark.parametrize("prec", [V.VM_FP32_MIXED, V.VM_FP64])
def test_batch_graph_matches_individual_solves(prec):
    cfgs = [I.batch_member(i).with_(n_s=10) for i in range(6)]
    alone = [_solver(rc, prec) for rc in cfgs]
    for s in alone:
        s.step(23)                      # two remaps included
    batched = [_solver(rc, prec) for rc in cfgs]
    b = V.Batch(batched, nstreams=4)
    b.step(20)
    b.step(3)
    assert b.launches_per_step(False) > 0 and b.launches_per_step(True) > b.launches_per_step(False)
    for s1, s2 in zip(alone, batched):
        s1.sync()
        s2.sync()
        np.testing.assert_array_equal(s1.read_f(), s2.read_f())
        np.testing.assert_array_equal(s1.read_fini(), s2.read_fini())
        np.testing.assert_array_equal(s1.elements(), s2.elements())
        d1, d2 = s1.density_force(), s2.density_force()
        for k in d1:
            np.testing.assert_array_equal(d1[k], d2[k])
    b.close()


def test_batch_refuses_solves_out_of_phase():
    a = _solver(I.batch_member(0).with_(n_s=10), V.VM_FP32_MIXED)
    c = _solver(I.batch_member(1).with_(n_s=10), V.VM_FP32_MIXED)
    a.step(1)
    with pytest.raises(V.VlametError) as e:
        V.Batch([a, c])
    assert e.value.status == 7


def test_served_result_is_the_same_alone_and_in_the_mix():
    mk = lambda i, nx, nv, steps: Request(i, I.HALOS_4096.with_(nx=nx, nv=nv, seed=100 + i), steps, 0.0)  # noqa: E731
    target = lambda: mk(0, 384, 320, 30)  # noqa: E731
    srv = Server(GpuBackend(), budget_bytes=8 << 30, max_active=8, ic_fn=I.initial_f)
    srv.run([target()])
    alone = srv.done[0].result
    mix = [target()] + [mk(i, 256 + 64 * i, 512 - 32 * i, 10 + 7 * i) for i in range(1, 6)]
    srv2 = Server(GpuBackend(), budget_bytes=8 << 30, max_active=4, ic_fn=I.initial_f)
    rep = srv2.run(mix)
    assert rep["requests"] == 6 and srv2.peak_active >= 2
    in_mix = next(r for r in srv2.done if r.rid == 0).result
    for k in alone:
        np.testing.assert_array_equal(alone[k], in_mix[k])
