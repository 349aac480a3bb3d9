"""Batched and served solves give what the same solves give alone.

Every kernel of a solve is deterministic (claims are resolved by exact keys,
reductions run in a fixed order), and a group launch runs, for each solve,
exactly the blocks of that solve's own launches, so a solve advanced inside
a batch graph, or among other requests on the library's serving loop, must
match the same solve advanced on its own bit for bit, whatever the launch
shapes the tuner picks.
"""
import time

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
from paper_1705_03750_gb300.serve import Request, run_open_loop  # noqa: E402


def _solver(rc, prec):
    s = V.Solver(V.Config.from_run(rc, prec), stream=torch.cuda.Stream())
    s.set_f(I.initial_f(rc))
    return s


def _same(s1, s2):
    s1.sync()
    s2.sync()
    np.testing.assert_array_equal(s1.read_f(), s2.read_f())
    np.testing.assert_array_equal(s1.read_fini(), s2.read_fini())
    np.testing.assert_array_equal(s1.elements(), s2.elements())
    d1, d2 = s1.density_force(), s2.density_force()
    for k in d1:
        np.testing.assert_array_equal(d1[k], d2[k])


def _solver_mode(rc, prec, mode):
    cfg = V.Config.from_run(rc, prec)
    cfg.recon_mode = mode
    s = V.Solver(cfg, stream=torch.cuda.Stream())
    s.set_f(I.initial_f(rc))
    return s


@pytest.mark.parametrize("prec,mode", [(V.VM_FP32_MIXED, 0), (V.VM_FP64, 0), (V.VM_FP32_MIXED, 1)],
                         ids=["fp32", "fp64", "fp32-tiles"])
def test_batch_graph_matches_individual_solves(prec, mode):
    cfgs = [I.batch_member(i).with_(n_s=10) for i in range(6)]
    _solver = lambda rc, prec: _solver_mode(rc, prec, mode)  # noqa: E731
    alone = [_solver(rc, prec) for rc in cfgs]
    for s in alone:
        s.step(23)                      # two remaps included
    batched = [_solver(rc, prec) for rc in cfgs]
    b = V.Batch(batched)
    b.step(20)
    b.step(3)
    # about twenty launches per step for the whole batch
    assert 0 < b.launches_per_step(False) < 40 and b.launches_per_step(True) > b.launches_per_step(False)
    for s1, s2 in zip(alone, batched):
        _same(s1, s2)
        assert s2.diagnostics()["step"] == 23
    b.close()


def test_batch_autotune_changes_no_result():
    cfgs = [I.batch_member(i).with_(n_s=6) for i in range(10, 18)]
    prec = V.VM_FP32_MIXED
    alone = [_solver(rc, prec) for rc in cfgs]
    for s in alone:
        s.step(20)
    batched = [_solver(rc, prec) for rc in cfgs]
    b = V.Batch(batched)
    t = b.autotune(1)                   # 4 shapes x 1 timed step (and a remap step when one comes)
    assert t["tuned"] and set(t["blocks_per_sm"].values()) <= {1, 2, 4, 8}
    done = batched[0].diagnostics()["step"]
    assert done >= 4
    b.step(20 - done)
    for s1, s2 in zip(alone, batched):
        _same(s1, s2)
    b.close()


def test_batch_refuses_solves_out_of_phase_or_precision():
    a = _solver(I.batch_member(0).with_(n_s=10), V.VM_FP32_MIXED)
    c = _solver(I.batch_member(1).with_(n_s=10), V.VM_FP32_MIXED)
    a.step(1)
    with pytest.raises(V.VlametError) as e:
        V.Batch([a, c])
    assert e.value.status == 7
    d = _solver(I.batch_member(2).with_(n_s=10), V.VM_FP64)
    with pytest.raises(V.VlametError) as e:
        V.Batch([c, d])
    assert e.value.status == 1


def _emap_solver(rc, prec, thr):
    cfg = V.Config.from_run(rc, prec)
    cfg.emap_remap = thr
    s = V.Solver(cfg, stream=torch.cuda.Stream())
    s.set_f(I.initial_f(rc))
    return s


def _median_emap(rc, prec, steps=8):
    s = _solver(rc, prec)
    seen = []
    for _ in range(steps):
        s.step(1)
        seen.append(s.diagnostics()["emap"])
    return float(np.median(seen))


@pytest.mark.parametrize("prec", [V.VM_FP32_MIXED, V.VM_FP64], ids=["fp32", "fp64"])
def test_batch_with_emap_remap_solves_matches_individual_solves(prec):
    # host-cycle solves (one shared remap phase) and E_map solves, which keep
    # their cycles on the device and join at other positions in them
    host = [I.batch_member(i).with_(n_s=10) for i in range(3)]
    emap = [I.batch_member(i).with_(n_s=6) for i in range(3, 7)]
    thr = [_median_emap(rc, prec) for rc in emap]
    pre = [0, 2, 5, 1]                  # steps each E_map solve takes before joining
    alone = [_solver(rc, prec) for rc in host] + [_emap_solver(rc, prec, t) for rc, t in zip(emap, thr)]
    for k, s in enumerate(alone):
        s.step(24 + (pre[k - 3] if k >= 3 else 0))
    batched = [_solver(rc, prec) for rc in host] + [_emap_solver(rc, prec, t) for rc, t in zip(emap, thr)]
    for k, p in enumerate(pre):
        batched[3 + k].step(p)
    b = V.Batch(batched)
    b.step(24)
    forced = 0
    for s1, s2 in zip(alone, batched):
        _same(s1, s2)
        d1, d2 = s1.diagnostics(), s2.diagnostics()
        assert (d1["cycle"], d1["emap_remaps"], d1["step"]) == (d2["cycle"], d2["emap_remaps"], d2["step"])
        forced += d2["emap_remaps"]
    assert forced > 0                   # some E_map remaps happened inside the batch
    b.close()


def _served(reqs, budget=8 << 30, max_active=8, tick=3, emap_remap=0.0):
    srv = V.NativeServer(budget, max_active=max_active, steps_per_tick=tick, emap_remap=emap_remap)
    rep = run_open_loop(srv, reqs, ic_fn=I.initial_f, keep_results=True)
    return srv, rep


def test_served_result_is_the_same_alone_in_the_mix_and_stepped_directly():
    mk = lambda i, nx, nv, steps, t: Request(i, I.HALOS_4096.with_(nx=nx, nv=nv, s=8, n_s=7, seed=100 + i),  # noqa: E731
                                              steps, t)
    target = lambda: mk(0, 384, 320, 30, 0.0)  # noqa: E731
    _, rep = _served([target()])
    assert rep["requests"] == 1 and rep["failed"] == 0
    # the same solve stepped by vm_step on its own
    rc = target().config
    s = V.Solver(V.Config.from_run(rc, V.VM_FP32_MIXED))
    s.set_f(I.initial_f(rc))
    s.step(30)
    direct = s.density_force()
    mix = [target()] + [mk(i, 256 + 64 * i, 512 - 32 * i, 10 + 7 * i, 0.002 * i) for i in range(1, 6)]
    srv, rep2 = _served(mix, max_active=4)
    assert rep2["requests"] == 6 and rep2["failed"] == 0 and rep2["peak_active"] >= 2
    res = next(r for r in mix if r.rid == 0).result
    for k in direct:
        np.testing.assert_array_equal(direct[k], res[k])
    st = srv.stats()
    assert st["group_steps"] < sum(r.steps for r in mix)   # steps of different requests shared launches
    assert st["used_bytes"] == 0 and st["active"] == 0


def test_served_emap_remap_request_matches_vm_step():
    # requests that remap on E_map keep their cycles on the device inside
    # the serving loop's group steps
    mk = lambda i, nx, nv, steps, t: Request(i, I.HALOS_4096.with_(nx=nx, nv=nv, s=8, n_s=7, seed=300 + i),  # noqa: E731
                                              steps, t)
    mix = [mk(i, 256 + 32 * i, 448 - 32 * i, 20 + 5 * i, 0.003 * i) for i in range(5)]
    thr = _median_emap(mix[0].config, V.VM_FP32_MIXED)
    srv, rep = _served(mix, max_active=3, emap_remap=thr)
    assert rep["requests"] == 5 and rep["failed"] == 0
    forced = 0
    for r in mix:
        cfg = V.Config.from_run(r.config, V.VM_FP32_MIXED)
        cfg.emap_remap = thr
        s = V.Solver(cfg)
        s.set_f(I.initial_f(r.config))
        s.step(r.steps)
        direct = s.density_force()
        forced += s.diagnostics()["emap_remaps"]
        for k in direct:
            np.testing.assert_array_equal(direct[k], r.result[k])
    assert forced > 0
    srv.close()


def test_server_mixes_emap_and_fixed_cycle_requests():
    # requests with and without the E_map criterion in one serving loop: the
    # gated remaps of the first and the host-cycle remap subsets of the
    # second share the steps; each result equals its solve stepped alone
    mk = lambda i, nx, nv, steps, t: Request(i, I.HALOS_4096.with_(nx=nx, nv=nv, s=8, n_s=5, seed=500 + i),  # noqa: E731
                                              steps, t)
    mix = [mk(i, 224 + 32 * i, 416 - 32 * i, 18 + 4 * i, 0.002 * i) for i in range(6)]
    thr = _median_emap(mix[0].config, V.VM_FP32_MIXED)
    use = {r.rid: (thr if r.rid % 2 == 0 else 0.0) for r in mix}
    srv = V.NativeServer(8 << 30, max_active=4, steps_per_tick=3)
    orig = srv.submit
    srv.submit = lambda rc, f0, steps: orig(rc, f0, steps, emap_remap=use[int(rc.name[3:])])  # noqa: E731
    for r in mix:
        r.config = r.config.with_(name=f"req{r.rid}")
    rep = run_open_loop(srv, mix, ic_fn=I.initial_f, keep_results=True)
    assert rep["requests"] == 6 and rep["failed"] == 0
    forced = 0
    for r in mix:
        cfg = V.Config.from_run(r.config, V.VM_FP32_MIXED)
        cfg.emap_remap = use[r.rid]
        s = V.Solver(cfg)
        s.set_f(I.initial_f(r.config))
        s.step(r.steps)
        forced += s.diagnostics()["emap_remaps"]
        direct = s.density_force()
        for k in direct:
            np.testing.assert_array_equal(direct[k], r.result[k])
    assert forced > 0
    srv.close()


def test_batch_autotune_with_emap_solves_changes_no_result():
    # the tuner's real steps include the gated remaps of the E_map solves
    host = [I.batch_member(i).with_(n_s=6) for i in range(20, 23)]
    emap = [I.batch_member(i).with_(n_s=6) for i in range(23, 26)]
    prec = V.VM_FP32_MIXED
    thr = [_median_emap(rc, prec) for rc in emap]
    alone = [_solver(rc, prec) for rc in host] + [_emap_solver(rc, prec, t) for rc, t in zip(emap, thr)]
    for s in alone:
        s.step(16)
    batched = [_solver(rc, prec) for rc in host] + [_emap_solver(rc, prec, t) for rc, t in zip(emap, thr)]
    b = V.Batch(batched)
    t = b.autotune(1)
    assert t["tuned"]
    done = batched[0].diagnostics()["step"]
    b.step(16 - done)
    for s1, s2 in zip(alone, batched):
        _same(s1, s2)
        assert s1.diagnostics()["emap_remaps"] == s2.diagnostics()["emap_remaps"]
    b.close()


def test_server_budget_bounds_the_resident_set_and_refuses_what_never_fits():
    rc = I.HALOS_4096.with_(nx=256, nv=256, s=8, n_s=5)
    need = V.workspace_bytes(V.Config.from_run(rc, V.VM_FP32_MIXED))
    reqs = [Request(i, rc.with_(seed=i), 12, 0.0) for i in range(4)]
    big = Request(9, rc.with_(nx=2048, nv=2048), 3, 0.0)
    srv, rep = _served(reqs + [big], budget=int(1.5 * need))
    assert rep["requests"] == 5 and rep["failed"] == 1 and "status 6" in big.error
    assert rep["peak_active"] == 1 and srv.stats()["peak_bytes"] <= 1.5 * need


def test_served_results_stay_exact_through_many_remap_subsets():
    """Requests admitted at different times remap in different steps: every
    step builds a plan for its remap subset (more than the server's ring of
    plan tables holds over the run) while the transport plan of the active
    set stays in use.  Each result must equal its solve stepped alone, and
    every served solve must report success."""
    mk = lambda i: Request(i, I.HALOS_4096.with_(nx=192 + 32 * (i % 3), nv=160 + 32 * (i % 4), s=4,  # noqa: E731
                                                 n_s=2 + (i % 3), seed=300 + i), 24 + 3 * i, 0.004 * i)
    reqs = [mk(i) for i in range(8)]
    srv, rep = _served(reqs, max_active=8, tick=2)
    assert rep["requests"] == 8 and rep["failed"] == 0
    assert srv.stats()["remap_groups"] > 20
    for r in reqs:
        s = V.Solver(V.Config.from_run(r.config, V.VM_FP32_MIXED))
        s.set_f(I.initial_f(r.config))
        s.step(r.steps)
        direct = s.density_force()
        for k in direct:
            np.testing.assert_array_equal(direct[k], r.result[k], err_msg=f"request {r.rid} {k}")
