"""GB300-native metric semi-Lagrangian Vlasov-Poisson solver (Colombi & Alard).

The solver lives in a C-ABI CUDA library (``csrc/``, declared in
``include/vlamet.h``); ``vlamet`` is its thin ctypes binding.  Importing the
package loads nothing: the library is opened on first use and the binding
raises if it is missing.
"""
__all__ = ["inputs", "vlamet"]
