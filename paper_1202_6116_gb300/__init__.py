"""GB300-native time-domain ferroelectric phase-field step (TDGL + Poisson).

The computation lives in the CUDA library behind the C ABI of
``include/pf.h``; ``pf`` is its ctypes binding (same function names),
``film.Film`` a convenience wrapper holding the state in torch tensors, and
``workloads`` the seeded synthetic inputs.  Nothing is loaded at import time;
the first ABI call loads the library and raises if it is not built.
"""
__all__ = ["pf", "film", "workloads", "build"]
