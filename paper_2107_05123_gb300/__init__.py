"""GB300 (sm_103a) library for the matrix-free hot path of the projection-based CHNS scheme on
adaptive octrees (arXiv:2107.05123): mesh tables from a leaf list, matrix-free operator applies,
Krylov solves and the two-block time step, behind the C ABI of include/chns.h.

``paper_2107_05123_gb300.capi`` is the thin ctypes binding (same names as the C entry points);
``paper_2107_05123_gb300.session`` holds small conveniences on top of it (torch device buffers,
default solver settings). Accessing ``capi`` loads libchns.so and raises ImportError when it has
not been built: there is no fallback implementation.
"""


def __getattr__(name):
    if name == "capi":
        from . import _lib
        return _lib
    raise AttributeError(name)
