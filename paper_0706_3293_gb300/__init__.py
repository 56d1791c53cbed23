"""GB300 (sm_103a) sector Lanczos for Heisenberg spin models.

Hot path of Schnack, Hage and Schmidt, "Optimized implementation of the Lanczos method
for magnetic systems" (arXiv:0706.3293): the matrix-free product y = H x on one sector
H(M) with the paper's direct D(N, A) basis coding, row-oriented (Eq. E-4-b), and the
Lanczos recurrence around it.  The compute runs in libhm.so (include/hm.h); this package
is its Python binding.
"""
from . import workloads  # noqa: F401  (input generators, no CUDA needed)


def __getattr__(name):
    # the binding needs torch and the built library; import it on first use
    if name in ("api", "autograd", "_capi"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
