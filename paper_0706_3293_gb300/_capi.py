"""ctypes declarations of the C ABI in include/hm.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libhm.so")

HM_OK, HM_BREAKDOWN, HM_DEGENERATE = 0, 1, 2
HM_EINVAL, HM_EPARITY, HM_EOVERFLOW, HM_ECUDA, HM_ENOMEM, HM_ETIMEOUT, HM_EWORKSPACE = (
    -1, -2, -3, -4, -5, -6, -7)
HM_F64, HM_F32 = 0, 1
HM_MAX_BONDS = 512

# every function the header declares (checked by tests/test_abi.py)
EXPORTS = [
    "hm_last_error", "basis_dim_query", "bonds_check", "basis_build", "basis_build_flip", "basis_build_momentum",
    "basis_free", "basis_dim",
    "basis_encode", "basis_decode", "matvec", "count_nnz", "bond_corr_workspace", "bond_corr", "bond_corr_static",
    "start_vector",
    "lanczos_workspace", "lanczos_init", "lanczos_step", "lanczos_substep", "lanczos_read", "lanczos_free",
    "lanczos_kernel_name", "matvec_kernel_name",
    "lanczos_run", "sector_ground_energies_workspace", "sector_ground_energies", "e0_grad_workspace", "e0_grad",
    "ftlm_workspace", "ftlm_run",
    "arnoldi_workspace", "arnoldi_run", "projection_workspace", "projection_run", "sym_eigenvalues",
]

_lib = None


class HMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def load() -> ctypes.CDLL:
    """Loads libhm.so; raises ImportError if it has not been built (no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(python -m paper_0706_3293_gb300.build)")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u64, sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                             ctypes.c_size_t)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    i64p = ctypes.POINTER(ctypes.c_int64)
    szp = ctypes.POINTER(ctypes.c_size_t)
    sig = {
        "hm_last_error": (ctypes.c_char_p, []),
        "basis_dim_query": (i32, [i32, i32, i32, i64p]),
        "bonds_check": (i32, [i32, i32, vp, vp, vp]),
        "basis_build": (i32, [i32, i32, i32, ctypes.POINTER(vp)]),
        "basis_build_flip": (i32, [i32, i32, ctypes.POINTER(vp)]),
        "basis_build_momentum": (i32, [i32, i32, i32, i32, ctypes.POINTER(vp)]),
        "basis_free": (i32, [vp]),
        "basis_dim": (i32, [vp, i64p]),
        "basis_encode": (i32, [vp, vp, vp, i64, vp]),
        "basis_decode": (i32, [vp, vp, vp, i64, vp]),
        "matvec": (i32, [vp, i32, vp, vp, vp, vp, vp, i32, i32, vp]),
        "count_nnz": (i32, [vp, i32, vp, vp, vp, vp]),
        "bond_corr_workspace": (i32, [vp, i32, szp]),
        "bond_corr": (i32, [vp, i32, vp, vp, vp, vp, vp, i32, vp, sz, vp]),
        "bond_corr_static": (i32, [vp, i32, vp, vp, vp, vp, vp, i32, vp]),
        "start_vector": (i32, [vp, u64, i32, vp, i32, vp]),
        "lanczos_workspace": (i32, [vp, i32, i32, szp]),
        "lanczos_init": (i32, [vp, i32, vp, vp, vp, vp, u64, i32, i32, vp, sz, vp,
                               ctypes.POINTER(vp)]),
        "lanczos_step": (i32, [vp, vp]),
        "lanczos_substep": (i32, [vp, i32, vp]),
        "lanczos_read": (i32, [vp, dp, dp, ip, vp]),
        "lanczos_free": (i32, [vp]),
        "lanczos_kernel_name": (i32, [vp, ctypes.c_char_p, i32]),
        "matvec_kernel_name": (i32, [vp, i32, vp, vp, vp, i32, i32, ctypes.c_char_p, i32]),
        "lanczos_run": (i32, [vp, i32, vp, vp, vp, vp, u64, i32, i32, vp, sz, dp, dp, ip, dp,
                              i32, vp]),
        "sector_ground_energies_workspace": (i32, [i32, i32, i32, i32, szp]),
        "sector_ground_energies": (i32, [i32, i32, i32, vp, vp, vp, i32, u64, i32, vp, sz, dp, ip, vp]),
        "e0_grad_workspace": (i32, [vp, i32, i32, szp]),
        "e0_grad": (i32, [vp, i32, vp, vp, vp, vp, u64, i32, vp, sz, dp, dp, vp, vp]),
        "ftlm_workspace": (i32, [i32, i32, i32, vp, vp, vp, i32, i32, i32, szp]),
        "ftlm_run": (i32, [i32, i32, i32, vp, vp, vp, i32, i32, u64, vp, i32, vp, vp, dp, vp, vp,
                           vp, i32, vp, sz, vp]),
        "arnoldi_workspace": (i32, [vp, i32, szp]),
        "arnoldi_run": (i32, [vp, i32, vp, vp, vp, vp, u64, i32, vp, sz, dp, ip, dp, i32, vp]),
        "projection_workspace": (i32, [vp, i32, szp]),
        "projection_run": (i32, [vp, i32, vp, vp, vp, vp, u64, i32, ctypes.c_double, vp, sz, dp, vp, vp]),
        "sym_eigenvalues": (i32, [i32, dp, dp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(rc: int, allow_positive: bool = True) -> int:
    if rc < 0 or (rc > 0 and not allow_positive):
        msg = load().hm_last_error().decode(errors="replace")
        raise HMError(rc, msg)
    return rc
