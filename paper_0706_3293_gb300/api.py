"""Python binding of libhm.so: the same entry points as include/hm.h.

PyTorch provides device memory (tensors, workspaces) and the current CUDA stream; every
step of the computation runs in the library's CUDA kernels.  Nothing here falls back to
a CPU implementation: a missing library raises ImportError, a failing call HMError.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _capi
from ._capi import HM_F32, HM_F64, HMError, check

_DT = {torch.float64: HM_F64, torch.float32: HM_F32}


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _vp(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class BondList:
    """Host bond arrays (u, v, J): the terms -J s_u.s_v of Eq. (E-2-1)."""
    u: np.ndarray
    v: np.ndarray
    J: np.ndarray

    @staticmethod
    def make(u, v, J) -> "BondList":
        return BondList(np.ascontiguousarray(u, dtype=np.int32),
                        np.ascontiguousarray(v, dtype=np.int32),
                        np.ascontiguousarray(J, dtype=np.float64))

    def __len__(self):
        return int(self.u.shape[0])

    def args(self):
        return (len(self), self.u.ctypes.data_as(ctypes.c_void_p),
                self.v.ctypes.data_as(ctypes.c_void_p), self.J.ctypes.data_as(ctypes.c_void_p))


def bonds_of(inst) -> BondList:
    return BondList.make(inst.u, inst.v, inst.J)


def basis_dim_query(n_sites: int, two_s: int, two_m: int) -> int:
    d = ctypes.c_int64()
    check(_capi.load().basis_dim_query(n_sites, two_s, two_m, ctypes.byref(d)))
    return d.value


def bonds_check(n_sites: int, bonds: BondList) -> None:
    check(_capi.load().bonds_check(n_sites, *bonds.args()))


class Basis:
    """hm_basis: the tables of one sector H(M) on the current device (Sec. 3)."""

    def __init__(self, n_sites: int, two_s: int, two_m: int, parity: int = 0, momentum: int | None = None):
        """parity = +1 / -1: the spin-flip block of the s = 1/2 sector M = 0 (basis_build_flip);
        momentum = 0 or n_sites // 2: the momentum block of a ring (basis_build_momentum)."""
        self.n_sites, self.two_s, self.two_m, self.parity = n_sites, two_s, two_m, parity
        self.momentum = momentum
        h = ctypes.c_void_p()
        if parity:
            assert two_s == 1 and two_m == 0, "the spin-flip basis is the s = 1/2 sector M = 0"
            check(_capi.load().basis_build_flip(n_sites, parity, ctypes.byref(h)))
        elif momentum is not None:
            check(_capi.load().basis_build_momentum(n_sites, two_s, two_m, momentum, ctypes.byref(h)))
        else:
            check(_capi.load().basis_build(n_sites, two_s, two_m, ctypes.byref(h)))
        self._h = h
        d = ctypes.c_int64()
        check(_capi.load().basis_dim(self._h, ctypes.byref(d)))
        self.dim = d.value
        self.A = (n_sites * two_s - two_m) // 2

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _capi.load().basis_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def encode(self, states: torch.Tensor) -> torch.Tensor:
        assert states.dtype == torch.int64 and states.is_cuda
        st = states.contiguous()
        out = torch.empty_like(st)
        check(_capi.load().basis_encode(self._h, _vp(st), _vp(out), st.numel(), _stream()))
        return out

    def decode(self, idx: torch.Tensor) -> torch.Tensor:
        assert idx.dtype == torch.int64 and idx.is_cuda
        ix = idx.contiguous()
        out = torch.empty_like(ix)
        check(_capi.load().basis_decode(self._h, _vp(ix), _vp(out), ix.numel(), _stream()))
        return out


def matvec(basis: Basis, bonds: BondList, x: torch.Tensor, out: torch.Tensor | None = None):
    """y = H x (Eq. E-4-b) for x of shape [dim] or [dim, nvec], float64 or float32."""
    assert x.is_cuda and x.dtype in _DT and x.shape[0] == basis.dim
    x = x.contiguous()
    nvec = 1 if x.dim() == 1 else x.shape[1]
    y = torch.empty_like(x) if out is None else out
    check(_capi.load().matvec(basis.handle, *bonds.args(), _vp(x), _vp(y), _DT[x.dtype], nvec,
                              _stream()))
    return y


def matvec_kernel_name(basis: Basis, bonds: BondList, dtype=torch.float64, nvec: int = 1) -> str:
    """The kernel matvec launches for these arguments (matvec_kernel_name)."""
    buf = ctypes.create_string_buffer(64)
    check(_capi.load().matvec_kernel_name(basis.handle, *bonds.args(), _DT[dtype], nvec, buf, 64))
    return buf.value.decode()


def count_nnz(basis: Basis, bonds: BondList, device="cuda") -> int:
    """Non-zero elements of H(M): one diagonal per row plus every allowed exchange."""
    out = torch.zeros(1, dtype=torch.int64, device=device)
    check(_capi.load().count_nnz(basis.handle, *bonds.args()[:3], _vp(out), _stream()))
    return int(out.item())


def bond_corr(basis: Basis, bonds: BondList, g: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """out[b] = sum_i g_i [(s_u.s_v) x]_i (device float64[n_bonds])."""
    assert g.dtype == x.dtype and g.shape == x.shape == (basis.dim,)
    L = _capi.load()
    n = ctypes.c_size_t()
    check(L.bond_corr_workspace(basis.handle, len(bonds), ctypes.byref(n)))
    work = torch.empty(max(n.value, 8), dtype=torch.uint8, device=x.device)
    out = torch.empty(max(len(bonds), 1), dtype=torch.float64, device=x.device)
    check(L.bond_corr(basis.handle, len(bonds), bonds.args()[1], bonds.args()[2], _vp(g.contiguous()),
                      _vp(x.contiguous()), _vp(out), _DT[x.dtype], _vp(work), n.value, _stream()))
    return out[: len(bonds)]


def start_vector(basis: Basis, seed: int, kind: int = 0, dtype=torch.float64, device="cuda"):
    x = torch.empty(basis.dim, dtype=dtype, device=device)
    check(_capi.load().start_vector(basis.handle, seed & (2**64 - 1), kind, _vp(x), _DT[dtype],
                                    _stream()))
    return x


def _workspace(nbytes: int, device) -> torch.Tensor:
    # torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


@dataclass
class LanczosResult:
    alpha: np.ndarray
    beta: np.ndarray
    steps_done: int
    ritz: np.ndarray
    status: int


def lanczos_workspace(basis: Basis, dtype=torch.float64, steps: int = 100) -> int:
    n = ctypes.c_size_t()
    check(_capi.load().lanczos_workspace(basis.handle, _DT[dtype], steps, ctypes.byref(n)))
    return n.value


def lanczos_run(basis: Basis, bonds: BondList, steps: int, v0: torch.Tensor | None = None,
                seed: int = 0, dtype=torch.float64, n_ritz: int = 5, work: torch.Tensor | None = None,
                device="cuda") -> LanczosResult:
    """A whole Lanczos run (one graph launch) and the n_ritz lowest Ritz values."""
    L = _capi.load()
    nbytes = lanczos_workspace(basis, dtype, steps)
    if work is None or work.numel() < nbytes:
        work = _workspace(nbytes, device)
    al = np.zeros(steps)
    be = np.zeros(steps)
    rz = np.zeros(max(n_ritz, 1))
    done = ctypes.c_int()
    if v0 is not None:
        assert v0.dtype == dtype and v0.shape == (basis.dim,)
        v0 = v0.contiguous()
    rc = check(L.lanczos_run(basis.handle, *bonds.args(), _vp(v0) if v0 is not None else None,
                             seed & (2**64 - 1), steps, _DT[dtype], _vp(work), work.numel(),
                             al.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             be.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(done),
                             rz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n_ritz, _stream()))
    m = done.value
    return LanczosResult(al[:m], be[:m], m, rz[:n_ritz], rc)


class LanczosRun:
    """Step-wise Lanczos (lanczos_init / lanczos_step / lanczos_read)."""

    def __init__(self, basis: Basis, bonds: BondList, max_steps: int, v0=None, seed: int = 0,
                 dtype=torch.float64, work: torch.Tensor | None = None, device="cuda"):
        L = _capi.load()
        nbytes = lanczos_workspace(basis, dtype, max_steps)
        self.work = work if work is not None and work.numel() >= nbytes else _workspace(nbytes, device)
        self.basis, self.bonds, self.max_steps = basis, bonds, max_steps
        h = ctypes.c_void_p()
        if v0 is not None:
            v0 = v0.contiguous()
        check(L.lanczos_init(basis.handle, *bonds.args(), _vp(v0) if v0 is not None else None,
                             seed & (2**64 - 1), _DT[dtype], max_steps, _vp(self.work),
                             self.work.numel(), _stream(), ctypes.byref(h)))
        self._h = h

    def step(self, n: int = 1):
        L = _capi.load()
        for _ in range(n):
            check(L.lanczos_step(self._h, _stream()))

    def substep(self, phase: int):
        check(_capi.load().lanczos_substep(self._h, phase, _stream()))

    def read(self):
        al = np.zeros(self.max_steps)
        be = np.zeros(self.max_steps)
        done = ctypes.c_int()
        rc = check(_capi.load().lanczos_read(self._h, al.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             be.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             ctypes.byref(done), _stream()))
        m = done.value
        return al[:m], be[:m], rc

    def kernel_name(self) -> str:
        """The kernel that forms H q in each step (lanczos_kernel_name)."""
        buf = ctypes.create_string_buffer(64)
        check(_capi.load().lanczos_kernel_name(self._h, buf, 64))
        return buf.value.decode()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _capi.load().lanczos_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class SectorEnergies:
    """Lowest energy of every magnetisation sector (sector_ground_energies)."""
    two_m: np.ndarray           # 2M of each sector, 2sN down to -2sN
    e0: np.ndarray
    steps_done: np.ndarray


def sector_ground_energies(n_sites: int, two_s: int, bonds: BondList, steps: int, seed: int = 0,
                           dtype=torch.float64, work: torch.Tensor | None = None,
                           device="cuda") -> SectorEnergies:
    L = _capi.load()
    nb = ctypes.c_size_t()
    check(L.sector_ground_energies_workspace(n_sites, two_s, steps, _DT[dtype], ctypes.byref(nb)))
    work = work if work is not None and work.numel() >= nb.value else _workspace(nb.value, device)
    nsec = two_s * n_sites + 1
    e0 = np.zeros(nsec)
    done = np.zeros(nsec, dtype=np.int32)
    check(L.sector_ground_energies(n_sites, two_s, *bonds.args(), steps, seed & (2**64 - 1), _DT[dtype],
                                   _vp(work), work.numel(), e0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   done.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _stream()))
    two_m = two_s * n_sites - 2 * np.arange(nsec)
    return SectorEnergies(two_m, e0, done)


def e0_grad(basis: Basis, bonds: BondList, steps: int, v0: torch.Tensor | None = None,
            seed: int = 0, want_psi: bool = False, device="cuda"):
    """Returns (E0, dE0/dJ as numpy, psi0 or None, status)."""
    L = _capi.load()
    n = ctypes.c_size_t()
    check(L.e0_grad_workspace(basis.handle, len(bonds), steps, ctypes.byref(n)))
    work = _workspace(n.value, device)
    e0 = ctypes.c_double()
    g = np.zeros(max(len(bonds), 1))
    psi = torch.empty(basis.dim, dtype=torch.float64, device=device) if want_psi else None
    if v0 is not None:
        assert v0.dtype == torch.float64
        v0 = v0.contiguous()
    rc = check(L.e0_grad(basis.handle, *bonds.args(), _vp(v0) if v0 is not None else None,
                         seed & (2**64 - 1), steps, _vp(work), work.numel(), ctypes.byref(e0),
                         g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                         _vp(psi) if psi is not None else None, _stream()))
    return e0.value, g[: len(bonds)], psi, rc


def ground_state_correlations(basis: Basis, bonds: BondList, pairs_u, pairs_v, steps: int,
                              v0: torch.Tensor | None = None, seed: int = 0, device="cuda"):
    """Ground energy and the correlations <psi0| s_u.s_v |psi0> of any site pairs (u, v) in the
    ground state of H(bonds) on the basis sector: psi0 (normalised) from e0_grad, then the
    bond-correlation kernel on (psi0, psi0).  Returns (E0, correlations as numpy, status)."""
    e0, _, psi, rc = e0_grad(basis, bonds, steps, v0=v0, seed=seed, want_psi=True, device=device)
    pairs = BondList.make(pairs_u, pairs_v, np.zeros(len(pairs_u)))
    check(_capi.load().bonds_check(basis.n_sites, *pairs.args()))
    corr = bond_corr(basis, pairs, psi, psi).cpu().numpy()
    return e0, corr, rc


@dataclass
class FTLMResult:
    Z: np.ndarray          # partition function / e^{-e_ref / T}
    E: np.ndarray          # energy expectation
    e_ref: float
    theta: np.ndarray      # [sector, 32, steps] Ritz values
    tau: np.ndarray        # [sector, 32, steps] weights
    mlen: np.ndarray       # [sector, 32] Krylov lengths
    vt: int                # vectors per lane used by the product


def ftlm_run(n_sites: int, bonds: BondList, R: int, steps: int, seed: int, temps, vt: int = 0,
             device="cuda") -> FTLMResult:
    """Finite-temperature Lanczos over all sectors of an s = 1/2 system (one graph)."""
    L = _capi.load()
    temps = np.ascontiguousarray(temps, dtype=np.float64)
    n_t = int(temps.shape[0])
    n = ctypes.c_size_t()
    check(L.ftlm_workspace(n_sites, 1, *bonds.args(), R, steps, n_t, ctypes.byref(n)))
    work = _workspace(n.value, device)
    nsec = n_sites + 1
    Z = np.zeros(max(n_t, 1))
    E = np.zeros(max(n_t, 1))
    eref = ctypes.c_double()
    theta = np.zeros(nsec * 32 * steps)
    tau = np.zeros(nsec * 32 * steps)
    mlen = np.zeros(nsec * 32, dtype=np.int32)
    dp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = check(L.ftlm_run(n_sites, 1, *bonds.args(), R, steps, seed & (2**64 - 1), dp(temps), n_t,
                          dp(Z), dp(E), ctypes.byref(eref), dp(theta), dp(tau), dp(mlen), vt,
                          _vp(work), work.numel(), _stream()))
    return FTLMResult(Z[:n_t], E[:n_t], eref.value, theta.reshape(nsec, 32, steps),
                      tau.reshape(nsec, 32, steps), mlen.reshape(nsec, 32), rc)


# ---- Arnoldi and projection methods on the same product -----------------------------------

@dataclass
class ArnoldiResult:
    H: np.ndarray          # [steps_done + 1, steps_done] Hessenberg matrix
    steps: int
    ritz: np.ndarray       # lowest eigenvalues of the symmetric part of H[:steps, :steps]
    rc: int


def arnoldi_run(basis: Basis, bonds: BondList, steps: int, v0: torch.Tensor | None = None,
                seed: int = 0, n_ritz: int = 5, device="cuda") -> ArnoldiResult:
    """Arnoldi with full re-orthogonalisation (arnoldi_run), FP64 vectors."""
    L = _capi.load()
    n = ctypes.c_size_t()
    check(L.arnoldi_workspace(basis.handle, steps, ctypes.byref(n)))
    work = _workspace(n.value, device)
    hess = np.zeros((steps, steps + 1))          # column major: row j = column j of H
    rz = np.zeros(max(n_ritz, 1))
    done = ctypes.c_int()
    if v0 is not None:
        assert v0.dtype == torch.float64 and v0.shape == (basis.dim,)
        v0 = v0.contiguous()
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    rc = check(L.arnoldi_run(basis.handle, *bonds.args(), _vp(v0) if v0 is not None else None,
                             seed & (2**64 - 1), steps, _vp(work), work.numel(), dp(hess),
                             ctypes.byref(done), dp(rz), n_ritz, _stream()))
    m = done.value
    return ArnoldiResult(hess.T[: m + 1, :m].copy(), m, rz[:n_ritz], rc)


def projection_run(basis: Basis, bonds: BondList, steps: int, sigma: float = 0.0,
                   v0: torch.Tensor | None = None, seed: int = 0, want_psi: bool = False,
                   device="cuda"):
    """Shifted power (projection) method (projection_run): energies E_0..E_{steps-1} and,
    if asked, the last iterate psi_steps (device)."""
    L = _capi.load()
    n = ctypes.c_size_t()
    check(L.projection_workspace(basis.handle, steps, ctypes.byref(n)))
    work = _workspace(n.value, device)
    E = np.zeros(steps)
    psi = torch.empty(basis.dim, dtype=torch.float64, device=device) if want_psi else None
    if v0 is not None:
        assert v0.dtype == torch.float64 and v0.shape == (basis.dim,)
        v0 = v0.contiguous()
    check(L.projection_run(basis.handle, *bonds.args(), _vp(v0) if v0 is not None else None,
                           seed & (2**64 - 1), steps, float(sigma), _vp(work), work.numel(),
                           E.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           _vp(psi) if psi is not None else None, _stream()))
    return (E, psi) if want_psi else E


def sym_eigenvalues(a: np.ndarray) -> np.ndarray:
    """Eigenvalues of the symmetric part of a small dense host matrix (the library's Jacobi
    solver that arnoldi_run applies to its Hessenberg matrix; no GPU involved)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    n = a.shape[0]
    ev = np.zeros(n)
    check(_capi.load().sym_eigenvalues(n, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       ev.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return ev
