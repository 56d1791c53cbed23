"""CPU oracle for the sector Lanczos method -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct restatement of Schnack, Hage and Schmidt,
"Optimized implementation of the Lanczos method for magnetic systems"
(arXiv:0706.3293).  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` may import it.  It shares no code with the CUDA library in
``paper_0706_3293_gb300``; both sides meet only in the seeded input generators of
``paper_0706_3293_gb300.workloads`` (which hold none of the method's arithmetic) and in
SplitMix64, which each side implements on its own from the published definition.

Two layers:

* ``hm_oracle.c`` (plain C, openMP over rows like the paper, Sec. 4): the D(N, A) table
  (Eq. E-3-c), decode (Sec. 3.1), encode (Sec. 3.2), successor (Sec. 3.1), the row
  matvec (Eq. E-4-b) of the Heisenberg model (Eq. E-2-1), bond correlations, the plain
  Lanczos recurrence and a Sturm bisection for the tridiagonal matrix.
* this module: ctypes bindings plus pure-Python/numpy brute force for tiny systems
  (stored sorted basis and binary search, Sec. 3.1 / Sec. 1; dense H built from
  Kronecker products of spin matrices), the ground-state gradient, the
  finite-temperature Lanczos estimator, the Arnoldi and projection iterations the
  paper's summary ports the product to, and the momentum blocks of a ring.  Library primitives used as single steps:
  ``numpy.linalg.eigh``/``eigvalsh`` and ``scipy.linalg.eigh_tridiagonal``.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py`` against
closed forms, worked examples of the paper, brute force, or invariants; none is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

# breakdown threshold of the Lanczos recurrence (relative to the largest |alpha|, beta)
LANCZOS_TOL = 1e-12
# finite-temperature runs: breakdown threshold of the Lanczos runs (sectors small enough to
# exhaust their Krylov space are diagonalised exactly, see ftlm_sector)
FTLM_TOL = 1e-5


def build(force: bool = False) -> str:
    """Compile hm_oracle.c into liboracle.so next to it (gcc, -O2, openMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        c_p, i64, i32, f64p = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        L.orc_basis_new.restype = c_p
        L.orc_basis_new.argtypes = [i32, i32, i32]
        L.orc_basis_free.argtypes = [c_p]
        L.orc_basis_dim.restype = i64
        L.orc_basis_dim.argtypes = [c_p]
        L.orc_table.restype = i64
        L.orc_table.argtypes = [c_p, i32, i32]
        L.orc_decode.restype = i32
        L.orc_decode.argtypes = [c_p, i64, c_p]
        L.orc_encode.restype = i64
        L.orc_encode.argtypes = [c_p, c_p]
        L.orc_successor.restype = i32
        L.orc_successor.argtypes = [i32, i32, c_p]
        L.orc_matvec.restype = i32
        L.orc_matvec.argtypes = [c_p, i32, c_p, c_p, c_p, f64p, f64p]
        L.orc_matvec_rows.restype = i32
        L.orc_matvec_rows.argtypes = [c_p, i32, c_p, c_p, c_p, f64p, f64p, i64, i64]
        L.orc_count_nnz.restype = i64
        L.orc_count_nnz.argtypes = [c_p, i32, c_p, c_p, i64, i64]
        L.orc_bond_corr.restype = i32
        L.orc_bond_corr.argtypes = [c_p, i32, c_p, c_p, f64p, f64p, f64p]
        L.orc_lanczos.restype = i32
        L.orc_lanczos.argtypes = [c_p, i32, c_p, c_p, c_p, f64p, i32, ctypes.c_double,
                                  f64p, f64p, f64p, f64p]
        L.orc_tridiag_lowest.argtypes = [i32, f64p, f64p, i32, f64p]
        L.orc_splitmix.restype = ctypes.c_uint64
        L.orc_splitmix.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.orc_start_uniform.argtypes = [ctypes.c_uint64, i64, f64p]
        L.orc_start_pm1.argtypes = [ctypes.c_uint64, i64, f64p]
        L.orc_stream_seed.restype = ctypes.c_uint64
        L.orc_stream_seed.argtypes = [ctypes.c_uint64, i32, i32]
        L.orc_num_threads.restype = i32
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return lib().orc_num_threads()


def sector_A(n_sites: int, two_s: int, two_m: int) -> int:
    """A = N s - M (Sec. 3); two_s = 2s, two_m = 2M must make N*2s - 2M even."""
    t = n_sites * two_s - two_m
    if t % 2 or t < 0 or t > 2 * n_sites * two_s:
        raise ValueError("M is not a magnetic quantum number of this system")
    return t // 2


class Bonds:
    """A bond list (u, v, J): the terms -J s_u.s_v of Eq. (E-2-1), each listed once."""

    def __init__(self, u: Sequence[int], v: Sequence[int], J: Sequence[float]):
        self.u = np.ascontiguousarray(u, dtype=np.int32)
        self.v = np.ascontiguousarray(v, dtype=np.int32)
        self.J = np.ascontiguousarray(J, dtype=np.float64)
        assert self.u.shape == self.v.shape == self.J.shape

    def __len__(self):
        return int(self.u.shape[0])


class Basis:
    """One sector H(M) of N spins s with the paper's D-table coding (Sec. 3)."""

    def __init__(self, n_sites: int, two_s: int, A: int):
        self.N, self.S2, self.A = n_sites, two_s, A
        self._h = lib().orc_basis_new(n_sites, two_s, A)
        if not self._h:
            raise ValueError("invalid basis or table overflow")
        self.dim = int(lib().orc_basis_dim(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_basis_free(h)
            self._h = None

    def D(self, k: int, a: int) -> int:
        return int(lib().orc_table(self._h, k, a))

    def decode(self, i: int) -> np.ndarray:
        d = np.zeros(self.N, dtype=np.int32)
        if lib().orc_decode(self._h, int(i), _ptr(d)) != 0:
            raise IndexError(i)
        return d

    def encode(self, digits: Sequence[int]) -> int:
        d = np.ascontiguousarray(digits, dtype=np.int32)
        assert d.shape == (self.N,)
        return int(lib().orc_encode(self._h, _ptr(d)))

    def matvec(self, bonds: Bonds, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.dim, dtype=np.float64)
        rc = lib().orc_matvec(self._h, len(bonds), _ptr(bonds.u), _ptr(bonds.v), _ptr(bonds.J),
                              _ptr(x), _ptr(y))
        if rc:
            raise ValueError("bad bond list")
        return y

    def matvec_rows(self, bonds: Bonds, x: np.ndarray, r0: int, r1: int) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(r1 - r0, dtype=np.float64)
        rc = lib().orc_matvec_rows(self._h, len(bonds), _ptr(bonds.u), _ptr(bonds.v),
                                   _ptr(bonds.J), _ptr(x), _ptr(y), r0, r1)
        if rc:
            raise ValueError("bad bond list or row range")
        return y

    def count_nnz(self, bonds: Bonds, r0: int = 0, r1: int | None = None) -> int:
        r1 = self.dim if r1 is None else r1
        return int(lib().orc_count_nnz(self._h, len(bonds), _ptr(bonds.u), _ptr(bonds.v), r0, r1))

    def bond_corr(self, bonds: Bonds, g: np.ndarray, x: np.ndarray) -> np.ndarray:
        g = np.ascontiguousarray(g, dtype=np.float64)
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.empty(len(bonds), dtype=np.float64)
        rc = lib().orc_bond_corr(self._h, len(bonds), _ptr(bonds.u), _ptr(bonds.v), _ptr(g),
                                 _ptr(x), _ptr(out))
        if rc:
            raise ValueError("bad bond list")
        return out

    def lanczos(self, bonds: Bonds, v0: np.ndarray, steps: int, tol: float = LANCZOS_TOL,
                coef: np.ndarray | None = None):
        """Plain Lanczos; returns (alpha, beta) of the steps done, and psi if coef given."""
        v0 = np.ascontiguousarray(v0, dtype=np.float64)
        al = np.zeros(steps)
        be = np.zeros(steps)
        psi = None
        cptr = None
        if coef is not None:
            coef = np.ascontiguousarray(np.pad(coef, (0, steps - len(coef))), dtype=np.float64)
            psi = np.empty(self.dim)
            cptr = _ptr(coef)
        done = lib().orc_lanczos(self._h, len(bonds), _ptr(bonds.u), _ptr(bonds.v), _ptr(bonds.J),
                                 _ptr(v0), steps, tol, _ptr(al), _ptr(be), cptr,
                                 _ptr(psi) if psi is not None else None)
        if done < 1:
            raise ValueError("lanczos failed")
        if coef is not None:
            return al[:done], be[:done], psi
        return al[:done], be[:done]


def successor(digits: Sequence[int], two_s: int):
    """Sec. 3.1 successor; returns the next digits or None for the last state."""
    d = np.ascontiguousarray(digits, dtype=np.int32).copy()
    ok = lib().orc_successor(len(d), two_s, _ptr(d))
    return d if ok else None


def tridiag_lowest(alpha: np.ndarray, beta: np.ndarray, k: int) -> np.ndarray:
    """k lowest eigenvalues of T(alpha, beta[:m-1]) by Sturm bisection."""
    al = np.ascontiguousarray(alpha, dtype=np.float64)
    m = len(al)
    be = np.ascontiguousarray(beta[: max(m - 1, 0)], dtype=np.float64)
    if be.size == 0:
        be = np.zeros(1)
    out = np.zeros(min(k, m))
    lib().orc_tridiag_lowest(m, _ptr(al), _ptr(be), len(out), _ptr(out))
    return out


def splitmix(seed: int, t: int) -> int:
    return int(lib().orc_splitmix(seed & (2**64 - 1), t))


def start_uniform(seed: int, n: int) -> np.ndarray:
    out = np.empty(n)
    lib().orc_start_uniform(seed & (2**64 - 1), n, _ptr(out))
    return out


def start_pm1(seed: int, n: int) -> np.ndarray:
    out = np.empty(n)
    lib().orc_start_pm1(seed & (2**64 - 1), n, _ptr(out))
    return out


def stream_seed(seed: int, A: int, r: int) -> int:
    return int(lib().orc_stream_seed(seed & (2**64 - 1), A, r))


# ----------------------------------------------------------------------------------------
# Brute force for tiny systems: independent of the D-table coding.
# ----------------------------------------------------------------------------------------

def full_basis_sorted(n_sites: int, two_s: int, A: int) -> list[tuple]:
    """The sector states in the paper's lexicographic order, by the "stored basis"
    route of Sec. 3.1: run through the full product basis (Eq. E-3-a: a_1 varies
    fastest, i.e. the natural number with base 2s+1 and a_N most significant) and keep
    the states with digit sum A."""
    base = two_s + 1
    out = []
    for code in range(base ** n_sites):
        d, c = [], code
        for _ in range(n_sites):
            d.append(c % base)
            c //= base
        if sum(d) == A:
            out.append(tuple(d))
    return out


def spin_matrices(two_s: int):
    """(sz, s+, s-) in the basis |a = 0..2s> with m = s - a (textbook matrices)."""
    s = two_s / 2.0
    n = two_s + 1
    m = np.array([s - a for a in range(n)])
    sz = np.diag(m)
    sp = np.zeros((n, n))
    for a in range(1, n):          # s+ |m> = sqrt(s(s+1) - m(m+1)) |m+1>; m+1 <-> a-1
        mm = m[a]
        sp[a - 1, a] = math.sqrt(s * (s + 1) - mm * (mm + 1))
    return sz, sp, sp.T.copy()


def dense_hamiltonian_full(n_sites: int, two_s: int, bonds: Bonds) -> np.ndarray:
    """H = -sum_b J_b s_u.s_v on the full product space from Kronecker products.
    Basis index of |a_1..a_N> = sum_k a_k (2s+1)^(k-1) (Eq. E-3-a)."""
    sz, sp, sm = spin_matrices(two_s)
    n = two_s + 1
    eye = np.eye(n)

    def site_op(op, k):
        # a_1 varies fastest -> it is the last factor of the Kronecker product
        mats = [eye] * n_sites
        mats[k] = op
        out = np.array([[1.0]])
        for q in reversed(range(n_sites)):
            out = np.kron(out, mats[q])
        return out

    dimf = n ** n_sites
    H = np.zeros((dimf, dimf))
    for u, v, J in zip(bonds.u, bonds.v, bonds.J):
        ss = (site_op(sz, u) @ site_op(sz, v)
              + 0.5 * (site_op(sp, u) @ site_op(sm, v) + site_op(sm, u) @ site_op(sp, v)))
        H -= J * ss
    return H


def dense_hamiltonian_sector(n_sites: int, two_s: int, A: int, bonds: Bonds) -> np.ndarray:
    """The block of dense_hamiltonian_full on the sorted sector states."""
    Hf = dense_hamiltonian_full(n_sites, two_s, bonds)
    base = two_s + 1
    idx = [sum(d[k] * base ** k for k in range(n_sites))
           for d in full_basis_sorted(n_sites, two_s, A)]
    return Hf[np.ix_(idx, idx)]


# ----------------------------------------------------------------------------------------
# Ground state, its gradient, and the finite-temperature Lanczos estimator
# ----------------------------------------------------------------------------------------

def converged_length(al: np.ndarray, be: np.ndarray, tol: float = 1e-10) -> int:
    """Shortest leading T_k whose lowest Ritz pair has converged: the residual norm of a
    Ritz pair of T_k is beta_k |s_k| (s_k the last component of its normalised
    eigenvector); take the first k with beta_k |s_k| <= tol * max(1, |theta|), else m.
    Stopping there keeps ghost copies of the ground state (which appear after
    convergence without re-orthogonalisation) out of T."""
    from scipy.linalg import eigh_tridiagonal
    m = len(al)
    for k in range(1, m + 1):
        if k == 1:
            th, s = al[0], 1.0
        else:
            w, c = eigh_tridiagonal(al[:k], be[: k - 1], select="i", select_range=(0, 0))
            th, s = w[0], c[k - 1, 0]
        if be[k - 1] * abs(s) <= tol * max(1.0, abs(th)):
            return k
    return m


def flip_matvec(basis: Basis, bonds: Bonds, x: np.ndarray, parity: int) -> np.ndarray:
    """H on the spin-flip parity subspace of an s = 1/2 sector with M = 0 (N even).

    The flip a_p -> 1 - a_p of every digit maps the sector onto itself and commutes with
    Eq. E-2-1.  Representatives of the pairs {w, flip(w)} are the states whose digit at
    position N - 1 is 0, i.e. the first half of the indices; flip reverses the order of the
    sector, index(flip(w)) = dim - 1 - index(w).  A parity-p vector x on the representatives
    is the full vector [x, p reversed(x)], and its image is the first half of H applied to it."""
    n = basis.dim
    assert basis.S2 == 1 and 2 * basis.A == basis.N and n % 2 == 0 and parity in (1, -1)
    x = np.asarray(x, dtype=np.float64)
    assert x.shape == (n // 2,)
    full = np.concatenate([x, parity * x[::-1]])
    return basis.matvec(bonds, full)[: n // 2]


def ground_state(basis: Basis, bonds: Bonds, v0: np.ndarray, steps: int):
    """Lanczos E0 and psi0: a first pass gives T, cut at the converged length (see
    converged_length); a library eigensolver gives its lowest eigenvector c, a second pass
    accumulates psi0 = sum_j c_j v_j (normalised)."""
    from scipy.linalg import eigh_tridiagonal
    al, be = basis.lanczos(bonds, v0, steps)
    m = converged_length(al, be)
    al, be = al[:m], be[:m]
    if m == 1:
        w, c = np.array([al[0]]), np.ones((1, 1))
    else:
        w, c = eigh_tridiagonal(al, be[: m - 1])
    al2, be2, psi = basis.lanczos(bonds, v0, m, coef=c[:, 0])
    psi = psi / np.linalg.norm(psi)
    return float(tridiag_lowest(al, be, 1)[0]), psi, (al, be)


def e0_grad(basis: Basis, bonds: Bonds, v0: np.ndarray, steps: int):
    """dE0/dJ_b = -<psi0| s_u.s_v |psi0> (Hellmann-Feynman on Eq. E-2-1)."""
    e0, psi, _ = ground_state(basis, bonds, v0, steps)
    return e0, -basis.bond_corr(bonds, psi, psi)


# ----------------------------------------------------------------------------------------
# Translation symmetry of a ring: the momentum blocks k = 0 and k = pi of a sector.  The
# paper names symmetries as a further reduction of H(M) without constructing them; this
# is the textbook projection onto the real characters of the cyclic group of the ring.
# ----------------------------------------------------------------------------------------

def packed_word(digits: Sequence[int], two_s: int) -> int:
    """The digits packed site by site, 1, 2 or 4 bits per digit (2s = 1, 2..3, 4..7), site u
    at bits u*b .. u*b + b - 1: the order that picks an orbit's representative."""
    b = 1 if two_s == 1 else (2 if two_s <= 3 else 4)
    return sum(int(a) << (u * b) for u, a in enumerate(digits))


def momentum_vectors(basis: Basis, k_pi: bool) -> np.ndarray:
    """Columns = the momentum basis as sector vectors: for every orbit of the translation T
    (the digit of site u moves to site u + 1 mod N) whose period p has chi(p) = 1 (any p for
    k = 0, even p for k = pi), |r^> = p^(-1/2) sum_{m<p} chi(m) T^m |r>, chi(m) = 1 or
    (-1)^m, r the orbit member with the smallest packed word; ordered by the sector index
    of r."""
    N = basis.N
    cols = []
    for i in range(basis.dim):
        d = basis.decode(i)
        orbit = [np.roll(d, m) for m in range(N)]
        words = [packed_word(o, basis.S2) for o in orbit]
        if words[0] != min(words):
            continue                                   # i is not its orbit's representative
        p = next(m for m in range(1, N + 1) if m == N or words[m] == words[0])
        if k_pi and p % 2:
            continue
        v = np.zeros(basis.dim)
        for m in range(p):
            v[basis.encode(orbit[m])] += (-1.0) ** m if k_pi else 1.0
        cols.append(v / math.sqrt(p))
    return np.column_stack(cols) if cols else np.zeros((basis.dim, 0))


def momentum_hamiltonian(basis: Basis, bonds: Bonds, k_pi: bool) -> np.ndarray:
    """<r'^| H |r^> for the momentum basis of momentum_vectors (dense, small N): the sector
    product applied to each basis vector, projected back."""
    B = momentum_vectors(basis, k_pi)
    HB = np.column_stack([basis.matvec(bonds, B[:, c]) for c in range(B.shape[1])])
    return B.T @ HB


# ----------------------------------------------------------------------------------------
# Arnoldi and projection methods on the same product.  The paper's closing summary names
# them as methods its product ports to but gives no steps; these are the textbook
# iterations (Arnoldi 1951 with classical Gram-Schmidt applied twice; the power method on
# sigma - H), written plainly on Basis.matvec.
# ----------------------------------------------------------------------------------------

ARNOLDI_TOL = 1e-12


def arnoldi(basis: Basis, bonds: Bonds, v0: np.ndarray, steps: int, tol: float = ARNOLDI_TOL):
    """Arnoldi with full re-orthogonalisation: v_1 = v0/|v0|; per step w = H v_j, then
    twice h = V^T w, w -= V h, H[:j, j] += h; H[j+1, j] = |w|; stop when |w| <= tol times
    the largest |H| entry so far.  Returns (H of shape [m+1, m], m)."""
    V = [np.asarray(v0, dtype=np.float64) / np.linalg.norm(v0)]
    H = np.zeros((steps + 1, steps))
    scale = 0.0
    m = 0
    for j in range(steps):
        w = basis.matvec(bonds, V[j])
        for _ in range(2):
            h = np.array([np.dot(V[i], w) for i in range(j + 1)])
            for i in range(j + 1):
                w = w - h[i] * V[i]
            H[: j + 1, j] += h
        beta = np.linalg.norm(w)
        scale = max(scale, np.abs(H[: j + 1, j]).max())
        H[j + 1, j] = beta
        m = j + 1
        if beta <= tol * scale:
            break
        scale = max(scale, beta)
        V.append(w / beta)
    return H[: m + 1, :m], m


def arnoldi_ritz(H: np.ndarray, m: int, k: int) -> np.ndarray:
    """k lowest eigenvalues of the symmetric part of H[:m, :m] (library eigensolver)."""
    A = H[:m, :m]
    return np.linalg.eigvalsh(0.5 * (A + A.T))[:k]


def projection(basis: Basis, bonds: Bonds, v0: np.ndarray, steps: int, sigma: float) -> np.ndarray:
    """Shifted power method: psi_0 = v0/|v0|; E_k = psi_k . H psi_k;
    psi_{k+1} = (sigma psi_k - H psi_k) / |sigma psi_k - H psi_k|.  Returns E_0..E_{steps-1}."""
    psi = np.asarray(v0, dtype=np.float64) / np.linalg.norm(v0)
    E = np.zeros(steps)
    for k in range(steps):
        y = basis.matvec(bonds, psi)
        E[k] = np.dot(psi, y)
        nxt = sigma * psi - y
        psi = nxt / np.linalg.norm(nxt)
    return E


def projection_default_sigma(two_s: int, J: Sequence[float]) -> float:
    """sum_b |J_b| s (s + 1): |s_u.s_v| <= s (s + 1), so this bounds the spectrum of H."""
    s = two_s / 2.0
    return float(sum(abs(j) for j in J) * s * (s + 1.0))


def ftlm_sector(basis: Basis, bonds: Bonds, seed: int, R: int, steps: int, tol: float = FTLM_TOL):
    """Per start vector r of one sector: Ritz values theta_j and weights tau_j (squared
    first components of T's eigenvectors), the start vector being the +-1 vector of
    stream (seed, A, r).  A run stops at beta_j <= tol max(|alpha|, beta) (tol defaults
    to FTLM_TOL, the threshold the FP32 device runs use).
    A sector of dimension <= steps (and <= 512) would exhaust its Krylov space; it is
    diagonalised exactly instead: theta_k = E_k, tau_k = <r/|r| | psi_k>^2, the limit of
    the Lanczos quadrature (alpha, beta are then returned empty)."""
    from scipy.linalg import eigh_tridiagonal
    res = []
    exact = basis.dim <= steps and basis.dim <= 512
    if exact:
        Hd = np.column_stack([basis.matvec(bonds, np.eye(basis.dim)[i]) for i in range(basis.dim)])
        E, V = np.linalg.eigh(Hd)
    for r in range(R):
        v0 = start_pm1(stream_seed(seed, basis.A, r), basis.dim)
        if exact:
            o = V.T @ (v0 / np.sqrt(basis.dim))
            res.append((E.copy(), o * o, np.zeros(0), np.zeros(0)))
            continue
        al, be = basis.lanczos(bonds, v0, steps, tol=tol)
        m = len(al)
        if m == 1:
            th, c = np.array([al[0]]), np.ones((1, 1))
        else:
            th, c = eigh_tridiagonal(al, be[: m - 1])
        res.append((th, c[0, :] ** 2, al, be))
    return res


def ftlm_thermo(per_sector: list, temps: Sequence[float]):
    """Finite-temperature Lanczos (Jaklic-Prelovsek) estimator over sectors:
    Z(T) = sum_A (D_A/R) sum_r sum_j tau_rj exp(-theta_rj/T),
    E(T) = [same with theta_rj inside] / Z.  per_sector is a list of (D_A, results) with
    results a list of (theta, tau, ...) per start vector.  Energies are shifted by the
    lowest Ritz value for the exponentials; returns (Z, E, e_ref) with the true
    Z = Z * exp(-e_ref / T)."""
    e_ref = min(float(np.min(th)) for (_, lst) in per_sector for (th, tau, *_) in lst)
    Z = np.zeros(len(temps))
    EZ = np.zeros(len(temps))
    for (dim, lst) in per_sector:
        R = len(lst)
        for (th, tau, *_) in lst:
            for k, T in enumerate(temps):
                wgt = tau * np.exp(-(th - e_ref) / T)
                Z[k] += dim / R * float(np.sum(wgt))
                EZ[k] += dim / R * float(np.sum(wgt * th))
    return Z, EZ / Z, e_ref
