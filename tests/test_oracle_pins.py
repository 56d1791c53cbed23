"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values printed in the
paper's worked examples (tests/golden/paper_worked_examples.json), closed forms,
brute-force enumeration on tiny systems, a dense Hamiltonian built from Kronecker
products of textbook spin matrices, an independent stored-basis sparse construction,
and invariants.  No GPU is involved.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import Basis, Bonds
from paper_0706_3293_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_worked_examples.json")


def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def bonds_of(inst):
    return Bonds(inst.u, inst.v, inst.J)


# ---- D(N, A): Eq. (E-3-c) -------------------------------------------------------------

@pytest.mark.parametrize("N,S2", [(1, 1), (5, 1), (9, 2), (6, 3), (4, 4), (12, 2), (32, 1)])
def test_D_boundary_values(orc, N, S2):
    """Sec. 3: D(1, 0..2s) = 1, D(N, 0) = 1, D(N, 1) = N, zero outside 0..2Ns."""
    b = Basis(N, S2, 0)
    for a in range(S2 + 1):
        assert b.D(1, a) == 1
    for k in range(1, N + 1):
        assert b.D(k, 0) == 1
        assert b.D(k, 1) == k
        assert b.D(k, -1) == 0
        assert b.D(k, S2 * k + 1) == 0


@pytest.mark.parametrize("N,S2", [(7, 1), (10, 2), (6, 3), (5, 5), (20, 2), (32, 1)])
def test_D_generating_function_and_sum(orc, N, S2):
    """D(N, A) is the coefficient of x^A in (1 + x + ... + x^{2s})^N (counting digit
    strings with a fixed sum), computed here by exact integer polynomial powers; the
    coefficients add up to dim H = (2s+1)^N (Sec. 2)."""
    poly = [1]
    for _ in range(N):
        new = [0] * (len(poly) + S2)
        for i, c in enumerate(poly):
            for n in range(S2 + 1):
                new[i + n] += c
        poly = new
    b = Basis(N, S2, 0)
    assert [b.D(N, a) for a in range(S2 * N + 1)] == poly
    assert sum(poly) == (S2 + 1) ** N


def test_D_known_dimensions(orc):
    """Binomials for s = 1/2 and the central trinomial coefficient for s = 1."""
    def trinomial(n):
        return sum(math.comb(n, 2 * k) * math.comb(2 * k, k) for k in range(n // 2 + 1))

    assert Basis(16, 1, 8).dim == math.comb(16, 8) == 12870
    assert Basis(24, 1, 12).dim == math.comb(24, 12) == 2704156
    assert Basis(32, 1, 16).dim == math.comb(32, 16) == 601080390
    assert Basis(20, 2, 20).dim == trinomial(20) == 377379369
    assert Basis(12, 2, 12).dim == trinomial(12) == 73789
    g = golden()["fig_fa_vector_length"]
    assert Basis(g["n_sites"], g["two_s"], g["A"]).dim == g["dim"]


def test_D_table_overflow_rejected(orc):
    with pytest.raises(ValueError):
        Basis(64, 4, 128)   # 5^64 states overflow int64


# ---- decode / encode / successor: Sec. 3.1 and 3.2 --------------------------------------

def test_encode_worked_example(orc):
    g = golden()["encode"]
    b = Basis(g["n_sites"], g["two_s"], g["A"])
    expected = sum(b.D(k, a) for (k, a) in g["terms"])   # plus one in the paper's 1-based count
    assert expected == 41
    assert b.encode(g["state"]) == expected
    assert list(b.decode(expected)) == g["state"]


def test_successor_worked_example(orc):
    g = golden()["successor"]
    nxt = oracle.successor(g["state"], g["two_s"])
    assert list(nxt) == g["successor"]
    b = Basis(g["n_sites"], g["two_s"], g["A"])
    assert b.encode(g["successor"]) == b.encode(g["state"]) + 1


@pytest.mark.parametrize("N,S2", [(1, 1), (2, 1), (5, 1), (7, 1), (4, 2), (6, 2), (3, 3),
                                  (5, 3), (3, 4)])
def test_codec_bruteforce(orc, N, S2):
    """decode/encode against the stored sorted basis (all (2s+1)^N product states
    filtered by the digit sum), for every sector."""
    for A in range(S2 * N + 1):
        states = oracle.full_basis_sorted(N, S2, A)
        b = Basis(N, S2, A)
        assert b.dim == len(states)
        for i, st in enumerate(states):
            assert tuple(b.decode(i)) == st
            assert b.encode(st) == i


@pytest.mark.parametrize("N,S2,A", [(8, 1, 4), (6, 2, 5), (5, 3, 7), (9, 2, 2)])
def test_successor_walks_the_order(orc, N, S2, A):
    b = Basis(N, S2, A)
    st = b.decode(0)
    # lowest state: boxes filled from the left (Sec. 3.1)
    left = []
    rest = A
    for _ in range(N):
        t = min(rest, S2)
        left.append(t)
        rest -= t
    assert list(st) == left
    for i in range(1, b.dim):
        st = oracle.successor(st, S2)
        assert st is not None
        assert b.encode(st) == i
    assert oracle.successor(st, S2) is None


def test_codec_rejects_bad_input(orc):
    b = Basis(6, 1, 3)
    with pytest.raises(IndexError):
        b.decode(b.dim)
    assert b.encode([1, 1, 1, 1, 0, 0]) == -1     # wrong digit sum
    assert b.encode([2, 1, 0, 0, 0, 0]) == -1     # digit > 2s


# ---- the matvec: Eqs. (E-2-1), (E-4-b) ----------------------------------------------------

def _random_bonds(rng, N, nb, allow_dup=True):
    u, v = [], []
    while len(u) < nb:
        a, c = rng.integers(0, N, 2)
        if a == c:
            continue
        u.append(int(a)); v.append(int(c))
    J = rng.uniform(-1.5, 1.5, nb)
    return Bonds(u, v, J)


@pytest.mark.parametrize("N,S2", [(4, 1), (6, 1), (7, 1), (4, 2), (5, 2), (3, 3), (4, 3),
                                  (3, 4)])
def test_matvec_vs_dense_kronecker(orc, N, S2):
    """Row matvec equals the sector block of H = -sum J s_u.s_v built from Kronecker
    products of the textbook spin matrices (covers signs, ladder factors, diagonal,
    bonds listed as u > v and repeated bonds)."""
    rng = np.random.default_rng(100 * N + S2)
    bonds = _random_bonds(rng, N, 2 * N)
    for A in range(S2 * N + 1):
        H = oracle.dense_hamiltonian_sector(N, S2, A, bonds)
        b = Basis(N, S2, A)
        x = rng.standard_normal(b.dim)
        y = b.matvec(bonds, x)
        np.testing.assert_allclose(y, H @ x, rtol=1e-13, atol=1e-13)


def _stored_basis_sparse(N, A, bonds):
    """Independent s = 1/2 sparse H: sorted integer codes of the sector states and
    binary search for the targets (the stored-basis / search route of Sec. 1, 3.1)."""
    import scipy.sparse as sp
    codes = np.array(sorted(c for c in range(1 << N) if bin(c).count("1") == A), dtype=np.int64)
    n = len(codes)
    rows, cols, vals = [np.arange(n)], [np.arange(n)], [np.zeros(n)]
    diag = np.zeros(n)
    for u, v, J in zip(bonds.u, bonds.v, bonds.J):
        bu = (codes >> u) & 1
        bv = (codes >> v) & 1
        # a = 1 means m = -1/2: s^z_u s^z_v = +1/4 if equal, -1/4 if different
        diag += -J * np.where(bu == bv, 0.25, -0.25)
        hop = bu != bv
        tgt = codes[hop] ^ ((1 << int(u)) | (1 << int(v)))
        j = np.searchsorted(codes, tgt)
        rows.append(np.nonzero(hop)[0]); cols.append(j); vals.append(np.full(len(j), -0.5 * J))
    vals[0] = diag
    H = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    return H


@pytest.mark.parametrize("inst", [W.ring16(), W.small_ring(12, -1.0, -0.5),
                                  W.small_ring(14, -1.0, -0.3)], ids=lambda i: i.name)
def test_matvec_vs_stored_basis_s12(orc, inst):
    b = Basis(inst.n_sites, 1, inst.A)
    bonds = bonds_of(inst)
    H = _stored_basis_sparse(inst.n_sites, inst.A, bonds)
    x = np.random.default_rng(5).uniform(-1, 1, b.dim)
    np.testing.assert_allclose(b.matvec(bonds, x), H @ x, rtol=1e-13, atol=1e-13)


def test_matvec_symmetry(orc):
    """<x|Hy> = <Hx|y> on an s = 1 random graph sector."""
    inst = W.s1_random_graph(10, 21)
    b = Basis(10, 2, inst.A)
    bonds = bonds_of(inst)
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal(b.dim), rng.standard_normal(b.dim)
    lhs = x @ b.matvec(bonds, y)
    rhs = b.matvec(bonds, x) @ y
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)


def test_nnz_closed_form(orc):
    """s = 1/2, M = 0 ring: every bond connects C(N-2, N/2-1) states of each of the two
    orientations, so nnz = dim + 2 * n_bonds * C(N-2, N/2-1)."""
    inst = W.ring16()
    b = Basis(16, 1, 8)
    nnz = b.count_nnz(bonds_of(inst))
    assert nnz == 12870 + 2 * 16 * math.comb(14, 7) == 122694
    inst = W.small_ring(20, -1.0, -0.5)
    b = Basis(20, 1, 10)
    assert b.count_nnz(bonds_of(inst)) == b.dim + 2 * 40 * math.comb(18, 9)


def test_trace_zero_over_all_sectors(orc):
    """Tr H over the full space is 0 (s_u.s_v is traceless for u != v): the diagonal
    elements of all sectors add up to zero."""
    inst = W.s1_random_graph(8, 5)
    bonds = bonds_of(inst)
    tot = 0.0
    for A in range(0, 2 * 8 + 1):
        b = Basis(8, 2, A)
        for i in range(b.dim):
            e = np.zeros(b.dim); e[i] = 1.0
            tot += b.matvec(bonds, e)[i]
    assert abs(tot) < 1e-10


# ---- energies ---------------------------------------------------------------------------

def _dense_sector_spectrum(N, S2, A, bonds):
    b = Basis(N, S2, A)
    H = np.column_stack([b.matvec(bonds, np.eye(b.dim)[i]) for i in range(b.dim)])
    return np.linalg.eigvalsh(H)


def test_polarised_and_one_magnon(orc):
    """Fully polarised sector: E = -s^2 sum J.  One-magnon sector of the s = 1/2 ring:
    E(k) = -J N/4 + J (1 - cos k), k = 2 pi q / N."""
    N, J = 8, 0.7
    inst = W.small_ring(N, J)
    bonds = bonds_of(inst)
    assert abs(_dense_sector_spectrum(N, 1, 0, bonds)[0] - (-0.25 * N * J)) < 1e-13
    ev = _dense_sector_spectrum(N, 1, 1, bonds)
    ref = np.sort([-J * N / 4 + J * (1 - math.cos(2 * math.pi * q / N)) for q in range(N)])
    np.testing.assert_allclose(ev, ref, atol=1e-12)
    inst2 = W.small_ring(5, 1.3, two_s=2, two_m=10)
    assert abs(_dense_sector_spectrum(5, 2, 0, bonds_of(inst2))[0] - (-1.0 * 5 * 1.3)) < 1e-12


def test_small_ring_ground_energies(orc):
    """s = 1/2 antiferromagnetic rings: E0(N=4) = -2|J| (each bond listed once),
    E0(N=6) = -(1 + sqrt(13)/2)."""
    e4 = _dense_sector_spectrum(4, 1, 2, bonds_of(W.small_ring(4, -1.0)))[0]
    assert abs(e4 - (-2.0)) < 1e-13
    e6 = _dense_sector_spectrum(6, 1, 3, bonds_of(W.small_ring(6, -1.0)))[0]
    assert abs(e6 - (-(1 + math.sqrt(13) / 2))) < 1e-13


@pytest.mark.parametrize("N", [8, 10, 12])
def test_majumdar_ghosh(orc, N):
    """J2 = J1/2 ring (J1 = -1): E0 = -3N/8, doubly degenerate (two dimer singlets)."""
    ev = _dense_sector_spectrum(N, 1, N // 2, bonds_of(W.small_ring(N, -1.0, -0.5)))
    assert abs(ev[0] + 3 * N / 8) < 1e-12
    assert abs(ev[1] + 3 * N / 8) < 1e-12


def test_complete_graph_spectrum(orc):
    """All pairs with J = -1: H = (S_tot^2 - N s(s+1))/2, eigenvalues (S(S+1) -
    N s(s+1))/2 for every total spin S >= |M| that occurs."""
    N, S2 = 5, 2
    pairs = [(a, c) for a in range(N) for c in range(a + 1, N)]
    bonds = Bonds([p[0] for p in pairs], [p[1] for p in pairs], [-1.0] * len(pairs))
    ev = _dense_sector_spectrum(N, S2, 5, bonds)     # M = 0
    ref = {(S * (S + 1) - N * 2) / 2 for S in range(0, 6)}
    got = {round(e, 9) for e in ev}
    assert got == {round(r, 9) for r in ref}


# ---- Lanczos and the tridiagonal eigensolver --------------------------------------------

def test_tridiag_bisection_vs_dense(orc):
    rng = np.random.default_rng(3)
    for m in [1, 2, 5, 40, 100]:
        al = rng.standard_normal(m)
        be = rng.uniform(0.1, 1.0, m)
        T = np.diag(al) + np.diag(be[: m - 1], 1) + np.diag(be[: m - 1], -1)
        ref = np.linalg.eigvalsh(T)[:5]
        got = oracle.tridiag_lowest(al, be, 5)
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * max(1, np.abs(ref).max()))


def test_lanczos_ground_energy_small(orc):
    inst = W.s1_random_graph(8, 9)
    b = Basis(8, 2, 8)
    bonds = bonds_of(inst)
    ev = _dense_sector_spectrum(8, 2, 8, bonds)
    v0 = oracle.start_uniform(77, b.dim)
    al, be = b.lanczos(bonds, v0, 120)
    e0 = oracle.tridiag_lowest(al, be, 1)[0]
    assert abs(e0 - ev[0]) < 1e-10 * abs(ev[0])


def test_lanczos_ring16_config(orc):
    """The 16-site ring (M = 0, 100 steps, uniform start seed 1001): E0 against an
    independent sparse diagonalisation of the stored-basis Hamiltonian."""
    from scipy.sparse.linalg import eigsh
    inst = W.ring16()
    bonds = bonds_of(inst)
    H = _stored_basis_sparse(16, 8, bonds)
    ref = np.sort(eigsh(H, k=6, which="SA", tol=1e-14)[0])
    b = Basis(16, 1, 8)
    v0 = oracle.start_uniform(inst.seed, b.dim)
    al, be = b.lanczos(bonds, v0, inst.steps)
    assert len(al) == 100
    e0 = oracle.tridiag_lowest(al, be, 5)
    assert abs(e0[0] - ref[0]) < 1e-10 * abs(ref[0])
    assert abs(ref[0] - (-7.142296360617)) < 1e-11


def test_lanczos_breakdown(orc):
    """A dim-1 sector stops after one step with alpha = E; a sector smaller than the
    step count stops when the Krylov space is exhausted."""
    inst = W.small_ring(6, -1.0)
    bonds = bonds_of(inst)
    b = Basis(6, 1, 0)
    al, be = b.lanczos(bonds, np.ones(1), 10)
    assert len(al) == 1 and abs(al[0] - (-0.25 * 6 * -1.0)) < 1e-15
    b = Basis(6, 1, 1)
    al, be = b.lanczos(bonds, oracle.start_uniform(3, b.dim), 20)
    assert len(al) <= b.dim
    ev = _dense_sector_spectrum(6, 1, 1, bonds)
    assert abs(oracle.tridiag_lowest(al, be, 1)[0] - ev[0]) < 1e-12


# ---- gradients ------------------------------------------------------------------------------

def test_bond_corr_homogeneity_and_linearity(orc):
    """H is linear in J: sum_b J_b dL/dJ_b = g^T H x exactly, and a central difference in
    one coupling reproduces -out[b]."""
    inst = W.s1_random_graph(8, 11)
    bonds = bonds_of(inst)
    b = Basis(8, 2, 8)
    rng = np.random.default_rng(4)
    g, x = rng.standard_normal(b.dim), rng.standard_normal(b.dim)
    c = b.bond_corr(bonds, g, x)
    gHx = g @ b.matvec(bonds, x)
    assert abs(np.dot(bonds.J, -c) - gHx) < 1e-10 * abs(gHx)
    t, h = 3, 1e-3
    Jp, Jm = bonds.J.copy(), bonds.J.copy()
    Jp[t] += h; Jm[t] -= h
    fd = (g @ b.matvec(Bonds(bonds.u, bonds.v, Jp), x) - g @ b.matvec(Bonds(bonds.u, bonds.v, Jm), x)) / (2 * h)
    assert abs(fd - (-c[t])) < 1e-9 * (1 + abs(fd))


def test_e0_grad_finite_difference_and_sum_rules(orc):
    inst = W.small_ring(10, -1.0, -0.3)
    rng = np.random.default_rng(8)
    J = rng.uniform(-1.2, -0.8, inst.n_bonds)
    bonds = Bonds(inst.u, inst.v, J)
    b = Basis(10, 1, 5)
    v0 = oracle.start_uniform(11, b.dim)
    e0, grad = oracle.e0_grad(b, bonds, v0, 150)
    ev = _dense_sector_spectrum(10, 1, 5, bonds)
    assert abs(e0 - ev[0]) < 1e-11
    assert abs(np.dot(J, grad) - e0) < 1e-9           # Euler: E0 is homogeneous of degree 1
    h = 1e-6
    for t in [0, 7, 13]:
        Jp, Jm = J.copy(), J.copy()
        Jp[t] += h; Jm[t] -= h
        ep = _dense_sector_spectrum(10, 1, 5, Bonds(inst.u, inst.v, Jp))[0]
        em = _dense_sector_spectrum(10, 1, 5, Bonds(inst.u, inst.v, Jm))[0]
        assert abs((ep - em) / (2 * h) - grad[t]) < 1e-6


def test_singlet_and_dimer_sum_rules(orc):
    """Singlet ground state: sum over all pairs <s_u.s_v> = (0 - N s(s+1))/2; a dimer of
    two s = 1/2 spins: <s_1.s_2> = -3/4."""
    b = Basis(2, 1, 1)
    e0, grad = oracle.e0_grad(b, Bonds([0], [1], [-1.0]), np.array([1.0, 0.3]), 5)
    assert abs(-grad[0] - (-0.75)) < 1e-13
    N = 8
    inst = W.small_ring(N, -1.0, -0.2)
    b = Basis(N, 1, N // 2)
    _, psi, _ = oracle.ground_state(b, bonds_of(inst), oracle.start_uniform(5, b.dim), 80)
    pairs = [(a, c) for a in range(N) for c in range(a + 1, N)]
    allp = Bonds([p[0] for p in pairs], [p[1] for p in pairs], [1.0] * len(pairs))
    corr = b.bond_corr(allp, psi, psi)
    assert abs(corr.sum() - (-N * 0.75 / 2)) < 1e-10


# ---- finite-temperature Lanczos ---------------------------------------------------------

def test_ftlm_small_sector_exact(orc):
    """When Lanczos exhausts a sector (dim <= steps), sum_j tau_j e^{-theta_j/T} equals
    <r|e^{-H/T}|r>/<r|r> for the start vector r, and sum_j tau_j = 1."""
    from scipy.linalg import expm
    inst = W.small_ring(8, -1.0, -0.3)
    bonds = bonds_of(inst)
    for A in [1, 2, 3]:
        b = Basis(8, 1, A)
        res = oracle.ftlm_sector(b, bonds, 99, 3, 80)
        H = np.column_stack([b.matvec(bonds, np.eye(b.dim)[i]) for i in range(b.dim)])
        for r, (th, tau, *_) in enumerate(res):
            assert abs(tau.sum() - 1.0) < 1e-12
            v = oracle.start_pm1(oracle.stream_seed(99, A, r), b.dim)
            for T in [0.3, 1.0, 5.0]:
                ref = v @ expm(-H / T) @ v / (v @ v)
                assert abs(np.sum(tau * np.exp(-th / T)) - ref) < 1e-10 * ref


def test_ftlm_high_temperature_and_mirror_sectors(orc):
    """Z(T -> infinity) = (2s+1)^N; sectors A and 2Ns - A have equal spectra."""
    N = 8
    inst = W.small_ring(N, -1.0, -0.3)
    bonds = bonds_of(inst)
    per = []
    for A in range(N + 1):
        b = Basis(N, 1, A)
        per.append((b.dim, oracle.ftlm_sector(b, bonds, 5, 2, 40)))
    Z, E, eref = oracle.ftlm_thermo(per, [1e9])
    assert abs(Z[0] * math.exp(-eref / 1e9) - 2 ** N) < 1e-5
    for A in range(N // 2):
        np.testing.assert_allclose(_dense_sector_spectrum(N, 1, A, bonds),
                                   _dense_sector_spectrum(N, 1, N - A, bonds), atol=1e-12)


# ---- the seeded start vectors (SplitMix64) ----------------------------------------------

def _splitmix_py(seed, t):
    """SplitMix64 (Steele, Lea, Flood 2014) in Python integers: output t of the
    generator seeded with `seed` is mix(seed + (t+1) gamma)."""
    M = (1 << 64) - 1
    z = (seed + (t + 1) * 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def test_splitmix_reference_outputs(orc):
    """Published first outputs of SplitMix64 seeded with 0."""
    ref = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [_splitmix_py(0, t) for t in range(3)] == ref
    for seed in [0, 1, 1001, 2**63 + 5]:
        for t in [0, 1, 17, 10**9]:
            assert oracle.splitmix(seed, t) == _splitmix_py(seed, t)


def test_start_vectors(orc):
    u = oracle.start_uniform(1001, 1000)
    ref = np.array([2.0 * ((_splitmix_py(1001, t) >> 11) * 2.0**-53) - 1.0 for t in range(1000)])
    assert np.array_equal(u, ref)
    assert u.min() >= -1.0 and u.max() < 1.0
    p = oracle.start_pm1(42, 1000)
    assert set(np.unique(p)) <= {-1.0, 1.0}
    assert np.array_equal(p, np.array([-1.0 if _splitmix_py(42, t) >> 63 else 1.0 for t in range(1000)]))
    assert oracle.stream_seed(1005, 12, 3) == _splitmix_py(1005, (12 << 20) + 3)


def test_ftlm_lanczos_quadrature_large_sector(orc):
    """A sector larger than the step count runs Lanczos: the quadrature
    sum_j tau_j e^{-theta_j/T} of 40 steps matches <r|e^{-H/T}|r>/<r|r> (dense) for smooth
    f; the error of a degree-40 Gauss quadrature is far below 1e-8 at these T."""
    from scipy.linalg import expm
    inst = W.small_ring(10, -1.0, -0.3)
    bonds = bonds_of(inst)
    b = Basis(10, 1, 5)
    assert b.dim == 252
    res = oracle.ftlm_sector(b, bonds, 21, 2, 40)
    H = np.column_stack([b.matvec(bonds, np.eye(b.dim)[i]) for i in range(b.dim)])
    for r, (th, tau, al, be) in enumerate(res):
        assert len(al) == 40
        v = oracle.start_pm1(oracle.stream_seed(21, 5, r), b.dim)
        for T in [1.0, 3.0]:
            ref = v @ expm(-H / T) @ v / (v @ v)
            assert abs(np.sum(tau * np.exp(-th / T)) - ref) < 1e-8 * ref


def _ftlm_ring_sectors(N, seed, R, steps, tol=oracle.FTLM_TOL):
    inst = W.small_ring(N, -1.0, -0.3)
    bonds = bonds_of(inst)
    per = []
    for A in range(N + 1):
        b = Basis(N, 1, A)
        per.append((b.dim, oracle.ftlm_sector(b, bonds, seed, R, steps, tol=tol)))
    return inst, bonds, per


def test_ftlm_energy_is_minus_dlnZ_dbeta(orc):
    """Thermodynamics fixes E = -d ln Z / d beta (beta = 1/T) for any set of weights: on the
    same Ritz values and weights, E(T) from ftlm_thermo must equal the derivative of its
    ln Z (true units, Z e^{-e_ref/T}) taken by central differences in beta with Richardson
    extrapolation.  Weighting E by theta - e_ref, or dropping D_A/R from one of the two
    sums, fails by far more than the tolerance."""
    _, _, per = _ftlm_ring_sectors(10, 17, 3, 30)

    def lnZ(beta):
        Z, _, e_ref = oracle.ftlm_thermo(per, [1.0 / beta])
        return math.log(Z[0]) - e_ref * beta

    for T in [0.4, 1.0, 3.0, 20.0]:
        beta = 1.0 / T
        E = oracle.ftlm_thermo(per, [T])[1][0]
        h = 1e-2 * beta

        def cd(hh):
            return (lnZ(beta + hh) - lnZ(beta - hh)) / (2 * hh)
        dlnz = (4 * cd(h / 2) - cd(h)) / 3
        assert abs(E - (-dlnz)) < 1e-8 * max(1.0, abs(E)), (T, E, -dlnz)


def test_ftlm_thermo_exact_with_basis_vectors(orc):
    """With every basis vector of every sector as a start vector (R = D_A) and the exact
    per-vector quadrature (theta = the sector's eigenvalues, tau = squared components of
    its eigenvectors), the estimator is the trace: Z(T) = sum_k e^{-E_k/T} and
    E(T) = sum_k E_k e^{-E_k/T} / Z over the whole spectrum of the N = 8 ring, here from
    the dense Kronecker-product Hamiltonian of all 2^8 states."""
    N = 8
    inst = W.small_ring(N, -1.0, -0.3)
    bonds = bonds_of(inst)
    per = []
    for A in range(N + 1):
        Hs = oracle.dense_hamiltonian_sector(N, 1, A, bonds)
        ev, V = np.linalg.eigh(Hs)
        per.append((len(ev), [(ev.copy(), V[r, :] ** 2) for r in range(len(ev))]))
    spec = np.linalg.eigvalsh(oracle.dense_hamiltonian_full(N, 1, bonds))
    temps = [0.2, 0.5, 1.0, 4.0, 50.0]
    Z, E, e_ref = oracle.ftlm_thermo(per, temps)
    for k, T in enumerate(temps):
        w = np.exp(-(spec - spec[0]) / T)
        z_ref = float(np.sum(w)) * math.exp(-spec[0] / T)
        e_ref_T = float(np.sum(spec * w) / np.sum(w))
        assert abs(Z[k] * math.exp(-e_ref / T) - z_ref) < 1e-12 * z_ref, (T, Z[k], z_ref)
        assert abs(E[k] - e_ref_T) < 1e-12 * max(1.0, abs(e_ref_T)), (T, E[k], e_ref_T)


def test_ftlm_thermo_matches_dense_estimator(orc):
    """The Jaklic-Prelovsek estimator on the oracle's own start vectors (R = 3 +-1 vectors
    per sector, 30 Lanczos steps; sectors of dimension 45..252 take the Lanczos branch)
    against the same estimator formed densely with the matrix exponential:
    Z = sum_A (D_A/R) sum_r <r|e^{-H/T}|r>/<r|r>,
    E = [sum_A (D_A/R) sum_r <r|H e^{-H/T}|r>/<r|r>] / Z.
    A 30-node Gauss quadrature of e^{-H/T} is exact far below 1e-10 at these T."""
    from scipy.linalg import expm
    seed, R, steps, N = 23, 3, 30, 10
    inst, bonds, per = _ftlm_ring_sectors(N, seed, R, steps)
    temps = [0.7, 2.0, 10.0]
    Z, E, e_ref = oracle.ftlm_thermo(per, temps)
    for k, T in enumerate(temps):
        zd, ed = 0.0, 0.0
        for A in range(N + 1):
            b = Basis(N, 1, A)
            H = np.column_stack([b.matvec(bonds, np.eye(b.dim)[i]) for i in range(b.dim)])
            Ex = expm(-H / T)
            for r in range(R):
                v = oracle.start_pm1(oracle.stream_seed(seed, A, r), b.dim)
                zd += b.dim / R * (v @ Ex @ v) / (v @ v)
                ed += b.dim / R * (v @ H @ Ex @ v) / (v @ v)
        assert abs(Z[k] * math.exp(-e_ref / T) - zd) < 1e-10 * zd, (T, Z[k] * math.exp(-e_ref / T), zd)
        assert abs(E[k] - ed / zd) < 1e-10 * max(1.0, abs(ed / zd)), (T, E[k], ed / zd)


def test_ftlm_stop_threshold_leaves_quadrature_unchanged(orc):
    """The oracle stops its finite-temperature runs at beta_j <= 1e-5 max(|alpha|, beta),
    the threshold of the FP32 device runs.  On sectors larger than the step count the FP64
    runs never come near it: a 1e-12 threshold gives the same Ritz values, weights and
    thermodynamics."""
    _, _, per5 = _ftlm_ring_sectors(10, 31, 2, 30)
    _, _, per12 = _ftlm_ring_sectors(10, 31, 2, 30, tol=1e-12)
    for (d5, l5), (d12, l12) in zip(per5, per12):
        for (th5, tau5, al5, _), (th12, tau12, al12, _) in zip(l5, l12):
            assert len(al5) == len(al12)
            assert np.array_equal(th5, th12) and np.array_equal(tau5, tau12)
    temps = [0.5, 2.0]
    for a, b in zip(oracle.ftlm_thermo(per5, temps), oracle.ftlm_thermo(per12, temps)):
        np.testing.assert_array_equal(a, b)


# ---- spin-flip parity sectors (M = 0) ------------------------------------------------------

@pytest.mark.parametrize("N", [6, 8, 10])
def test_flip_reverses_the_index(orc, N):
    """Brute force: complementing every digit of a sector state at M = 0 maps index i to
    dim - 1 - i (the flip reverses the numerical order of words of weight N/2)."""
    b = Basis(N, 1, N // 2)
    for i in range(b.dim):
        d = b.decode(i)
        assert b.encode(1 - d) == b.dim - 1 - i
        assert (d[N - 1] == 0) == (i < b.dim // 2)     # representatives: first half


def _flip_dense(b, bonds, parity):
    n = b.dim // 2
    return np.stack([oracle.flip_matvec(b, bonds, np.eye(n)[:, j], parity) for j in range(n)], axis=1)


@pytest.mark.parametrize("N,j2,seed", [(8, -0.3, 1), (10, -0.5, 2), (10, 0.7, 3)])
def test_flip_sectors_split_the_spectrum(orc, N, j2, seed):
    """The two parity blocks are symmetric and their spectra together are the sector's
    spectrum (dense diagonalisation of the full M = 0 sector)."""
    inst = W.small_ring(N, -1.0, j2)
    J = np.random.default_rng(seed).uniform(-1.3, 0.6, inst.n_bonds)
    bonds = Bonds(inst.u, inst.v, J)
    b = Basis(N, 1, N // 2)
    Hp, Hm = _flip_dense(b, bonds, 1), _flip_dense(b, bonds, -1)
    np.testing.assert_allclose(Hp, Hp.T, atol=1e-13)
    np.testing.assert_allclose(Hm, Hm.T, atol=1e-13)
    full = np.linalg.eigvalsh(oracle.dense_hamiltonian_sector(N, 1, N // 2, bonds))
    both = np.sort(np.concatenate([np.linalg.eigvalsh(Hp), np.linalg.eigvalsh(Hm)]))
    np.testing.assert_allclose(both, full, rtol=0, atol=1e-10)


def test_flip_majumdar_ghosh_parity(orc):
    """N = 8 ring at J2 = J1/2 (J1 = -1): the ground states are the two dimer coverings by
    singlets, each singlet odd under the flip, so a product of N/2 = 4 singlets is even:
    E0 = -3N/8 = -3 lies in the parity +1 block, and the -1 block lies above it."""
    inst = W.small_ring(8, -1.0, -0.5)
    bonds = Bonds(inst.u, inst.v, inst.J)
    b = Basis(8, 1, 4)
    ep = np.linalg.eigvalsh(_flip_dense(b, bonds, 1))
    em = np.linalg.eigvalsh(_flip_dense(b, bonds, -1))
    assert abs(ep[0] + 3.0) < 1e-12
    assert em[0] > -3.0 + 1e-6


# ---- Arnoldi and projection iterations (the summary's other Krylov-type methods) ----------

def _kron_spectrum(N, S2, A, bonds):
    """Spectrum of the sector block of the Kronecker-product Hamiltonian (no codec)."""
    return np.linalg.eigvalsh(oracle.dense_hamiltonian_sector(N, S2, A, bonds))


@pytest.mark.parametrize("N,S2,A,seed", [(8, 1, 4, 1), (7, 1, 3, 2), (5, 2, 5, 3)])
def test_arnoldi_ritz_values_in_the_spectrum(orc, N, S2, A, seed):
    """Run to exhaustion of the Krylov space: every Ritz value is an eigenvalue of the
    Kronecker-product sector Hamiltonian (1e-10), the lowest one is E0, and H is
    tridiagonal (Hermitian H: entries above the superdiagonal vanish to rounding)."""
    rng = np.random.default_rng(seed)
    u, v = np.triu_indices(N, 1)
    keep = rng.random(len(u)) < 0.6
    bonds = Bonds(u[keep].astype(np.int32), v[keep].astype(np.int32), rng.uniform(-1.3, 0.4, keep.sum()))
    b = Basis(N, S2, A)
    H, m = oracle.arnoldi(b, bonds, oracle.start_uniform(seed, b.dim), b.dim + 5)
    assert m <= b.dim
    ev = _kron_spectrum(N, S2, A, bonds)
    ritz = oracle.arnoldi_ritz(H, m, m)
    for t in ritz:
        assert np.abs(ev - t).min() < 1e-10 * max(1.0, abs(ev).max())
    assert abs(ritz[0] - ev[0]) < 1e-10 * max(1.0, abs(ev[0]))
    scale = np.abs(H).max()
    assert np.abs(np.triu(H[:m, :m], 2)).max() < 1e-12 * scale


def test_arnoldi_equals_lanczos_early(orc):
    """Before rounding separates them, Arnoldi's diagonal and subdiagonal are the
    Lanczos alpha_j and beta_j of the C oracle's three-term recurrence (same start)."""
    inst = W.small_ring(12, -1.0, -0.4)
    bonds = bonds_of(inst)
    b = Basis(12, 1, 6)
    v0 = oracle.start_uniform(5, b.dim)
    H, m = oracle.arnoldi(b, bonds, v0, 15)
    al, be = b.lanczos(bonds, v0, 15)
    assert m == 15
    np.testing.assert_allclose(np.diag(H[:m, :m]), al, rtol=0, atol=1e-12 * np.abs(al).max())
    np.testing.assert_allclose(np.diag(H, -1), be, rtol=0, atol=1e-12 * np.abs(al).max())


def test_arnoldi_four_site_ring(orc):
    """Four-site s = 1/2 antiferromagnetic ring (J = -1): E0 = -2 |J| (closed form)."""
    inst = W.small_ring(4, -1.0)
    b = Basis(4, 1, 2)
    H, m = oracle.arnoldi(b, bonds_of(inst), oracle.start_uniform(1, b.dim), 10)
    assert abs(oracle.arnoldi_ritz(H, m, 1)[0] - (-2.0)) < 1e-13


def test_projection_monotone_and_converges(orc):
    """Power method on sigma - H with sigma >= E_max: the energies E_k never increase
    (sigma - H is positive semi-definite) and tend to E0 of the Kronecker-product
    Hamiltonian; for the four-site ring to -2 |J|."""
    inst = W.small_ring(8, -1.0, -0.3)
    bonds = bonds_of(inst)
    b = Basis(8, 1, 4)
    sigma = oracle.projection_default_sigma(1, inst.J)
    ev = _kron_spectrum(8, 1, 4, bonds)
    assert sigma >= ev[-1]
    E = oracle.projection(b, bonds, oracle.start_uniform(2, b.dim), 3000, sigma)
    assert np.all(np.diff(E) <= 1e-12)
    assert abs(E[-1] - ev[0]) < 1e-8 * abs(ev[0])
    r4 = W.small_ring(4, -1.0)
    b4 = Basis(4, 1, 2)
    E4 = oracle.projection(b4, bonds_of(r4), oracle.start_uniform(1, b4.dim), 400,
                           oracle.projection_default_sigma(1, r4.J))
    assert abs(E4[-1] - (-2.0)) < 1e-12


# ---- momentum blocks of a ring (translation symmetry) ------------------------------------

def _ring_bonds(N, j1, j2):
    inst = W.small_ring(N, j1, j2)
    return Bonds(inst.u, inst.v, inst.J)


@pytest.mark.parametrize("N,S2,two_m,k_pi", [(4, 1, 0, False), (4, 1, 0, True), (8, 1, 0, True),
                                             (9, 1, 1, False), (6, 2, 0, True), (7, 2, 2, False)])
def test_momentum_basis_invariant_and_orthonormal(orc, N, S2, two_m, k_pi):
    """The momentum vectors are orthonormal, H maps their span into itself (H commutes
    with the translation for a ring), and every eigenvalue of the block is an eigenvalue
    of the Kronecker-product sector Hamiltonian."""
    A = oracle.sector_A(N, S2, two_m)
    b = Basis(N, S2, A)
    bonds = _ring_bonds(N, -1.0, -0.35)
    B = oracle.momentum_vectors(b, k_pi)
    np.testing.assert_allclose(B.T @ B, np.eye(B.shape[1]), atol=1e-13)
    Hk = oracle.momentum_hamiltonian(b, bonds, k_pi)
    HB = np.column_stack([b.matvec(bonds, B[:, c]) for c in range(B.shape[1])])
    assert np.abs(HB - B @ Hk).max() < 1e-12
    np.testing.assert_allclose(Hk, Hk.T, atol=1e-13)
    ev = np.linalg.eigvalsh(oracle.dense_hamiltonian_sector(N, S2, A, bonds))
    for t in np.linalg.eigvalsh(Hk):
        assert np.abs(ev - t).min() < 1e-10


def test_momentum_four_site_ring_and_marshall_rule(orc):
    """Four-site s = 1/2 ring, M = 0: orbits {0011, 0110, 1100, 1001} (period 4) and
    {0101, 1010} (period 2), so k = 0 and k = pi each hold two states, and E0 = -2 |J|.
    Nearest-neighbour antiferromagnetic rings (Marshall's sign rule): the ground state has
    momentum 0 when N/2 is even and pi when N/2 is odd, strictly below the other block."""
    b = Basis(4, 1, 2)
    bonds = _ring_bonds(4, -1.0, None)
    H0 = oracle.momentum_hamiltonian(b, bonds, False)
    Hpi = oracle.momentum_hamiltonian(b, bonds, True)
    assert H0.shape == (2, 2) and Hpi.shape == (2, 2)
    assert abs(np.linalg.eigvalsh(H0)[0] - (-2.0)) < 1e-13
    for N in (4, 6, 8, 10):
        b = Basis(N, 1, N // 2)
        bonds = _ring_bonds(N, -1.0, None)
        e = [np.linalg.eigvalsh(oracle.momentum_hamiltonian(b, bonds, kp))[0] for kp in (False, True)]
        gs_pi = (N // 2) % 2 == 1
        assert (e[1] < e[0] - 1e-9) if gs_pi else (e[0] < e[1] - 1e-9)


def test_momentum_blocks_hold_the_ground_state(orc):
    """Even J1-J2 rings: the sector ground state lies in the k = 0 or the k = pi block."""
    for N in (8, 10):
        b = Basis(N, 1, N // 2)
        bonds = _ring_bonds(N, -1.0, -0.3)
        ev = np.linalg.eigvalsh(oracle.dense_hamiltonian_sector(N, 1, N // 2, bonds))
        e0 = min(np.linalg.eigvalsh(oracle.momentum_hamiltonian(b, bonds, kp))[0] for kp in (False, True))
        assert abs(e0 - ev[0]) < 1e-10
