"""GPU: momentum blocks k = 0 and k = pi of ring sectors (basis_build_momentum) against the
oracle's dense blocks (momentum vectors projected from the sector product), Marshall's sign
rule, the Majumdar-Ghosh point at N = 32 in both blocks, and the calls that refuse such a
basis or a bond list that is not translation invariant."""
import numpy as np
import pytest

import oracle
from paper_0706_3293_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0706_3293_gb300 import build
    build.build()
    from paper_0706_3293_gb300 import api
    return api


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


CASES = [(4, 1, 0, 0), (4, 1, 0, 2), (8, 1, 0, 4), (9, 1, 1, 0), (10, 1, 2, 5), (12, 1, 0, 0),
         (6, 2, 0, 3), (7, 2, 2, 0), (5, 3, 1, 0), (14, 1, 0, 7)]


@pytest.mark.parametrize("N,S2,two_m,k", CASES, ids=lambda v: str(v))
def test_momentum_matvec_vs_oracle(hm, N, S2, two_m, k):
    """y = H_k x against the oracle's dense block, FP64 (1e-12) and FP32 (1e-5); the
    basis size equals the oracle's count of momentum states."""
    inst = W.small_ring(N, -1.0, -0.35, two_s=S2, two_m=two_m)
    b = hm.Basis(N, S2, two_m, momentum=k)
    ob = oracle.Basis(N, S2, oracle.sector_A(N, S2, two_m))
    Hk = oracle.momentum_hamiltonian(ob, oracle.Bonds(inst.u, inst.v, inst.J), k != 0)
    assert b.dim == Hk.shape[0]
    bl = hm.bonds_of(inst)
    assert hm.matvec_kernel_name(b, bl) == "k_mom_matvec"
    x = np.random.default_rng(N + k).standard_normal(b.dim)
    y = hm.matvec(b, bl, torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, Hk @ x) <= 1e-12
    x32 = x.astype(np.float32)
    y32 = hm.matvec(b, bl, torch.from_numpy(x32).cuda()).cpu().numpy().astype(np.float64)
    assert rel(y32, Hk @ x32.astype(np.float64)) <= 1e-5


@pytest.mark.parametrize("N,S2,two_m,k", [(12, 1, 0, 0), (12, 1, 0, 6), (8, 2, 0, 4)], ids=lambda v: str(v))
def test_momentum_lanczos_and_arnoldi(hm, N, S2, two_m, k):
    """Lanczos (FP64 and FP32) and Arnoldi on a momentum basis reach the lowest eigenvalue
    of the oracle's dense block (1e-10; FP32 1e-6)."""
    inst = W.small_ring(N, -1.0, -0.3, two_s=S2, two_m=two_m)
    b = hm.Basis(N, S2, two_m, momentum=k)
    ob = oracle.Basis(N, S2, oracle.sector_A(N, S2, two_m))
    e_ref = np.linalg.eigvalsh(oracle.momentum_hamiltonian(ob, oracle.Bonds(inst.u, inst.v, inst.J), k != 0))[0]
    bl = hm.bonds_of(inst)
    steps = min(120, b.dim)
    run = hm.LanczosRun(b, bl, 5, seed=3)
    assert run.kernel_name() == "k_mom_matvec"
    run.close()
    r64 = hm.lanczos_run(b, bl, steps, seed=3, n_ritz=1)
    assert abs(r64.ritz[0] - e_ref) <= 1e-10 * abs(e_ref)
    r32 = hm.lanczos_run(b, bl, steps, seed=3, n_ritz=1, dtype=torch.float32)
    assert abs(r32.ritz[0] - e_ref) <= 1e-6 * abs(e_ref)
    ar = hm.arnoldi_run(b, bl, min(60, b.dim), seed=3, n_ritz=1)
    assert abs(ar.ritz[0] - e_ref) <= 1e-10 * abs(e_ref)


@pytest.mark.parametrize("N", [16, 18, 20])
def test_momentum_marshall_rule_and_sector_e0(hm, N):
    """Nearest-neighbour antiferromagnetic rings: the ground state has momentum 0 for even
    N/2 and pi for odd N/2 (Marshall's sign rule), and that block's E0 is the sector's
    (Lanczos on the full sector, 1e-10)."""
    inst = W.small_ring(N, -1.0, None, two_m=0)
    bl = hm.bonds_of(inst)
    e = [hm.lanczos_run(hm.Basis(N, 1, 0, momentum=k), bl, 150, seed=1, n_ritz=1).ritz[0] for k in (0, N // 2)]
    e_sec = hm.lanczos_run(hm.Basis(N, 1, 0), bl, 150, seed=1, n_ritz=1).ritz[0]
    gs = 1 if (N // 2) % 2 else 0
    assert e[gs] < e[1 - gs] - 1e-6
    assert abs(e[gs] - e_sec) <= 1e-10 * abs(e_sec)


def test_momentum_full_size_majumdar_ghosh(hm):
    """N = 32, J2 = J1/2, M = 0 (the bench ring at its Majumdar-Ghosh point): the two dimer
    coverings combine into one state of momentum 0 and one of momentum pi, so both blocks
    have E0 = -3N/8 = -12 exactly.  About 18.8 million states per block."""
    inst = W.j1j2_ring32()
    bl = hm.bonds_of(inst)
    for k in (0, 16):
        b = hm.Basis(32, 1, 0, momentum=k)
        assert 18_700_000 < b.dim < 18_900_000
        res = hm.lanczos_run(b, bl, 150, seed=inst.seed, n_ritz=1)
        assert abs(res.ritz[0] - (-12.0)) <= 1e-9 * 12.0, (k, res.ritz[0])
        del b


def test_momentum_rejections(hm):
    """A bond list that is not translation invariant, a bad k, and the calls that do not
    apply to a momentum basis are refused."""
    from paper_0706_3293_gb300._capi import HMError
    inst = W.small_ring(10, -1.0, -0.3)
    b = hm.Basis(10, 1, 0, momentum=0)
    J = np.array(inst.J, dtype=np.float64)
    J[3] = -0.9
    bad = hm.BondList.make(inst.u, inst.v, J)
    x = torch.zeros(b.dim, dtype=torch.float64, device="cuda")
    with pytest.raises(HMError):
        hm.matvec(b, bad, x)
    with pytest.raises(HMError):
        hm.Basis(10, 1, 0, momentum=3)
    with pytest.raises(HMError):
        hm.Basis(9, 1, 1, momentum=4)
    bl = hm.bonds_of(inst)
    with pytest.raises(HMError):
        hm.e0_grad(b, bl, 20)
    with pytest.raises(HMError):
        hm.bond_corr(b, bl, x, x)


@pytest.mark.parametrize("N,S2,two_m,k", [(8, 1, 0, 0), (8, 1, 0, 4), (7, 2, 2, 0), (10, 1, 2, 5)], ids=lambda v: str(v))
def test_momentum_count_nnz(hm, N, S2, two_m, k):
    """count_nnz on a momentum basis: one term per representative plus every allowed
    exchange whose target orbit has a basis state, counted here from the oracle's codec."""
    inst = W.small_ring(N, -1.0, -0.35, two_s=S2, two_m=two_m)
    ob = oracle.Basis(N, S2, oracle.sector_A(N, S2, two_m))
    kpi = k != 0

    def orbit(d):
        words = [oracle.packed_word(np.roll(d, m), S2) for m in range(N)]
        p = next(m for m in range(1, N + 1) if m == N or words[m] == words[0])
        return words, p

    want = 0
    for i in range(ob.dim):
        d = ob.decode(i)
        words, p = orbit(d)
        if words[0] != min(words) or (kpi and p % 2):
            continue
        want += 1
        for u, v in zip(inst.u, inst.v):
            a, c = min(u, v), max(u, v)
            for da in (-1, 1):
                t = d.copy()
                t[a] += da
                t[c] -= da
                if min(t[a], t[c]) < 0 or max(t[a], t[c]) > S2:
                    continue
                _, p2 = orbit(t)
                want += 0 if (kpi and p2 % 2) else 1
    b = hm.Basis(N, S2, two_m, momentum=k)
    assert hm.count_nnz(b, hm.bonds_of(inst)) == want
