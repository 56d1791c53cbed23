"""GPU parity of sector_ground_energies (the lowest energy of every magnetisation sector)
against the oracle: the same FP64 Lanczos on the same start vector per sector, dense
diagonalisation of the small sectors, and closed forms (the fully polarised sector, the
spin-flip symmetry E0(M) = E0(-M) of an isotropic model at zero field)."""
import math

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


def test_sector_energies_ring14(hm):
    """N = 14 J1-J2 ring (J2 = -0.3), 120 steps, seed 9: every sector against the oracle's
    Lanczos from the same start vector (and its run length), sectors up to 1001 states
    against the eigenvalues of their dense matrix."""
    inst = W.small_ring(14, -1.0, -0.3)
    seed, steps = 9, 120
    res = hm.sector_ground_energies(14, 1, hm.bonds_of(inst), steps, seed=seed)
    ob = oracle.Bonds(inst.u, inst.v, inst.J)
    assert list(res.two_m) == list(range(14, -15, -2))
    for A in range(15):
        b = oracle.Basis(14, 1, A)
        v0 = oracle.start_uniform(oracle.stream_seed(seed, A, 0), b.dim)
        al, be = b.lanczos(ob, v0, steps)
        if b.dim > steps:   # no exhausted Krylov space: both sides run every step
            assert res.steps_done[A] == len(al) == steps, (A, res.steps_done[A], len(al))
        ref = oracle.tridiag_lowest(al, be, 1)[0]
        assert abs(res.e0[A] - ref) <= 1e-10 * max(1.0, abs(ref)), (A, res.e0[A], ref)
        if b.dim <= 1001:
            Hd = np.column_stack([b.matvec(ob, np.eye(b.dim)[i]) for i in range(b.dim)])
            ev = np.linalg.eigvalsh(Hd)
            assert abs(res.e0[A] - ev[0]) <= 1e-9 * max(1.0, abs(ev[0])), (A, res.e0[A], ev[0])
    # fully polarised sector: every bond parallel, E = -sum_b J_b / 4
    assert abs(res.e0[0] + sum(inst.J) / 4.0) < 1e-12
    # spin flip: E0(M) = E0(-M)
    np.testing.assert_allclose(res.e0, res.e0[::-1], rtol=0, atol=1e-9)
    # in a field h along z the Zeeman term -h sum s^z commutes with H(J) and shifts sector M
    # by -h M: zero field gives a singlet ground state (M = 0), a strong field full polarisation
    def field_magnetisation(h):
        return res.two_m[int(np.argmin(res.e0 - h * res.two_m / 2.0))] / 2.0
    assert field_magnetisation(0.0) == 0.0
    assert field_magnetisation(10.0) == 7.0


def test_sector_energies_s1_dense(hm):
    """s = 1, N = 6, random bonds: all 13 sectors against dense eigenvalues."""
    rng = np.random.default_rng(21)
    u = [0, 1, 2, 3, 4, 5, 0, 2]
    v = [1, 2, 3, 4, 5, 0, 3, 5]
    J = list(rng.uniform(-1.5, -0.5, len(u)))
    bl = hm.BondList.make(u, v, J)
    res = hm.sector_ground_energies(6, 2, bl, 200, seed=3)
    ob = oracle.Bonds(u, v, J)
    for A in range(13):
        ev = np.linalg.eigvalsh(oracle.dense_hamiltonian_sector(6, 2, A, ob))
        assert abs(res.e0[A] - ev[0]) <= 1e-9 * max(1.0, abs(ev[0])), (A, res.e0[A], ev[0])
    np.testing.assert_allclose(res.e0, res.e0[::-1], rtol=0, atol=1e-9)


def test_sector_energies_fp32(hm):
    """FP32 Lanczos vectors: the sector energies of the N = 14 ring within 1e-6 of FP64."""
    inst = W.small_ring(14, -1.0, -0.3)
    r64 = hm.sector_ground_energies(14, 1, hm.bonds_of(inst), 120, seed=9)
    r32 = hm.sector_ground_energies(14, 1, hm.bonds_of(inst), 120, seed=9, dtype=torch.float32)
    np.testing.assert_allclose(r32.e0, r64.e0, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("N,steps", [(16, 90), (24, 100)])
def test_sector_graph_equals_separate_runs(hm, N, steps):
    """The one-graph driver runs each sector on a branch of its own with the same kernels and
    start vector (stream seed(seed, A 2^20)) as a separate lanczos_run of that sector, so
    every sector's lowest Ritz value and step count agree bit for bit; the graph is timed
    against the separate runs."""
    import time
    inst = W.small_ring(N, -1.0, -0.5)
    bl = hm.bonds_of(inst)
    seed = 1234
    hm.sector_ground_energies(N, 1, bl, steps, seed=seed)            # plans and kernels ready
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = hm.sector_ground_energies(N, 1, bl, steps, seed=seed)
    t_graph = time.perf_counter() - t0
    t_sep = 0.0
    for A in range(N + 1):
        b = hm.Basis(N, 1, N - 2 * A)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = hm.lanczos_run(b, bl, steps, seed=oracle.stream_seed(seed, A, 0), n_ritz=1)
        t_sep += time.perf_counter() - t0
        assert res.steps_done[A] == r.steps_done, A
        assert res.e0[A] == r.ritz[0], (A, res.e0[A], r.ritz[0])
    print(f"N={N}: {N + 1} sectors x {steps} steps: one graph {t_graph * 1e3:.1f} ms, "
          f"separate runs {t_sep * 1e3:.1f} ms")
