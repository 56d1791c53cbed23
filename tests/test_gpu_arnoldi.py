"""GPU: Arnoldi with full re-orthogonalisation and the projection (shifted power) method
on the library's products (arnoldi_run, projection_run) against the oracle's plain
iterations on the same start vectors, in every product path: s = 1/2 block kernel, the
per-bond specialised kernel (random couplings), the general row kernel (s = 1)."""
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


def cases():
    ring = W.small_ring(14, -1.0, -0.4)
    rj = W.small_ring(16, -1.0, -0.4)
    J = np.random.default_rng(8).uniform(-1.2, -0.8, rj.n_bonds)
    s1 = W.s1_random_graph(8, 31)
    return {
        "ring14_block": (ring, ring.J),
        "ring16_perbond": (rj, J),
        "s1_n8_general": (s1, s1.J),
    }


@pytest.mark.parametrize("name", ["ring14_block", "ring16_perbond", "s1_n8_general"])
def test_arnoldi_vs_oracle(hm, name):
    """The first 25 columns of H to 1e-12 of the largest entry, the step count, and the
    lowest Ritz values to 1e-10 (after 60 steps, converged)."""
    inst, J = cases()[name]
    b = hm.Basis(inst.n_sites, inst.two_s, inst.two_m)
    ob = oracle.Basis(inst.n_sites, inst.two_s, inst.A)
    bl = hm.BondList.make(inst.u, inst.v, J)
    obl = oracle.Bonds(inst.u, inst.v, J)
    steps = 60
    res = hm.arnoldi_run(b, bl, steps, seed=17, n_ritz=3)
    H, m = oracle.arnoldi(ob, obl, oracle.start_uniform(17, b.dim), steps)
    assert res.steps == m
    k = min(25, m)
    scale = np.abs(H).max()
    np.testing.assert_allclose(res.H[: k + 1, :k], H[: k + 1, :k], rtol=0, atol=1e-12 * scale)
    ref = oracle.arnoldi_ritz(H, m, 3)
    np.testing.assert_allclose(res.ritz, ref, rtol=0, atol=1e-10 * abs(ref[0]))


def test_arnoldi_breakdown_and_spectrum(hm):
    """A sector smaller than the step count: the run stops when its Krylov space is
    exhausted (HM_BREAKDOWN), every Ritz value is an eigenvalue of the Kronecker-product
    sector Hamiltonian, the lowest is E0."""
    inst = W.small_ring(8, -1.0, -0.3)
    b = hm.Basis(8, 1, 2)
    res = hm.arnoldi_run(b, hm.bonds_of(inst), 80, seed=3, n_ritz=b.dim)
    assert res.rc == 1 and res.steps <= b.dim
    A = oracle.sector_A(8, 1, 2)
    ev = np.linalg.eigvalsh(oracle.dense_hamiltonian_sector(8, 1, A, oracle.Bonds(inst.u, inst.v, inst.J)))
    ritz = res.ritz[: res.steps]
    for t in ritz:
        assert np.abs(ev - t).min() < 1e-10
    assert abs(ritz[0] - ev[0]) < 1e-10


def test_arnoldi_start_vector_and_errors(hm):
    """A caller's start vector gives the same run as the seeded one it copies; a zero start
    vector and a spin-flip basis are rejected."""
    inst = W.small_ring(12, -1.0, -0.3)
    b = hm.Basis(12, 1, 0)
    bl = hm.bonds_of(inst)
    v0 = torch.from_numpy(oracle.start_uniform(5, b.dim)).cuda()
    r1 = hm.arnoldi_run(b, bl, 20, v0=v0)
    r2 = hm.arnoldi_run(b, bl, 20, seed=5)
    assert np.array_equal(r1.H, r2.H)
    from paper_0706_3293_gb300._capi import HMError
    with pytest.raises(HMError):
        hm.arnoldi_run(b, bl, 5, v0=torch.zeros(b.dim, dtype=torch.float64, device="cuda"))
    bf = hm.Basis(12, 1, 0, parity=1)
    with pytest.raises(HMError):
        hm.arnoldi_run(bf, bl, 5)


@pytest.mark.parametrize("name", ["ring14_block", "ring16_perbond", "s1_n8_general"])
def test_projection_vs_oracle(hm, name):
    """Energies of the shifted power method against the oracle's iteration (1e-11 of |E0|
    over 300 steps, default shift), monotone, and the last iterate normalised."""
    inst, J = cases()[name]
    b = hm.Basis(inst.n_sites, inst.two_s, inst.two_m)
    ob = oracle.Basis(inst.n_sites, inst.two_s, inst.A)
    bl = hm.BondList.make(inst.u, inst.v, J)
    sigma = oracle.projection_default_sigma(inst.two_s, J)
    E, psi = hm.projection_run(b, bl, 300, seed=4, want_psi=True)
    ref = oracle.projection(ob, oracle.Bonds(inst.u, inst.v, J), oracle.start_uniform(4, b.dim), 300, sigma)
    np.testing.assert_allclose(E, ref, rtol=0, atol=1e-11 * abs(ref[-1]))
    assert np.all(np.diff(E) <= 1e-12 * abs(E[0]) + 1e-14)
    assert abs(float(torch.linalg.vector_norm(psi)) - 1.0) < 1e-12


def test_projection_converges_to_lanczos_e0(hm):
    """N = 12 J1-J2 ring: after enough steps the projection energy reaches the Lanczos E0
    of the same product (1e-9)."""
    inst = W.small_ring(12, -1.0, -0.3)
    b = hm.Basis(12, 1, 0)
    bl = hm.bonds_of(inst)
    e0 = hm.lanczos_run(b, bl, 120, seed=1, n_ritz=1).ritz[0]
    E = hm.projection_run(b, bl, 6000, seed=1)
    assert abs(E[-1] - e0) < 1e-9 * abs(e0)
