"""Every workload of the scope at its stated size and tolerance, through the C ABI.

ring16 (plain method): the five lowest Ritz values of 100 FP64 steps against the oracle's.
s1_rrg20 (precision): FP32 Lanczos vectors against an FP64 run of the same start vector at
N = 20 (377,379,369 rows), |dE0/E0| <= 1e-6.
ring24_randJ (differentiation): autograd through the product and dE0/dJ at N = 24 with 48
couplings, against the oracle's whole-sector product, adjoint and ground-state gradient,
and central finite differences (h = 1e-6) of the GPU's own ground energy.
ftlm_ring24 (batching): the M = 0 sector's lowest Ritz value of the FP32 batched run against
an FP64 Lanczos run from the same +-1 start vector, |dE0/E0| <= 1e-6.
"""
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


def obonds(inst, J=None):
    return oracle.Bonds(inst.u, inst.v, inst.J if J is None else J)


def ritz_with_residuals(al, be, k):
    """The k lowest eigenvalues theta of the m x m tridiagonal (al, be[:m-1]) and the residual
    norms beta_m |s_m| of their Ritz pairs: each theta lies within its residual of an
    eigenvalue of H (be[m-1] couples T_m to the next Lanczos vector)."""
    from scipy.linalg import eigh_tridiagonal
    m = len(al)
    th, S = eigh_tridiagonal(al, be[:m - 1])
    return th[:k], np.abs(be[m - 1] * S[m - 1, :k])


def test_ring16_five_ritz_values(hm):
    """ring16, 100 steps from the uniform start vector of seed 1001.  After 100 steps the
    five lowest Ritz values hold converged eigenvalues and converging ghost copies (no
    re-orthogonalisation).  A converged value is unique: GPU and oracle agree to 1e-10.  A
    value still converging depends on the rounding history of its run (a 1e-15 change of the
    start vector moves it by up to 1e-3), so there both must lie within their residual norms
    of one another, and each within its own residual of an exact eigenvalue of H.  A Ritz
    value with residual r lies within r^2 / gap of its eigenvalue, so values with r < 1e-5
    (gap 0.27) count as converged."""
    from scipy.sparse.linalg import LinearOperator, eigsh
    inst = W.ring16()
    b = hm.Basis(16, 1, 0)
    ob = oracle.Basis(16, 1, 8)
    res = hm.lanczos_run(b, hm.bonds_of(inst), inst.steps, seed=inst.seed, n_ritz=5)
    al, be = ob.lanczos(obonds(inst), oracle.start_uniform(inst.seed, b.dim), inst.steps)
    assert res.steps_done == len(al) == 100
    th_o, r_o = ritz_with_residuals(al, be, 5)
    th_g, r_g = ritz_with_residuals(res.alpha, res.beta, 5)
    np.testing.assert_allclose(res.ritz, th_g, rtol=0, atol=1e-12)   # device bisection
    op = LinearOperator((ob.dim, ob.dim), matvec=lambda x: ob.matvec(obonds(inst), np.ravel(x)), dtype=float)
    exact = np.sort(eigsh(op, k=8, which="SA", tol=1e-13, v0=oracle.start_uniform(5, ob.dim))[0])
    n_conv = 0
    for j in range(5):
        if r_o[j] < 1e-5 and r_g[j] < 1e-5:
            n_conv += 1
            assert abs(res.ritz[j] - th_o[j]) <= 1e-10 * abs(th_o[j]), (j, res.ritz[j], th_o[j])
        else:
            assert abs(res.ritz[j] - th_o[j]) <= r_g[j] + r_o[j] + 1e-10, (j, res.ritz[j], th_o[j], r_g[j], r_o[j])
        assert np.min(np.abs(exact - res.ritz[j])) <= r_g[j] + 1e-9, (j, res.ritz[j])
    assert n_conv >= 4
    assert abs(res.ritz[0] - (-7.142296360617)) < 1e-10


@pytest.mark.slow
def test_s1_rrg20_fp32_against_fp64(hm):
    """s = 1, N = 20, 4-regular random graph, M = 0 (dim 377,379,369), start vector seed
    1003: FP32 Lanczos vectors (FP64 reductions and eigensolve) against FP64 vectors from
    the same start vector, after the stated 80 steps and once converged (200 steps):
    |dE0/E0| <= 1e-6."""
    inst = W.s1_random_graph()
    b = hm.Basis(20, 2, 0)
    assert b.dim == 377379369
    bl = hm.bonds_of(inst)
    for steps in (inst.steps, 200):
        r64 = hm.lanczos_run(b, bl, steps, seed=inst.seed, n_ritz=1)
        torch.cuda.empty_cache()
        r32 = hm.lanczos_run(b, bl, steps, seed=inst.seed, n_ritz=1, dtype=torch.float32)
        torch.cuda.empty_cache()
        err = abs(r32.ritz[0] - r64.ritz[0]) / abs(r64.ritz[0])
        print(f"s1_rrg20 steps={steps}: E0(f64)={r64.ritz[0]:.12f} E0(f32)={r32.ritz[0]:.12f} |dE0/E0|={err:.2e}")
        assert r64.steps_done == r32.steps_done == steps
        assert err <= 1e-6, (steps, r64.ritz[0], r32.ritz[0])


@pytest.fixture(scope="module")
def ring24(hm):
    inst = W.ring24_random_j()
    assert inst.n_bonds == 48
    return inst, hm.Basis(24, 1, 0), oracle.Basis(24, 1, 12)


def test_ring24_autograd_full_sector(hm, ring24):
    """y = H(J) x through the autograd function on the whole N = 24 sector (2,704,156 rows,
    48 distinct couplings), loss L = w.y + |y|^2/2: dL/dx = H g and dL/dJ = -g^T (s_u.s_v) x
    with g = w + y, against the oracle's whole-sector product and bond correlations."""
    from paper_0706_3293_gb300.autograd import HeisenbergMatvec
    inst, b, ob = ring24
    x = torch.from_numpy(oracle.start_uniform(7, b.dim)).cuda().requires_grad_(True)
    J = torch.tensor(inst.J, dtype=torch.float64, requires_grad=True)
    w = torch.from_numpy(oracle.start_uniform(8, b.dim)).cuda()
    y = HeisenbergMatvec.apply(x, J, b, inst.u, inst.v)
    loss = (w * y).sum() + 0.5 * (y * y).sum()
    loss.backward()
    xn = x.detach().cpu().numpy()
    yr = ob.matvec(obonds(inst), xn)
    assert np.linalg.norm(y.detach().cpu().numpy() - yr) <= 1e-12 * np.linalg.norm(yr)
    g = w.cpu().numpy() + yr
    gx = ob.matvec(obonds(inst), g)
    assert np.linalg.norm(x.grad.cpu().numpy() - gx) <= 1e-12 * np.linalg.norm(gx)
    gJ = -ob.bond_corr(obonds(inst), g, xn)
    np.testing.assert_allclose(J.grad.numpy(), gJ, rtol=1e-10, atol=1e-12 * np.abs(gJ).max())
    # Euler: L's J-part is homogeneous: J . dL/dJ = g . H x exactly (H linear in J)
    assert abs(float(J.detach().numpy() @ J.grad.numpy()) - float(g @ yr)) <= 1e-9 * abs(float(g @ yr))


@pytest.mark.slow
def test_ring24_e0_grad_full_sector(hm, ring24):
    """dE0/dJ_b = -<psi0|s_u.s_v|psi0> at N = 24 with 48 couplings: e0_grad against the
    oracle's two-pass ground state on the same start vector (E0 1e-10, gradient 1e-8), the
    Euler identity sum_b J_b dE0/dJ_b = E0, and central finite differences of the GPU's own
    converged ground energy, h = 1e-6, for six bonds (about 1e-6)."""
    inst, b, ob = ring24
    bl = hm.bonds_of(inst)
    steps = 120
    e0, g, psi, rc = hm.e0_grad(b, bl, steps, seed=inst.seed, want_psi=True)
    assert rc == 0
    oe0, og = oracle.e0_grad(ob, obonds(inst), oracle.start_uniform(inst.seed, b.dim), steps)
    assert abs(e0 - oe0) <= 1e-10 * abs(oe0), (e0, oe0)
    np.testing.assert_allclose(g, og, rtol=0, atol=1e-8)
    assert abs(float(np.dot(inst.J, g)) - e0) < 1e-8 * abs(e0)
    h = 1e-6
    for t in (0, 5, 17, 24, 33, 47):
        Jp, Jm = inst.J.copy(), inst.J.copy()
        Jp[t] += h
        Jm[t] -= h
        ep = hm.lanczos_run(b, hm.BondList.make(inst.u, inst.v, Jp), 200, seed=inst.seed, n_ritz=1).ritz[0]
        em = hm.lanczos_run(b, hm.BondList.make(inst.u, inst.v, Jm), 200, seed=inst.seed, n_ritz=1).ritz[0]
        fd = (ep - em) / (2 * h)
        print(f"ring24_randJ bond {t}: dE0/dJ = {g[t]:.10f}, central difference {fd:.10f}")
        assert abs(fd - g[t]) < 1e-6, (t, fd, g[t])


def test_ftlm_ring24_m0_sector_against_fp64(hm):
    """The batched FP32 run of the N = 24 J1-J2 ring (all 25 sectors, R = 32 +-1 vectors,
    80 steps): the lowest Ritz value of vector r = 0 in the M = 0 sector (2,704,156 rows)
    against an FP64 Lanczos run of 80 steps from the same +-1 vector (stream (1005, 12, 0)),
    |dE0/E0| <= 1e-6."""
    inst = W.ftlm_ring24()
    R, steps, seed = 32, inst.steps, inst.seed
    gpu = hm.ftlm_run(24, hm.bonds_of(inst), R, steps, seed, [1.0])
    b = hm.Basis(24, 1, 0)
    v0 = torch.from_numpy(oracle.start_pm1(oracle.stream_seed(seed, 12, 0), b.dim)).cuda()
    r64 = hm.lanczos_run(b, hm.bonds_of(inst), steps, v0=v0, n_ritz=1)
    m = int(gpu.mlen[12, 0])
    assert m == r64.steps_done == steps
    e32 = float(np.min(gpu.theta[12, 0, :m]))
    err = abs(e32 - r64.ritz[0]) / abs(r64.ritz[0])
    print(f"ftlm_ring24 M=0 r=0: E0(f64)={r64.ritz[0]:.12f} E0(f32 batched)={e32:.12f} |dE0/E0|={err:.2e}")
    assert err <= 1e-6, (e32, r64.ritz[0])
