"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the same seeded
inputs.  Tolerances: indices and states bit-exact; FP64 rows ||dy||/||y|| <= 1e-12;
FP32 rows (FP32 storage and accumulation) ||dy||/||y|| <= 1e-5; E0 <= 1e-10 relative."""
import math

import numpy as np
import pytest

import oracle
from paper_0706_3293_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL_F64 = 1e-12
TOL_F32 = 1e-5
TOL_E0 = 1e-10


@pytest.fixture(scope="module")
def hm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0706_3293_gb300 import build
    build.build()
    from paper_0706_3293_gb300 import api
    return api


def obonds(inst):
    return oracle.Bonds(inst.u, inst.v, inst.J)


def pack(digits, bits):
    w = 0
    for k, a in enumerate(digits):
        w |= int(a) << (k * bits)
    return w


def bits_of(two_s):
    return 1 if two_s == 1 else (2 if two_s <= 3 else 4)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


SMALL = [
    W.ring16(),
    W.small_ring(18, -1.0, -0.5),
    W.s1_random_graph(10, 21),
    W.s1_random_graph_small(),
    W.Instance("s32_N8_A6", 8, 3, 0, np.array([0, 1, 2, 3, 4, 5, 6, 7, 0, 2], np.int32),
               np.array([1, 2, 3, 4, 5, 6, 7, 0, 5, 6], np.int32),
               np.linspace(-1.2, 0.9, 10)),
    W.Instance("s2_N6", 6, 4, 2, np.array([0, 1, 2, 3, 4, 5, 0], np.int32),
               np.array([1, 2, 3, 4, 5, 0, 3], np.int32), np.linspace(-1.0, 0.5, 7)),
]


# ---- codec -------------------------------------------------------------------------------

@pytest.mark.parametrize("inst", SMALL[:5], ids=lambda i: i.name)
def test_codec_all_indices(hm, inst):
    b = hm.Basis(inst.n_sites, inst.two_s, inst.two_m)
    ob = oracle.Basis(inst.n_sites, inst.two_s, inst.A)
    assert b.dim == ob.dim
    idx = torch.arange(b.dim, dtype=torch.int64, device="cuda")
    st = b.decode(idx).cpu().numpy()
    bits = bits_of(inst.two_s)
    step = max(1, b.dim // 3000)
    for i in list(range(0, b.dim, step)) + [b.dim - 1]:
        assert int(st[i]) == pack(ob.decode(i), bits), i
    back = b.encode(torch.from_numpy(st).cuda()).cpu().numpy()
    assert np.array_equal(back, np.arange(b.dim))


def test_codec_worked_example(hm):
    """Sec. 3.2 example: N = 4, s = 3/2, A = 6, |1,0,2,3> has 0-based index 41."""
    b = hm.Basis(4, 3, 0)
    st = torch.tensor([pack([1, 0, 2, 3], 2)], dtype=torch.int64, device="cuda")
    assert int(b.encode(st)[0]) == 41
    assert int(b.decode(torch.tensor([41], device="cuda"))[0]) == pack([1, 0, 2, 3], 2)


def test_codec_rejects_outside(hm):
    b = hm.Basis(6, 1, 0)
    out = b.decode(torch.tensor([-1, b.dim, 0], dtype=torch.int64, device="cuda")).cpu()
    assert int(out[0]) == -1 and int(out[1]) == -1
    bad = torch.tensor([0b111, 0b1000111, 0b111000], dtype=torch.int64, device="cuda")
    e = b.encode(bad).cpu()
    assert int(e[0]) == 0 and int(e[1]) == -1 and int(e[2]) >= 0


@pytest.mark.parametrize("n,two_s,two_m", [(32, 1, 0), (20, 2, 0)])
def test_codec_full_size_sampled(hm, n, two_s, two_m):
    b = hm.Basis(n, two_s, two_m)
    ob = oracle.Basis(n, two_s, (n * two_s - two_m) // 2)
    rng = np.random.default_rng(1)
    idx = np.concatenate([[0, 1, 2, b.dim - 2, b.dim - 1], rng.integers(0, b.dim, 3000)])
    st = b.decode(torch.from_numpy(idx).cuda()).cpu().numpy()
    bits = bits_of(two_s)
    for i, s in zip(idx, st):
        assert int(s) == pack(ob.decode(int(i)), bits)
    assert np.array_equal(b.encode(torch.from_numpy(st).cuda()).cpu().numpy(), idx)


# ---- start vectors -----------------------------------------------------------------------

def test_start_vectors_bitwise(hm):
    b = hm.Basis(16, 1, 0)
    for kind, ref in [(0, oracle.start_uniform(1001, b.dim)), (1, oracle.start_pm1(77, b.dim))]:
        seed = 1001 if kind == 0 else 77
        x = hm.start_vector(b, seed, kind).cpu().numpy()
        assert np.array_equal(x, ref)
        xf = hm.start_vector(b, seed, kind, dtype=torch.float32).cpu().numpy()
        assert np.array_equal(xf, ref.astype(np.float32))


# ---- matvec ------------------------------------------------------------------------------

@pytest.mark.parametrize("inst", SMALL, ids=lambda i: i.name)
def test_matvec_f64(hm, inst):
    b = hm.Basis(inst.n_sites, inst.two_s, inst.two_m)
    ob = oracle.Basis(inst.n_sites, inst.two_s, inst.A)
    x = oracle.start_uniform(5, b.dim)
    ref = ob.matvec(obonds(inst), x)
    y = hm.matvec(b, hm.bonds_of(inst), torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, ref) <= TOL_F64
    assert np.max(np.abs(y - ref)) <= TOL_F64 * np.max(np.abs(ref)) * 10


@pytest.mark.parametrize("inst", SMALL, ids=lambda i: i.name)
def test_matvec_f32(hm, inst):
    b = hm.Basis(inst.n_sites, inst.two_s, inst.two_m)
    ob = oracle.Basis(inst.n_sites, inst.two_s, inst.A)
    x32 = oracle.start_uniform(6, b.dim).astype(np.float32)
    ref = ob.matvec(obonds(inst), x32.astype(np.float64))
    y = hm.matvec(b, hm.bonds_of(inst), torch.from_numpy(x32).cuda()).cpu().numpy()
    assert rel(y.astype(np.float64), ref) <= TOL_F32


@pytest.mark.parametrize("nvec", [2, 5, 32, 37])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_matvec_batched(hm, nvec, dtype):
    inst = W.small_ring(14, -1.0, -0.3)
    b = hm.Basis(14, 1, 0)
    ob = oracle.Basis(14, 1, 7)
    X = np.stack([oracle.start_pm1(100 + r, b.dim) * oracle.start_uniform(200 + r, b.dim)
                  for r in range(nvec)], axis=1)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    Xt = torch.from_numpy(X).to(tdt).cuda()
    Y = hm.matvec(b, hm.bonds_of(inst), Xt).cpu().numpy().astype(np.float64)
    Xr = Xt.cpu().numpy().astype(np.float64)
    for r in range(nvec):
        ref = ob.matvec(obonds(inst), Xr[:, r].copy())
        assert rel(Y[:, r], ref) <= (TOL_F64 if dtype == "f64" else TOL_F32)


@pytest.mark.parametrize("run", [3, 8])
@pytest.mark.parametrize("inst", SMALL[2:], ids=lambda i: i.name)
def test_general_rows_successor_runs(hm, inst, run, monkeypatch):
    """The general row kernels walking runs of consecutive rows by the successor rule
    (Sec. 3.1) instead of one decode per row: the same products as the oracle, single and
    batched, and the same Lanczos coefficients.  Run lengths 3 and 8 leave ragged last runs."""
    monkeypatch.setenv("HM_ROW_RUN", str(run))
    b = hm.Basis(inst.n_sites, inst.two_s, inst.two_m)
    ob = oracle.Basis(inst.n_sites, inst.two_s, inst.A)
    x = oracle.start_uniform(5, b.dim)
    ref = ob.matvec(obonds(inst), x)
    y = hm.matvec(b, hm.bonds_of(inst), torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, ref) <= TOL_F64
    X = np.stack([oracle.start_pm1(40 + r, b.dim) for r in range(5)], axis=1)
    Y = hm.matvec(b, hm.bonds_of(inst), torch.from_numpy(X).cuda()).cpu().numpy()
    for r in range(5):
        assert rel(Y[:, r], ob.matvec(obonds(inst), X[:, r].copy())) <= TOL_F64
    steps = min(20, b.dim)
    res = hm.lanczos_run(b, hm.bonds_of(inst), steps, seed=9, n_ritz=1)
    al, be = ob.lanczos(obonds(inst), oracle.start_uniform(9, b.dim), steps)
    k = min(len(al), res.steps_done, 12)
    np.testing.assert_allclose(res.alpha[:k], al[:k], rtol=0, atol=1e-12 * np.abs(al).max())


def test_matvec_empty_bonds_and_tiny_sectors(hm):
    """No bonds: y = 0.  A dim-1 sector: y = E x with E = -s^2 sum J."""
    b = hm.Basis(6, 1, 6)
    assert b.dim == 1
    inst = W.small_ring(6, 0.8)
    y = hm.matvec(b, hm.bonds_of(inst), torch.tensor([2.0], dtype=torch.float64, device="cuda"))
    assert abs(float(y[0]) - 2.0 * (-0.25 * 6 * 0.8)) < 1e-15
    b2 = hm.Basis(10, 1, 0)
    y2 = hm.matvec(b2, hm.BondList.make([], [], []), torch.ones(b2.dim, dtype=torch.float64, device="cuda"))
    assert float(y2.abs().max()) == 0.0


def test_matvec_full_size_sampled_rows(hm):
    """The 601,080,390-row J1-J2 ring sector in FP64: sampled rows of one product,
    computed one by one by the oracle, in the launch configuration the benchmark uses."""
    inst = W.j1j2_ring32()
    b = hm.Basis(32, 1, 0)
    ob = oracle.Basis(32, 1, 16)
    x = oracle.start_uniform(inst.seed, b.dim)
    xt = torch.from_numpy(x).cuda()
    y = hm.matvec(b, hm.bonds_of(inst), xt)
    rng = np.random.default_rng(7)
    starts = np.concatenate([[0, b.dim - 256], rng.integers(0, b.dim - 256, 12)])
    for r0 in starts:
        r0 = int(r0)
        ref = ob.matvec_rows(obonds(inst), x, r0, r0 + 256)
        got = y[r0:r0 + 256].cpu().numpy()
        assert rel(got, ref) <= TOL_F64
    del y, xt


# ---- bond correlations / autograd -------------------------------------------------------

@pytest.mark.parametrize("inst", [SMALL[1], SMALL[3], SMALL[4]], ids=lambda i: i.name)
def test_bond_corr(hm, inst):
    b = hm.Basis(inst.n_sites, inst.two_s, inst.two_m)
    ob = oracle.Basis(inst.n_sites, inst.two_s, inst.A)
    g, x = oracle.start_uniform(8, b.dim), oracle.start_uniform(9, b.dim)
    ref = ob.bond_corr(obonds(inst), g, x)
    got = hm.bond_corr(b, hm.bonds_of(inst), torch.from_numpy(g).cuda(), torch.from_numpy(x).cuda())
    np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_autograd_matvec(hm):
    from paper_0706_3293_gb300.autograd import HeisenbergMatvec
    inst = W.small_ring(16, -1.0, -0.4)
    rng = np.random.default_rng(3)
    Jn = rng.uniform(-1.2, -0.8, inst.n_bonds)
    b = hm.Basis(16, 1, 0)
    ob = oracle.Basis(16, 1, 8)
    x = torch.from_numpy(oracle.start_uniform(1, b.dim)).cuda().requires_grad_(True)
    J = torch.tensor(Jn, dtype=torch.float64, requires_grad=True)
    w = torch.from_numpy(oracle.start_uniform(2, b.dim)).cuda()
    y = HeisenbergMatvec.apply(x, J, b, inst.u, inst.v)
    loss = (w * y).sum() + 0.5 * (y * y).sum()
    loss.backward()
    ob_b = oracle.Bonds(inst.u, inst.v, Jn)
    yr = ob.matvec(ob_b, x.detach().cpu().numpy())
    g = w.cpu().numpy() + yr
    np.testing.assert_allclose(x.grad.cpu().numpy(), ob.matvec(ob_b, g), rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(J.grad.numpy(), -ob.bond_corr(ob_b, g, x.detach().cpu().numpy()),
                               rtol=1e-10)
    # directional finite difference in J (L is quadratic in J: central difference exact up
    # to rounding)
    d = rng.standard_normal(inst.n_bonds)
    h = 1e-4

    def L(Jv):
        yv = ob.matvec(oracle.Bonds(inst.u, inst.v, Jv), x.detach().cpu().numpy())
        return w.cpu().numpy() @ yv + 0.5 * yv @ yv
    fd = (L(Jn + h * d) - L(Jn - h * d)) / (2 * h)
    assert abs(fd - J.grad.numpy() @ d) < 1e-6 * abs(fd)


# ---- Lanczos -----------------------------------------------------------------------------

def test_lanczos_ring16_config(hm):
    """16-site ring, M = 0, FP64, uniform start seed 1001, 100 steps: E0 and the lowest 5
    Ritz values against the oracle run on the same start vector."""
    inst = W.ring16()
    b = hm.Basis(16, 1, 0)
    ob = oracle.Basis(16, 1, 8)
    res = hm.lanczos_run(b, hm.bonds_of(inst), inst.steps, seed=inst.seed, n_ritz=5)
    al, be = ob.lanczos(obonds(inst), oracle.start_uniform(inst.seed, b.dim), inst.steps)
    assert res.steps_done == len(al) == 100
    np.testing.assert_allclose(res.alpha[:30], al[:30], rtol=0, atol=1e-11)
    np.testing.assert_allclose(res.beta[:30], be[:30], rtol=0, atol=1e-11)
    ref = oracle.tridiag_lowest(al, be, 5)
    assert abs(res.ritz[0] - ref[0]) <= TOL_E0 * abs(ref[0])
    assert abs(res.ritz[0] - (-7.142296360617)) < 1e-10
    # Ritz values of T from the GPU's own alpha/beta, bisection on host vs device
    np.testing.assert_allclose(res.ritz, oracle.tridiag_lowest(res.alpha, res.beta, 5), rtol=0, atol=1e-13)


def test_lanczos_s1_small_f64_f32(hm):
    """s = 1, N = 12 random 4-regular graph (dim 73,789), 140 steps (E0 converged): FP64
    Lanczos against the oracle (first steps to 1e-12, E0 to 1e-10) and FP32 vectors
    against FP64 (|dE0/E0| <= 1e-6).  Before convergence two valid runs drift apart by
    amplified rounding, so E0 is compared where it has converged."""
    inst = W.s1_random_graph_small()
    b = hm.Basis(12, 2, 0)
    ob = oracle.Basis(12, 2, 12)
    r64 = hm.lanczos_run(b, hm.bonds_of(inst), 140, seed=inst.seed, n_ritz=1)
    al, be = ob.lanczos(obonds(inst), oracle.start_uniform(inst.seed, b.dim), 140)
    np.testing.assert_allclose(r64.alpha[:20], al[:20], rtol=0, atol=1e-12 * np.abs(al).max())
    np.testing.assert_allclose(r64.beta[:20], be[:20], rtol=0, atol=1e-12 * np.abs(al).max())
    e_ref = oracle.tridiag_lowest(al, be, 1)[0]
    assert abs(r64.ritz[0] - e_ref) <= TOL_E0 * abs(e_ref)
    r32 = hm.lanczos_run(b, hm.bonds_of(inst), 140, seed=inst.seed, n_ritz=1, dtype=torch.float32)
    assert abs(r32.ritz[0] - e_ref) <= 1e-6 * abs(e_ref)


def test_lanczos_stepwise_equals_graph(hm):
    inst = W.small_ring(14, -1.0, -0.3)
    b = hm.Basis(14, 1, 0)
    run = hm.LanczosRun(b, hm.bonds_of(inst), 40, seed=3)
    run.step(40)
    al, be, rc = run.read()
    res = hm.lanczos_run(b, hm.bonds_of(inst), 40, seed=3, n_ritz=1)
    assert np.array_equal(al, res.alpha) and np.array_equal(be, res.beta)


def test_lanczos_breakdown_small_sectors(hm):
    """Sectors of dim 1 and 8 exhaust their Krylov space: beta falls far below the
    breakdown threshold and both sides stop at the same step with the same Ritz value.
    The dim-28 sector loses orthogonality before beta gets that small (floating point);
    there only E0 is compared."""
    inst = W.small_ring(8, -1.0, -0.3)
    for two_m, dim, clean in [(8, 1, True), (6, 8, True), (4, 28, False)]:
        b = hm.Basis(8, 1, two_m)
        assert b.dim == dim
        res = hm.lanczos_run(b, hm.bonds_of(inst), 60, seed=11, n_ritz=1)
        ob = oracle.Basis(8, 1, (8 - two_m) // 2)
        al, be = ob.lanczos(obonds(inst), oracle.start_uniform(11, dim), 60)
        if clean:
            assert res.steps_done == len(al) <= dim
            assert res.status == 1    # HM_BREAKDOWN
        assert abs(res.ritz[0] - oracle.tridiag_lowest(al, be, 1)[0]) < 1e-12


def test_lanczos_user_start_vector(hm):
    inst = W.small_ring(12, -1.0)
    b = hm.Basis(12, 1, 0)
    ob = oracle.Basis(12, 1, 6)
    v0 = oracle.start_pm1(5, b.dim) * 0.25
    res = hm.lanczos_run(b, hm.bonds_of(inst), 30, v0=torch.from_numpy(v0).cuda(), n_ritz=2)
    al, be = ob.lanczos(obonds(inst), v0, 30)
    np.testing.assert_allclose(res.alpha[:10], al[:10], atol=1e-12)


# ---- ground-state gradient -------------------------------------------------------------

def test_e0_grad_vs_oracle(hm):
    inst = W.small_ring(14, -1.0, -0.3)
    rng = np.random.default_rng(12)
    J = rng.uniform(-1.2, -0.8, inst.n_bonds)
    b = hm.Basis(14, 1, 0)
    ob = oracle.Basis(14, 1, 7)
    bl = hm.BondList.make(inst.u, inst.v, J)
    e0, g, psi, rc = hm.e0_grad(b, bl, 120, seed=21, want_psi=True)
    oe0, og = oracle.e0_grad(ob, oracle.Bonds(inst.u, inst.v, J), oracle.start_uniform(21, b.dim), 120)
    assert abs(e0 - oe0) <= TOL_E0 * abs(oe0)
    np.testing.assert_allclose(g, og, rtol=0, atol=1e-8)
    assert abs(np.dot(J, g) - e0) < 1e-8        # Euler
    assert abs(float(torch.linalg.norm(psi)) - 1.0) < 1e-12


# ---- s = 1/2 block path (sites split 16 low / N-16 high) ---------------------------------

@pytest.mark.parametrize("two_m", [0, 2, 6, 12, 16, 18])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_matvec_block_path_all_sectors(hm, two_m, dtype):
    """N = 20 J1-J2 ring (two coupling classes): the block kernel over sectors whose
    blocks range from one row to C(16, 8)."""
    inst = W.small_ring(20, -1.0, -0.3, two_m=two_m)
    b = hm.Basis(20, 1, two_m)
    ob = oracle.Basis(20, 1, inst.A)
    x = oracle.start_uniform(31 + two_m, b.dim)
    if dtype == "f32":
        x = x.astype(np.float32).astype(np.float64)
    ref = ob.matvec(obonds(inst), x)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    y = hm.matvec(b, hm.bonds_of(inst), torch.from_numpy(x).to(tdt).cuda()).cpu().numpy()
    assert rel(y.astype(np.float64), ref) <= (TOL_F64 if dtype == "f64" else TOL_F32)


def test_matvec_block_path_three_classes_and_scaled_input(hm):
    """Three coupling classes, and an input scaled far from 1 (fixed-point unit follows
    the vector's largest exponent)."""
    u, v, _ = W.ring_bonds(22, 1.0, 1.0)
    J = np.where(np.arange(len(u)) % 3 == 0, -1.0, np.where(np.arange(len(u)) % 3 == 1, 0.7, -0.25))
    inst = W.Instance("r22c3", 22, 1, 0, u, v, J)
    b = hm.Basis(22, 1, 0)
    ob = oracle.Basis(22, 1, 11)
    for s in [1.0, 2.0**-40, 2.0**35]:
        x = oracle.start_uniform(4, b.dim) * s
        ref = ob.matvec(obonds(inst), x)
        y = hm.matvec(b, hm.bonds_of(inst), torch.from_numpy(x).cuda()).cpu().numpy()
        assert rel(y, ref) <= TOL_F64


def test_lanczos_block_path(hm):
    """N = 20 J1-J2 ring, M = 0 (dim 184,756) on the block path: first steps to 1e-12
    against the oracle, E0 to 1e-10 once converged, FP32 vectors to 1e-6."""
    inst = W.small_ring(20, -1.0, -0.3)
    b = hm.Basis(20, 1, 0)
    ob = oracle.Basis(20, 1, 10)
    r64 = hm.lanczos_run(b, hm.bonds_of(inst), 150, seed=9, n_ritz=1)
    al, be = ob.lanczos(obonds(inst), oracle.start_uniform(9, b.dim), 150)
    np.testing.assert_allclose(r64.alpha[:20], al[:20], rtol=0, atol=1e-12 * np.abs(al).max())
    np.testing.assert_allclose(r64.beta[:20], be[:20], rtol=0, atol=1e-12 * np.abs(al).max())
    e_ref = oracle.tridiag_lowest(al, be, 1)[0]
    assert abs(r64.ritz[0] - e_ref) <= TOL_E0 * abs(e_ref)
    r32 = hm.lanczos_run(b, hm.bonds_of(inst), 150, seed=9, n_ritz=1, dtype=torch.float32)
    assert abs(r32.ritz[0] - e_ref) <= 1e-6 * abs(e_ref)


def test_e0_grad_block_path(hm):
    inst = W.small_ring(18, -1.0, -0.3)
    b = hm.Basis(18, 1, 0)
    ob = oracle.Basis(18, 1, 9)
    e0, g, psi, rc = hm.e0_grad(b, hm.bonds_of(inst), 150, seed=5, want_psi=True)
    oe0, og = oracle.e0_grad(ob, obonds(inst), oracle.start_uniform(5, b.dim), 150)
    assert abs(e0 - oe0) <= TOL_E0 * abs(oe0)
    np.testing.assert_allclose(g, og, rtol=0, atol=1e-8)
    assert abs(np.dot(inst.J, g) - e0) < 1e-8


@pytest.mark.parametrize("inst", [SMALL[0], SMALL[1], SMALL[3], SMALL[4], SMALL[5]], ids=lambda i: i.name)
def test_count_nnz(hm, inst):
    b = hm.Basis(inst.n_sites, inst.two_s, inst.two_m)
    ob = oracle.Basis(inst.n_sites, inst.two_s, inst.A)
    assert hm.count_nnz(b, hm.bonds_of(inst)) == ob.count_nnz(obonds(inst))


def test_count_nnz_full_size_closed_form(hm):
    """s = 1/2, M = 0: nnz = C(N, N/2) + 2 n_bonds C(N-2, N/2-1) (601M-row sector)."""
    inst = W.j1j2_ring32()
    b = hm.Basis(32, 1, 0)
    assert hm.count_nnz(b, hm.bonds_of(inst)) == math.comb(32, 16) + 2 * 64 * math.comb(30, 15)


@pytest.mark.parametrize("case,row", [("j1j2_n20_f64", "table"), ("three_class_n18_f64", "table"),
                                      ("j1j2_n20_f32", "table"), ("four_class_j1j2_n20_f64", "table"),
                                      ("four_class_j1j2_n20_f32", "table"),
                                      ("j1j2_n20_f64", "slots"), ("three_class_n18_f64", "slots"),
                                      ("j1j2_n20_f32", "slots"), ("j1j2_n20_f64", "delta"),
                                      ("three_class_n18_f64", "delta"), ("j1j2_n20_f32", "delta")])
def test_block_product_specialised_equals_generic(hm, case, row, monkeypatch):
    """The block product compiled for the bond list at run time (NVRTC; three row policies:
    per-class target tables (the default), slots written out, or per-byte delta tables) and
    the generic block kernel form the same exact integer sums in FP64, so 60 Lanczos steps
    agree bit for bit.  In FP32 the sums round in another order (the delta policy adds x_r for
    parallel bonds and takes it back in the diagonal term): the recurrences agree to FP32
    accuracy."""
    if case == "three_class_n18_f64":
        n, J = 18, [-1.0 if i % 3 == 0 else (0.5 if i % 3 == 1 else -0.25) for i in range(18)]
        u = list(range(18)) + [0, 3, 2]
        v = [(i + 1) % 18 for i in range(18)] + [9, 12, 17]
        J = J + [-1.0, 0.5, -0.25]
        bonds = hm.BondList.make(u, v, J)
        two_m, dt = 2, torch.float64
    elif case.startswith("four_class"):
        # NN and NNN bonds with four couplings in integer ratios spread over both kinds, so
        # the triangles of the target tables mix classes (or are skipped where the two edges
        # at their shared site differ)
        n = 20
        inst = W.small_ring(n, -1.0, -0.5)
        J = [(-1.0, -0.5, -0.25, -0.75)[(3 * i + i // 5) % 4] for i in range(inst.n_bonds)]
        bonds = hm.BondList.make(inst.u, inst.v, J)
        two_m, dt = 2, (torch.float32 if case.endswith("f32") else torch.float64)
    else:
        n = 20
        bonds = hm.bonds_of(W.small_ring(n, -1.0, -0.3))
        two_m, dt = 0, (torch.float32 if case.endswith("f32") else torch.float64)
    b = hm.Basis(n, 1, two_m)
    monkeypatch.setenv("HM_JIT_ROW", row)
    runs = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("HM_JIT", mode)
        r = hm.LanczosRun(b, bonds, 60, seed=11, dtype=dt)
        name = r.kernel_name()
        r.step(60)
        runs[mode] = (name, r.read())
        r.close()
    assert runs["1"][0].endswith("_jit"), runs["1"][0]
    assert runs["0"][0].startswith("k_blk_lz") and not runs["0"][0].endswith("_jit")
    (a1, b1, _), (a0, b0, _) = runs["1"][1], runs["0"][1]
    if dt == torch.float64:
        assert np.array_equal(a1, a0) and np.array_equal(b1, b0)
    else:
        np.testing.assert_allclose(a1[:10], a0[:10], rtol=0, atol=2e-5)
        np.testing.assert_allclose(b1[:10], b0[:10], rtol=0, atol=2e-5)
        e1 = oracle.tridiag_lowest(a1, b1, 1)[0]
        e0 = oracle.tridiag_lowest(a0, b0, 1)[0]
        assert abs(e1 - e0) <= 1e-5 * abs(e0)


@pytest.mark.slow
def test_lanczos_full_size_majumdar_ghosh(hm):
    """The bench workload at full size (N = 32, J2 = J1/2, M = 0, 601,080,390 rows) through
    the same run type bench.py times: J2 = J1/2 on an even periodic ring is the
    Majumdar-Ghosh point, whose ground energy is exactly -3N/8 = -12 (two dimer
    singlets), independent of this code and of the oracle."""
    inst = W.j1j2_ring32()
    b = hm.Basis(32, 1, 0)
    run = hm.LanczosRun(b, hm.bonds_of(inst), 150, seed=inst.seed)
    assert run.kernel_name().startswith("k_blk_lz64")
    run.step(150)
    al, be, rc = run.read()
    run.close()
    e0 = oracle.tridiag_lowest(al, be, 1)[0]
    assert abs(e0 - (-12.0)) <= 1e-9 * 12.0, e0


@pytest.mark.slow
def test_lanczos_full_size_majumdar_ghosh_f32(hm):
    """The same full-size run with FP32 Lanczos vectors (FP64 reductions): the ground energy
    -12 of the Majumdar-Ghosh point within |dE0/E0| <= 1e-6."""
    inst = W.j1j2_ring32()
    b = hm.Basis(32, 1, 0)
    run = hm.LanczosRun(b, hm.bonds_of(inst), 150, seed=inst.seed, dtype=torch.float32)
    assert run.kernel_name().startswith("k_blk_lz32")
    run.step(150)
    al, be, rc = run.read()
    run.close()
    e0 = oracle.tridiag_lowest(al, be, 1)[0]
    assert abs(e0 - (-12.0)) <= 1e-6 * 12.0, e0


@pytest.mark.slow
def test_block_product_specialised_equals_generic_full_size(hm, monkeypatch):
    """At N = 32 (the bench's launch configuration: dynamic block schedule over 131,070
    blocks, 456 CTAs) the one-pass specialised product (the default), the split specialised
    product and the generic FP64 block product give the same Lanczos coefficients bit for
    bit over 4 steps."""
    inst = W.j1j2_ring32()
    b = hm.Basis(32, 1, 0)
    out = {}
    for mode, env in (("split", {"HM_BLK_SPLIT": "1"}), ("one", {}), ("generic", {"HM_JIT": "0"})):
        monkeypatch.delenv("HM_BLK_SPLIT", raising=False)
        monkeypatch.delenv("HM_JIT", raising=False)
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        run = hm.LanczosRun(b, hm.bonds_of(inst), 4, seed=inst.seed)
        name = run.kernel_name()
        run.step(4)
        out[mode] = (name, run.read())
        run.close()
        torch.cuda.empty_cache()
    assert out["split"][0] == "k_blk_lz64a_jit+k_blk_lz64b_jit"
    assert out["one"][0] == "k_blk_lz64_jit" and out["generic"][0] == "k_blk_lz64"
    (a1, b1, _) = out["split"][1]
    for mode in ("one", "generic"):
        a0, b0, _ = out[mode][1]
        assert np.array_equal(a1, a0) and np.array_equal(b1, b0), mode


@pytest.mark.parametrize("N,j2,two_m", [(20, -0.5, 0), (22, -0.25, 2), (24, -0.5, 0), (26, -0.5, 4)])
def test_split_product_equals_one_pass(hm, N, j2, two_m, monkeypatch):
    """The split FP64 product (near bonds in a first pass that leaves exact integer row
    sums, the bonds reaching site N-7 and above in a second pass over the blocks in rotated
    order) forced on smaller sectors: 40 Lanczos steps bit for bit equal to the one-pass
    product, whose first steps match the oracle."""
    inst = W.small_ring(N, -1.0, j2)
    b = hm.Basis(N, 1, two_m)
    out = {}
    for mode in ("1", "0"):
        monkeypatch.setenv("HM_BLK_SPLIT", mode)
        run = hm.LanczosRun(b, hm.bonds_of(inst), 40, seed=5)
        name = run.kernel_name()
        run.step(40)
        out[mode] = (name, run.read())
        run.close()
    assert out["1"][0] == "k_blk_lz64a_jit+k_blk_lz64b_jit", out["1"][0]
    assert out["0"][0] == "k_blk_lz64_jit"
    (a1, b1, _), (a0, b0, _) = out["1"][1], out["0"][1]
    assert np.array_equal(a1, a0) and np.array_equal(b1, b0)
    if N <= 22:
        ob = oracle.Basis(N, 1, (N - two_m) // 2)
        al, be = ob.lanczos(obonds(inst), oracle.start_uniform(5, ob.dim), 20)
        np.testing.assert_allclose(a1[:20], al, rtol=0, atol=1e-11 * np.abs(al).max())
        np.testing.assert_allclose(b1[:20], be, rtol=0, atol=1e-11 * np.abs(al).max())


# ---- per-bond plans: more distinct couplings than the block path's classes ---------------

def randj_ring(N, seed, j2=-0.4):
    inst = W.small_ring(N, -1.0, j2)
    return inst, np.random.default_rng(seed).uniform(-1.3, -0.5, inst.n_bonds)


@pytest.mark.parametrize("jit", ["1", "0"])
@pytest.mark.parametrize("N,seed", [(12, 1), (16, 2), (20, 3), (24, 4)])
def test_perbond_matvec_vs_oracle(hm, N, seed, jit, monkeypatch):
    """Every bond its own coupling: the specialised per-bond block kernel (jit=1) and the
    general row kernel it falls back to without run-time compilation (jit=0), FP64 and FP32."""
    monkeypatch.setenv("HM_JIT", jit)
    inst, J = randj_ring(N, seed)
    b = hm.Basis(N, 1, 0)
    ob = oracle.Basis(N, 1, N // 2)
    bl = hm.BondList.make(inst.u, inst.v, J)
    obl = oracle.Bonds(inst.u, inst.v, J)
    x = oracle.start_uniform(7, b.dim)
    ref = ob.matvec(obl, x)
    y = hm.matvec(b, bl, torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, ref) <= TOL_F64
    x32 = x.astype(np.float32)
    ref32 = ob.matvec(obl, x32.astype(np.float64))
    y32 = hm.matvec(b, bl, torch.from_numpy(x32).cuda()).cpu().numpy().astype(np.float64)
    assert rel(y32, ref32) <= TOL_F32


@pytest.mark.parametrize("parity", [1, -1])
def test_perbond_flip_matvec_vs_oracle(hm, parity):
    inst, J = randj_ring(20, 6)
    b = hm.Basis(20, 1, 0, parity=parity)
    ob = oracle.Basis(20, 1, 10)
    x = oracle.start_uniform(8, b.dim)
    ref = oracle.flip_matvec(ob, oracle.Bonds(inst.u, inst.v, J), x, parity)
    y = hm.matvec(b, hm.BondList.make(inst.u, inst.v, J), torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, ref) <= TOL_F64


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_perbond_lanczos_vs_oracle(hm, dtype):
    """N = 20 ring with 40 distinct couplings: the Lanczos product runs the specialised
    per-bond kernel; alpha, beta of the first steps and E0 against the oracle."""
    inst, J = randj_ring(20, 9)
    b = hm.Basis(20, 1, 0)
    ob = oracle.Basis(20, 1, 10)
    bl = hm.BondList.make(inst.u, inst.v, J)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    run = hm.LanczosRun(b, bl, 10, seed=4, dtype=tdt)
    assert run.kernel_name() == ("k_blk_lz64_jit" if dtype == "f64" else "k_blk_lz32_jit")
    run.close()
    res = hm.lanczos_run(b, bl, 200, seed=4, n_ritz=1, dtype=tdt)
    al, be = ob.lanczos(oracle.Bonds(inst.u, inst.v, J), oracle.start_uniform(4, b.dim), 200)
    e_ref = oracle.tridiag_lowest(al, be, 1)[0]
    if dtype == "f64":
        np.testing.assert_allclose(res.alpha[:20], al[:20], rtol=0, atol=1e-12 * np.abs(al).max())
        np.testing.assert_allclose(res.beta[:20], be[:20], rtol=0, atol=1e-12 * np.abs(al).max())
        assert abs(res.ritz[0] - e_ref) <= TOL_E0 * abs(e_ref)
    else:
        assert abs(res.ritz[0] - e_ref) <= 1e-6 * abs(e_ref)


def test_matvec_kernel_name_dispatch(hm):
    """The kernel matvec takes: block kernel (few couplings), block kernel compiled for the
    bond list (per-bond couplings), general row kernel (s = 1, or several vectors)."""
    inst, J = randj_ring(16, 2)
    b = hm.Basis(16, 1, 0)
    assert hm.matvec_kernel_name(b, hm.bonds_of(W.ring16())) == "k_blk_matvec"
    assert hm.matvec_kernel_name(b, hm.BondList.make(inst.u, inst.v, J)) == "k_blk_matvec_jit"
    assert hm.matvec_kernel_name(b, hm.bonds_of(W.ring16()), nvec=2) == "k_matvec"
    s1 = W.s1_random_graph(10, 21)
    assert hm.matvec_kernel_name(hm.Basis(10, 2, 0), hm.bonds_of(s1)) == "k_matvec"


@pytest.mark.parametrize("K", [11, 13])
def test_block_split_override(hm, K, monkeypatch):
    """HM_BLK_K moves the block split: more blocks (2^(N-K)) with fewer rows each.  The
    workspace sizes its per-block partials by the same split, and the Lanczos coefficients
    agree with the default split's to rounding."""
    inst = W.small_ring(24, -1.0, -0.5)
    b = hm.Basis(24, 1, 0)
    ref = hm.lanczos_run(b, hm.bonds_of(inst), 30, seed=6, n_ritz=1)
    monkeypatch.setenv("HM_BLK_K", str(K))
    b2 = hm.Basis(24, 1, 0)
    res = hm.lanczos_run(b2, hm.bonds_of(inst), 30, seed=6, n_ritz=1)
    np.testing.assert_allclose(res.alpha, ref.alpha, rtol=0, atol=1e-13)
    np.testing.assert_allclose(res.beta, ref.beta, rtol=0, atol=1e-13)


@pytest.mark.parametrize("N,extra", [(20, 0), (22, 0), (22, 5)])
def test_bond_corr_block_path(hm, N, extra):
    """Sectors of >= 100k rows: the bond correlations run through the block kernels compiled
    per chunk of 16 bonds (40-49 bonds: 3-4 chunks, the last one partial), FP64 and FP32
    inputs, against the oracle; extra bonds between distant sites add long exchanges."""
    inst = W.small_ring(N, -1.0, -0.5)
    rng = np.random.default_rng(N + extra)
    u, v = list(inst.u), list(inst.v)
    for _ in range(extra):
        a = int(rng.integers(0, N))
        u.append(a); v.append((a + N // 2 - 1) % N)
    u, v = np.array(u, np.int32), np.array(v, np.int32)
    J = rng.uniform(-1.3, -0.5, len(u))
    b = hm.Basis(N, 1, 0)
    ob = oracle.Basis(N, 1, N // 2)
    g, x = oracle.start_uniform(8, b.dim), oracle.start_uniform(9, b.dim)
    ref = ob.bond_corr(oracle.Bonds(u, v, J), g, x)
    got = hm.bond_corr(b, hm.BondList.make(u, v, J), torch.from_numpy(g).cuda(), torch.from_numpy(x).cuda())
    np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())
    g32, x32 = g.astype(np.float32), x.astype(np.float32)
    ref32 = ob.bond_corr(oracle.Bonds(u, v, J), g32.astype(np.float64), x32.astype(np.float64))
    got32 = hm.bond_corr(b, hm.BondList.make(u, v, J), torch.from_numpy(g32).cuda(), torch.from_numpy(x32).cuda())
    np.testing.assert_allclose(got32.cpu().numpy(), ref32, rtol=1e-5, atol=1e-5 * np.abs(ref32).max())


@pytest.mark.parametrize("two_m", [0, 4])
def test_s1_block_path(hm, two_m, monkeypatch):
    """s = 1 FP32 products through the s = 1 block kernels (N = 14 random 4-regular graph):
    rows of the kernel specialised to the bonds and of the generic one (HM_JIT=0) against
    the oracle, the Lanczos kernel names, and E0 against the oracle's FP64 run."""
    inst = W.s1_random_graph(14, 5)
    b = hm.Basis(14, 2, two_m)
    ob = oracle.Basis(14, 2, 14 - two_m // 2)
    bl = hm.bonds_of(inst)
    x32 = oracle.start_uniform(4, b.dim).astype(np.float32)
    ref = ob.matvec(obonds(inst), x32.astype(np.float64))
    for jit, name in (("1", "k_s1_mv_jit"), ("0", "k_s1_mv")):
        monkeypatch.setenv("HM_JIT", jit)
        assert hm.matvec_kernel_name(b, bl, dtype=torch.float32) == name
        y = hm.matvec(b, bl, torch.from_numpy(x32).cuda()).cpu().numpy().astype(np.float64)
        assert rel(y, ref) <= TOL_F32
        run = hm.LanczosRun(b, bl, 5, seed=3, dtype=torch.float32)
        assert run.kernel_name() == name.replace("mv", "lz32")
        run.close()
    monkeypatch.setenv("HM_JIT", "1")
    res = hm.lanczos_run(b, bl, 150, seed=3, n_ritz=1, dtype=torch.float32)
    al, be = ob.lanczos(obonds(inst), oracle.start_uniform(3, b.dim), 150)
    e_ref = oracle.tridiag_lowest(al, be, 1)[0]
    assert abs(res.ritz[0] - e_ref) <= 1e-6 * abs(e_ref)


@pytest.mark.parametrize("n,two_m", [(6, 0), (8, 0), (10, 2), (12, 0), (12, 4), (14, 6)])
def test_s1_lanczos_f64_block_path(hm, n, two_m, monkeypatch):
    """FP64 s = 1 Lanczos through the block product specialised to the bonds (exact int128
    row sums of integer-scaled couplings): the first 20 coefficients against the oracle's
    FP64 run to 1e-12, and the same run on the general row kernel (HM_JIT=0).  (Later
    coefficients of two valid runs drift apart by amplified rounding: at N = 6, dim 141,
    step 28 differs by 4e-9.)"""
    inst = W.s1_random_graph(n, 100 + n)
    b = hm.Basis(n, 2, two_m)
    ob = oracle.Basis(n, 2, n - two_m // 2)
    bl = hm.bonds_of(inst)
    steps = min(20, b.dim - 1)
    al, be = ob.lanczos(obonds(inst), oracle.start_uniform(9, b.dim), steps)
    m = len(al)
    for jit, name in (("1", "k_s1_lz64_jit"), ("0", "k_lz_matvec")):
        monkeypatch.setenv("HM_JIT", jit)
        run = hm.LanczosRun(b, bl, steps, seed=9)
        assert run.kernel_name() == name
        run.step(m)
        ga, gb, _ = run.read()
        run.close()
        np.testing.assert_allclose(ga[:m], al, rtol=0, atol=1e-12 * np.abs(al).max())
        np.testing.assert_allclose(gb[:m - 1], be[:m - 1], rtol=0, atol=1e-12 * np.abs(al).max())
    monkeypatch.setenv("HM_JIT", "1")


def test_s1_full_size_rows_and_first_steps(hm):
    """The s = 1, N = 20 sector (377,379,369 rows) of the s = 1 benchmark workload: sampled
    rows of the FP32 block product against the oracle one by one; the first FP64 Lanczos
    coefficients of the block product, in the launch configuration the benchmark times,
    against alpha_1, beta_1, alpha_2 formed from the general FP64 row kernel, whose
    sampled rows match the oracle to 1e-12."""
    inst = W.s1_random_graph()
    b = hm.Basis(20, 2, 0)
    ob = oracle.Basis(20, 2, 20)
    bl = hm.bonds_of(inst)
    ob_b = obonds(inst)
    x = oracle.start_uniform(inst.seed, b.dim)
    xt = torch.from_numpy(x).cuda()
    rng = np.random.default_rng(11)
    starts = [0, b.dim - 256] + [int(r) for r in rng.integers(0, b.dim - 256, 6)]
    # FP32 rows of the block product
    assert hm.matvec_kernel_name(b, bl, dtype=torch.float32) == "k_s1_mv_jit"
    x32 = xt.float()
    y32 = hm.matvec(b, bl, x32)
    x32h = x32.double().cpu().numpy()
    for r0 in starts:
        ref = ob.matvec_rows(ob_b, x32h, r0, r0 + 256)
        assert rel(y32[r0:r0 + 256].double().cpu().numpy(), ref) <= TOL_F32
    del y32, x32, x32h
    # FP64: general row kernel, checked on samples, then alpha_1, beta_1, alpha_2
    y = hm.matvec(b, bl, xt)
    for r0 in starts[:4]:
        assert rel(y[r0:r0 + 256].cpu().numpy(), ob.matvec_rows(ob_b, x, r0, r0 + 256)) <= TOL_F64
    nx = torch.linalg.vector_norm(xt)
    q1 = xt / nx
    y = y / nx
    a1 = float(torch.dot(q1, y))
    w = y - a1 * q1
    b1 = float(torch.linalg.vector_norm(w))
    q2 = w / b1
    del w, y
    a2 = float(torch.dot(q2, hm.matvec(b, bl, q2)))
    del q2, q1
    run = hm.LanczosRun(b, bl, 4, v0=xt)
    assert run.kernel_name() == "k_s1_lz64_jit"
    run.step(2)
    ga, gb, _ = run.read()
    run.close()
    scale = max(abs(a1), abs(a2))
    assert abs(ga[0] - a1) <= 1e-12 * scale and abs(gb[0] - b1) <= 1e-12 * scale
    assert abs(ga[1] - a2) <= 1e-12 * scale


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_four_class_triangles_vs_oracle(hm, dtype):
    """NN and NNN bonds with four couplings in integer ratios spread over both kinds (the
    target tables' triangles then mix classes or are skipped): the Lanczos coefficients of the
    block product against the oracle's (FP64 to 1e-11, FP32 to FP32 accuracy), N = 18."""
    n = 18
    inst = W.small_ring(n, -1.0, -0.5)
    J = [(-1.0, -0.5, -0.25, -0.75)[(3 * i + i // 5) % 4] for i in range(inst.n_bonds)]
    bonds = hm.BondList.make(inst.u, inst.v, J)
    b = hm.Basis(n, 1, 0)
    dt = torch.float64 if dtype == "f64" else torch.float32
    run = hm.LanczosRun(b, bonds, 20, seed=3, dtype=dt)
    assert run.kernel_name().startswith("k_blk_lz"), run.kernel_name()
    run.step(20)
    al, be, _ = run.read()
    run.close()
    ob = oracle.Basis(n, 1, n // 2)
    oal, obe = ob.lanczos(oracle.Bonds(inst.u, inst.v, J), oracle.start_uniform(3, ob.dim), 20)
    tol = 1e-11 if dtype == "f64" else 2e-5
    np.testing.assert_allclose(al, oal, rtol=0, atol=tol * np.abs(oal).max())
    np.testing.assert_allclose(be, obe, rtol=0, atol=tol * np.abs(oal).max())


@pytest.mark.parametrize("N,j2", [(20, -0.5), (24, -0.25)])
def test_block_rows_correctly_rounded(hm, N, j2, monkeypatch):
    """FP64 block rows with integer-ratio couplings and a power-of-two unit (J2 = J1/2,
    J1/4) are the exact row sums of Eq. (E-2-1) rounded once to binary64.  With
    x_i = k_i 2^-40 (|k_i| < 2^40), which the fixed-point copy holds exactly, each sampled
    row of y = H x equals, bit for bit, the correctly rounded exact rational sum
    sum_b -J_b/4 (+-1) x_i + sum over the allowed exchanges of -J_b/2 x_t (s = 1/2), built
    from the oracle's decode and encode; with and without run-time compilation (class plans
    run the block kernel either way)."""
    from fractions import Fraction
    inst = W.small_ring(N, -1.0, j2)
    b = hm.Basis(N, 1, 0)
    ob = oracle.Basis(N, 1, N // 2)
    bl = hm.bonds_of(inst)
    rng = np.random.default_rng(N)
    k = rng.integers(-(1 << 40) + 1, 1 << 40, size=b.dim, dtype=np.int64)
    x = k.astype(np.float64) * 2.0 ** -40
    assert np.array_equal((x * 2.0 ** 40).astype(np.int64), k)
    rows = np.unique(np.concatenate([rng.integers(0, b.dim, 300), [0, b.dim - 1]]))
    want = {}
    for i in rows:
        i = int(i)
        d = [int(a) for a in ob.decode(i)]
        acc = Fraction(0)
        for p, q, J in zip(inst.u, inst.v, inst.J):
            p, q, J = int(p), int(q), Fraction(float(J))
            if d[p] == d[q]:
                acc += -J / 4 * Fraction(int(k[i]), 1 << 40)
            else:
                acc += J / 4 * Fraction(int(k[i]), 1 << 40)
                t = list(d)
                t[p], t[q] = d[q], d[p]
                acc += -J / 2 * Fraction(int(k[ob.encode(t)]), 1 << 40)
        want[i] = float(acc)              # int / int true division: correctly rounded
    xt = torch.from_numpy(x).cuda()
    for jit in ("1", "0"):
        monkeypatch.setenv("HM_JIT", jit)
        name = hm.matvec_kernel_name(b, bl)
        assert name.startswith("k_blk_matvec"), name
        y = hm.matvec(b, bl, xt).cpu().numpy()
        got = y[rows]
        exp = np.array([want[int(i)] for i in rows])
        bad = np.nonzero(got.view(np.uint64) != exp.view(np.uint64))[0]
        assert bad.size == 0, (name, [(int(rows[j]), got[j], exp[j]) for j in bad[:5]])
    monkeypatch.setenv("HM_JIT", "1")
