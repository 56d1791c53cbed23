"""GPU: the spin-flip parity blocks of the s = 1/2 sector M = 0 (basis_build_flip) against
the oracle's flip_matvec (the first half of H applied to [x, p reversed(x)]), dense
spectra, the Majumdar-Ghosh point at full size, and the calls that refuse such a basis."""
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


def case(N, j2, seed):
    """Ring with NN and NNN bonds; seed: couplings drawn from four random values (the block
    kernels, which alone take a spin-flip basis, handle up to four coupling classes)."""
    inst = W.small_ring(N, -1.0, j2)
    if seed is None:
        return inst, inst.J
    rng = np.random.default_rng(seed)
    vals = rng.uniform(-1.3, -0.4, 4)
    return inst, vals[rng.integers(0, 4, inst.n_bonds)]


@pytest.mark.parametrize("parity", [1, -1])
@pytest.mark.parametrize("N,j2,seed", [(10, -0.3, 1), (12, -0.5, None), (16, -0.5, 4), (20, -0.3, None), (22, -0.5, 5)])
def test_flip_matvec_vs_oracle(hm, N, j2, seed, parity):
    inst, J = case(N, j2, seed)
    b = hm.Basis(N, 1, 0, parity=parity)
    ob = oracle.Basis(N, 1, N // 2)
    assert b.dim == ob.dim // 2
    bl = hm.BondList.make(inst.u, inst.v, J)
    obl = oracle.Bonds(inst.u, inst.v, J)
    x = oracle.start_uniform(9, b.dim)
    ref = oracle.flip_matvec(ob, obl, x, parity)
    y = hm.matvec(b, bl, torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, ref) <= 1e-12
    x32 = x.astype(np.float32)
    ref32 = oracle.flip_matvec(ob, obl, x32.astype(np.float64), parity)
    y32 = hm.matvec(b, bl, torch.from_numpy(x32).cuda()).cpu().numpy().astype(np.float64)
    assert rel(y32, ref32) <= 1e-5


@pytest.mark.parametrize("parity", [1, -1])
def test_flip_lanczos_vs_dense(hm, parity):
    """N = 12 J1-J2 ring with random couplings: the lowest Ritz value of each parity block
    against the dense block's lowest eigenvalue, and the two blocks' minimum against the
    whole sector's."""
    inst, J = case(12, -0.4, 7)
    ob = oracle.Basis(12, 1, 6)
    obl = oracle.Bonds(inst.u, inst.v, J)
    n = ob.dim // 2
    dense = np.stack([oracle.flip_matvec(ob, obl, np.eye(n)[:, j], parity) for j in range(n)], axis=1)
    e_dense = np.linalg.eigvalsh(dense)[0]
    b = hm.Basis(12, 1, 0, parity=parity)
    res = hm.lanczos_run(b, hm.BondList.make(inst.u, inst.v, J), 200, seed=3, n_ritz=1)
    assert abs(res.ritz[0] - e_dense) <= 1e-10 * abs(e_dense)


def test_flip_blocks_hold_the_sector_ground_state(hm):
    """N = 20 ring, J2 = 0.3 J1: min over the two parity blocks = the sector's E0 (GPU
    Lanczos on the full sector); the FP32 runs agree within 1e-6."""
    inst = W.small_ring(20, -1.0, -0.3)
    bl = hm.bonds_of(inst)
    full = hm.lanczos_run(hm.Basis(20, 1, 0), bl, 200, seed=4, n_ritz=1).ritz[0]
    e = [hm.lanczos_run(hm.Basis(20, 1, 0, parity=p), bl, 200, seed=4, n_ritz=1).ritz[0] for p in (1, -1)]
    assert abs(min(e) - full) <= 1e-10 * abs(full)
    e32 = [hm.lanczos_run(hm.Basis(20, 1, 0, parity=p), bl, 200, seed=4, n_ritz=1, dtype=torch.float32).ritz[0]
           for p in (1, -1)]
    assert abs(min(e32) - full) <= 1e-6 * abs(full)


@pytest.mark.parametrize("parity", [1, -1])
def test_flip_specialised_equals_generic(hm, parity, monkeypatch):
    """The run-time specialised product and the generic block product form the same exact
    integer sums: identical alpha, beta in FP64."""
    inst = W.small_ring(20, -1.0, -0.5)
    b = hm.Basis(20, 1, 0, parity=parity)
    a = hm.lanczos_run(b, hm.bonds_of(inst), 30, seed=2, n_ritz=1)
    monkeypatch.setenv("HM_JIT", "0")
    g = hm.lanczos_run(b, hm.bonds_of(inst), 30, seed=2, n_ritz=1)
    assert np.array_equal(a.alpha, g.alpha) and np.array_equal(a.beta, g.beta)


def test_flip_codec_and_refusals(hm):
    b = hm.Basis(12, 1, 0, parity=1)
    ob = oracle.Basis(12, 1, 6)
    idx = torch.arange(b.dim, dtype=torch.int64, device="cuda")
    st = b.decode(idx)
    assert torch.equal(b.encode(st), idx)
    # the other half of the sector is not in the basis
    upper = torch.tensor([sum(int(a) << p for p, a in enumerate(ob.decode(i))) for i in (b.dim, ob.dim - 1)],
                         dtype=torch.int64, device="cuda")
    assert b.encode(upper).tolist() == [-1, -1]
    bl = hm.bonds_of(W.small_ring(12, -1.0))
    x = torch.ones(b.dim, dtype=torch.float64, device="cuda")
    with pytest.raises(Exception):
        hm.count_nnz(b, bl)
    with pytest.raises(Exception):
        hm.bond_corr(b, bl, x, x)
    with pytest.raises(Exception):
        hm.e0_grad(b, bl, 30)
    with pytest.raises(Exception):
        hm.matvec(b, bl, torch.ones(b.dim, 2, dtype=torch.float64, device="cuda"))
    for n, p in [(11, 1), (8, 1), (12, 0), (34, -1)]:
        with pytest.raises(Exception):
            hm.Basis(n, 1, 0, parity=p) if p else hm.Basis(n, 1, 0, parity=2)


@pytest.mark.slow
def test_flip_full_size_majumdar_ghosh(hm):
    """N = 32 at J2 = J1/2: the dimer ground state (16 singlets, each odd under the flip) is
    even, so the +1 block holds E0 = -12 exactly; the -1 block lies above it."""
    inst = W.j1j2_ring32()
    e = {}
    for p in (1, -1):
        b = hm.Basis(32, 1, 0, parity=p)
        assert b.dim == 300540195
        run = hm.LanczosRun(b, hm.bonds_of(inst), 150, seed=inst.seed)
        run.step(150)
        al, be, rc = run.read()
        run.close()
        e[p] = oracle.tridiag_lowest(al, be, 1)[0]
    assert abs(e[1] + 12.0) <= 1e-9 * 12.0, e
    assert e[-1] > -12.0 + 1e-6
