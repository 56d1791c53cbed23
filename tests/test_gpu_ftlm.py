"""GPU parity of the batched finite-temperature Lanczos driver (ftlm_run) against the CPU
oracle.  The GPU keeps the Lanczos vectors in FP32 (reductions double-float/double), the
oracle in FP64, so Ritz values agree to ~1e-5 relative and Z, E to ~1e-4.

A sector no larger than the step count would exhaust its Krylov space; both sides
diagonalise it exactly (FP64), so its theta are the exact eigenvalues and its quadrature
sums sum_k tau_k f(theta_k) are exact (individual tau_k of degenerate eigenvalues are not
unique, their sums are)."""
import math

import numpy as np
import pytest

import oracle
from paper_0706_3293_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TEMPS = [0.3, 1.0, 3.0, 10.0]


@pytest.fixture(scope="module")
def hm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0706_3293_gb300 import build
    build.build()
    from paper_0706_3293_gb300 import api
    return api


def oracle_ftlm(inst, R, steps, seed, sectors=None):
    per = []
    out = {}
    for A in range(inst.n_sites + 1):
        b = oracle.Basis(inst.n_sites, 1, A)
        if sectors is not None and A not in sectors:
            continue
        res = oracle.ftlm_sector(b, oracle.Bonds(inst.u, inst.v, inst.J), seed, R, steps)
        out[A] = res
        per.append((b.dim, res))
    return out, per


@pytest.fixture(scope="module")
def small_case(hm):
    inst = W.small_ring(12, -1.0, -0.3)
    R, steps, seed = 4, 30, 77
    gpu = hm.ftlm_run(12, hm.bonds_of(inst), R, steps, seed, TEMPS, vt=1)
    ora, per = oracle_ftlm(inst, R, steps, seed)
    return inst, R, steps, seed, gpu, ora, per


def ritz_residuals(al, be):
    """Residual norms beta_m |s_mk| of the lowest and highest Ritz pair of the oracle's
    m-step tridiagonal (beta_m is the coupling to the next, unused, Lanczos vector)."""
    from scipy.linalg import eigh_tridiagonal
    m = len(al)
    if m == 1:
        return abs(be[0]) if len(be) else 0.0, abs(be[0]) if len(be) else 0.0
    _, c = eigh_tridiagonal(al, be[: m - 1])
    bm = abs(be[m - 1]) if len(be) >= m else 0.0
    return bm * abs(c[m - 1, 0]), bm * abs(c[m - 1, -1])


def check_vector(gpu, A, r, dim, steps, ora_run, tol_rel=2e-5):
    th, tau, al, be = ora_run
    m = int(gpu.mlen[A, r])
    if dim <= steps:
        assert m == dim
        np.testing.assert_allclose(np.sort(gpu.theta[A, r, :m]), th, rtol=0, atol=1e-10 * max(1.0, np.abs(th).max()))
        tol_rel = 1e-10
        res_lo = res_hi = 0.0
    else:
        assert m == len(al), (A, r, m, len(al))
        res_lo, res_hi = ritz_residuals(al, be)
    gth = gpu.theta[A, r, :m]
    gtau = gpu.tau[A, r, :m]
    assert abs(gtau.sum() - 1.0) < 1e-6
    # an extreme Ritz value lies within its residual beta_m |s_mk| of an eigenvalue; one
    # that has not converged after `steps` may differ between FP32 and FP64 runs by up to
    # about that residual
    assert abs(gth.min() - th[0]) <= max(tol_rel * max(1.0, abs(th[0])), 2 * res_lo), (A, r)
    assert abs(gth.max() - th[-1]) <= max(tol_rel * max(1.0, abs(th[-1])), 2 * res_hi), (A, r)
    for T in TEMPS:
        qg = float(np.sum(gtau * np.exp(-(gth - th[0]) / T)))
        qo = float(np.sum(tau * np.exp(-(th - th[0]) / T)))
        assert abs(qg - qo) <= (1e-10 if dim <= steps else 1e-4) * qo, (A, r, T, qg, qo)


def test_ftlm_krylov_lengths_and_ritz(small_case):
    inst, R, steps, seed, gpu, ora, per = small_case
    for A, res in ora.items():
        dim = math.comb(inst.n_sites, A)
        for r in range(R):
            check_vector(gpu, A, r, dim, steps, res[r])
    assert np.all(gpu.mlen[:, R:] == 0)


def test_ftlm_thermodynamics(small_case):
    inst, R, steps, seed, gpu, ora, per = small_case
    Z, E, eref = oracle.ftlm_thermo(per, TEMPS)
    assert abs(gpu.e_ref - eref) <= 2e-5 * abs(eref)
    for i, T in enumerate(TEMPS):
        z_gpu = gpu.Z[i] * math.exp(-(gpu.e_ref - eref) / T)      # same reference energy
        assert abs(z_gpu - Z[i]) <= 1e-4 * Z[i], (T, z_gpu, Z[i])
        assert abs(gpu.E[i] - E[i]) <= 1e-4 * max(1.0, abs(E[i])), (T, gpu.E[i], E[i])


@pytest.mark.parametrize("vt", [2, 4, 0])
def test_ftlm_tilings_agree(hm, small_case, vt):
    inst, R, steps, seed, gpu, ora, per = small_case
    other = hm.ftlm_run(12, hm.bonds_of(inst), R, steps, seed, TEMPS, vt=vt)
    assert other.vt in (1, 2, 4) and (vt == 0 or other.vt == vt)
    assert np.array_equal(other.mlen, gpu.mlen)
    np.testing.assert_allclose(other.Z, gpu.Z, rtol=1e-5)
    np.testing.assert_allclose(other.E, gpu.E, rtol=1e-5, atol=1e-6)


def test_ftlm_high_temperature_limit(hm):
    """sum_j tau_j = 1 makes Z(T -> infinity) the number of states, 2^N."""
    inst = W.small_ring(14, -1.0, -0.5)
    res = hm.ftlm_run(14, hm.bonds_of(inst), 8, 20, 5, [1e7])
    assert abs(res.Z[0] * math.exp(-res.e_ref / 1e7) / 2 ** 14 - 1.0) < 1e-5


def test_ftlm_ring24_config(hm):
    """The N = 24 J1-J2 ring (J2 = -0.3), all 25 sectors, R = 32 +-1 vectors, 80 steps in
    one launch: small sectors against the oracle vector by vector, a middle sector's first
    vector, and the mirror symmetry A <-> N - A of the converged ground energies."""
    inst = W.ftlm_ring24()
    R, steps, seed = 32, 80, inst.seed
    gpu = hm.ftlm_run(24, hm.bonds_of(inst), R, steps, seed, TEMPS)
    assert gpu.vt in (1, 2, 4)
    ora, _ = oracle_ftlm(inst, R, steps, seed, sectors={0, 1, 2, 22, 23, 24})
    for A, res in ora.items():
        dim = math.comb(24, A)
        for r in range(R):
            check_vector(gpu, A, r, dim, steps, res[r])
    # sector A = 6 (dim 134,596), first start vector
    b = oracle.Basis(24, 1, 6)
    v0 = oracle.start_pm1(oracle.stream_seed(seed, 6, 0), b.dim)
    al, be = b.lanczos(oracle.Bonds(inst.u, inst.v, inst.J), v0, steps)
    e_ref6 = oracle.tridiag_lowest(al, be, 1)[0]
    m = int(gpu.mlen[6, 0])
    assert abs(np.sort(gpu.theta[6, 0, :m])[0] - e_ref6) <= 1e-5 * abs(e_ref6)
    # lowest Ritz values of mirror sectors (both converged after 80 steps in small sectors)
    for A in range(0, 6):
        lo_a = min(np.sort(gpu.theta[A, r, :gpu.mlen[A, r]])[0] for r in range(R))
        lo_b = min(np.sort(gpu.theta[24 - A, r, :gpu.mlen[24 - A, r]])[0] for r in range(R))
        assert abs(lo_a - lo_b) <= 1e-4 * max(1.0, abs(lo_a))
    assert np.all(np.isfinite(gpu.Z)) and np.all(gpu.Z > 0)


def test_ftlm_barrier_gives_up_and_device_stays_usable(hm, monkeypatch):
    """The persistent kernel's grid barriers wait a bounded time.  With the limit set to
    0 ns the first wait gives up: the kernel sets its abort flag, every CTA returns, and
    ftlm_run reports HM_ETIMEOUT (no fault, no hang).  A normal run right after it on the
    same device gives the same result as before."""
    from paper_0706_3293_gb300 import _capi
    inst = W.small_ring(12, -1.0, -0.3)
    ok = hm.ftlm_run(12, hm.bonds_of(inst), 4, 20, 3, [1.0], vt=1)
    monkeypatch.setenv("HM_FT_BARRIER_NS", "0")
    with pytest.raises(_capi.HMError) as ei:
        hm.ftlm_run(12, hm.bonds_of(inst), 4, 20, 3, [1.0], vt=1)
    assert ei.value.code == _capi.HM_ETIMEOUT
    monkeypatch.delenv("HM_FT_BARRIER_NS")
    again = hm.ftlm_run(12, hm.bonds_of(inst), 4, 20, 3, [1.0], vt=1)
    assert again.Z[0] == ok.Z[0] and again.E[0] == ok.E[0]
    torch.cuda.synchronize()
