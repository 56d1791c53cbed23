"""GPU: ground-state correlations <psi0| s_u.s_v |psi0> of arbitrary site pairs (the
ground-state quantities the paper's cited applications use, Sec. 1), against closed forms,
sum rules and the oracle."""
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


def test_four_site_ring_closed_form(hm):
    """H = sum s_i.s_{i+1} on the 4-site ring (J = -1): E0 = -2 in a singlet.  Translation
    invariance gives <s_i.s_{i+1}> = E0 / 4 = -1/2, and S = 0 gives
    sum_{i,j} <s_i.s_j> = 4 (3/4) + 8 (-1/2) + 4 <s_0.s_2> = 0, so <s_0.s_2> = 1/4."""
    inst = W.small_ring(4, -1.0)
    b = hm.Basis(4, 1, 0)
    e0, corr, rc = hm.ground_state_correlations(b, hm.bonds_of(inst), [0, 0, 0, 1], [1, 2, 3, 3], 6, seed=3)
    assert rc >= 0
    assert abs(e0 + 2.0) < 1e-12
    np.testing.assert_allclose(corr, [-0.5, 0.25, -0.5, 0.25], rtol=0, atol=1e-12)   # (1, 3): distance 2


def test_ring16_sum_rule_and_translation(hm):
    """N = 16 antiferromagnetic ring, M = 0: the ground state is a singlet (Lieb-Mattis), so
    sum_r C(r) = 0 with C(0) = 3/4; C(r) = C(N - r) by reflection; E0 = N C(1)."""
    inst = W.ring16()
    b = hm.Basis(16, 1, 0)
    r = np.arange(1, 16)
    e0, C, rc = hm.ground_state_correlations(b, hm.bonds_of(inst), np.zeros(15, np.int32), r, 200, seed=5)
    assert rc >= 0
    assert abs(0.75 + C.sum()) < 1e-9
    np.testing.assert_allclose(C, C[::-1], rtol=0, atol=1e-9)
    assert abs(e0 - 16 * C[0]) < 1e-9 * abs(e0)
    assert C[0] < 0 < C[1]                # antiferromagnetic order: alternating signs


@pytest.mark.parametrize("case", ["j1j2_n14", "s1_n10"])
def test_correlations_vs_oracle(hm, case):
    """Pairs inside and outside the coupled bonds against the oracle's ground state (same
    start vector and steps): bond_corr(psi0, psi0) on the oracle's psi0."""
    if case == "j1j2_n14":
        inst = W.small_ring(14, -1.0, -0.3)
        J = np.random.default_rng(12).uniform(-1.2, -0.8, inst.n_bonds)
        steps, pu, pv = 120, [0, 0, 0, 0, 3, 5], [1, 2, 4, 7, 10, 6]
    else:
        inst = W.s1_random_graph(10, 21)
        J = inst.J
        steps, pu, pv = 120, [0, 1, 2, 4], [5, 7, 9, 8]
    b = hm.Basis(inst.n_sites, inst.two_s, inst.two_m)
    ob = oracle.Basis(inst.n_sites, inst.two_s, inst.A)
    bl = hm.BondList.make(inst.u, inst.v, J)
    e0, corr, rc = hm.ground_state_correlations(b, bl, pu, pv, steps, seed=21)
    assert rc >= 0
    oe0, psi, _ = oracle.ground_state(ob, oracle.Bonds(inst.u, inst.v, J), oracle.start_uniform(21, b.dim), steps)
    pairs = oracle.Bonds(np.array(pu, np.int32), np.array(pv, np.int32), np.zeros(len(pu)))
    ref = ob.bond_corr(pairs, psi, psi)
    assert abs(e0 - oe0) <= 1e-10 * abs(oe0)
    np.testing.assert_allclose(corr, ref, rtol=0, atol=1e-8)


def test_correlations_reject_bad_pairs(hm):
    inst = W.small_ring(8, -1.0)
    b = hm.Basis(8, 1, 0)
    with pytest.raises(Exception):
        hm.ground_state_correlations(b, hm.bonds_of(inst), [0], [0], 20)
