"""bond_corr_static: the adjoint for callers that cannot call cudaMalloc when they need it --
a host program that reserves its whole device-memory budget at start-up and forbids any
later allocation, or a library inside a framework whose allocator owns all device memory.
It allocates nothing: it runs the general row kernels (no block tables built on first use,
no run-time compiled kernel) and keeps its partial sums in a fixed device array instead of
a workspace.  Its output must match bond_corr (which may take the block kernels; the sums
then differ only in rounding order) on two consecutive calls, which share that array.  Kept
in its own file, collected last."""
import ctypes

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
    from paper_0706_3293_gb300 import api, _capi
    return api, _capi


def _static_call(capi, basis, bonds, g, x, dtype):
    out = torch.full((len(bonds),), float("nan"), dtype=torch.float64, device="cuda")
    rc = capi.load().bond_corr_static(
        basis.handle, len(bonds), bonds.u.ctypes.data_as(ctypes.c_void_p),
        bonds.v.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(g.data_ptr()),
        ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), dtype,
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    capi.check(rc)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("case", ["ring24_randJ", "s1_rrg12_f32"])
def test_bond_corr_static_matches_workspace_version(hm, case):
    api, capi = hm
    if case == "ring24_randJ":
        inst, tdt, dt = W.ring24_random_j(), torch.float64, capi.HM_F64
    else:
        inst, tdt, dt = W.s1_random_graph_small(), torch.float32, capi.HM_F32
    b = api.Basis(inst.n_sites, inst.two_s, inst.two_m)
    bonds = api.bonds_of(inst)
    ref = None
    for call in range(2):     # two calls in a row share (and overwrite) the static array
        g = torch.from_numpy(oracle.start_uniform(40 + call, b.dim)).to(tdt).cuda()
        x = torch.from_numpy(oracle.start_uniform(60 + call, b.dim)).to(tdt).cuda()
        got = _static_call(capi, b, bonds, g, x, dt)
        ref = api.bond_corr(b, bonds, g, x).cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
        assert np.all(np.isfinite(got))


def test_bond_corr_static_rejects_oversize(hm):
    api, capi = hm
    pairs = [(a, c) for a in range(20) for c in range(a + 1, 20)]   # 190 bonds x 722 blocks > 1 MiB
    bonds = api.BondList.make([p[0] for p in pairs], [p[1] for p in pairs], [1.0] * len(pairs))
    b = api.Basis(20, 1, 0)
    g = torch.zeros(b.dim, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.HMError) as ei:
        _static_call(capi, b, bonds, g, g, capi.HM_F64)
    assert ei.value.code == capi.HM_EINVAL and "static" in str(ei.value)
