"""CPU checks of the C ABI: libhm.so builds, loads and exports every symbol of
include/hm.h; host-only entry points validate their arguments.  No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_0706_3293_gb300 import build
    build.build()
    from paper_0706_3293_gb300 import _capi
    return _capi.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "hm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)))


def test_every_header_symbol_is_exported(lib):
    from paper_0706_3293_gb300 import _capi
    names = header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(_capi.EXPORTS) == names


def test_dimension_query(lib):
    from paper_0706_3293_gb300 import api
    assert api.basis_dim_query(16, 1, 0) == 12870
    assert api.basis_dim_query(32, 1, 0) == 601080390
    assert api.basis_dim_query(20, 2, 0) == 377379369
    assert api.basis_dim_query(20, 2, 26) == 484500          # Fig. F-A vector length (s=1, M=13)
    assert api.basis_dim_query(24, 1, 24) == 1                # fully polarised


@pytest.mark.parametrize("args,code", [((16, 1, 1), -2), ((16, 1, 34), -2), ((16, 0, 0), -1),
                                       ((0, 1, 0), -1), ((65, 1, 1), -1), ((40, 2, 0), -1)])
def test_dimension_query_errors(lib, args, code):
    from paper_0706_3293_gb300 import api, _capi
    with pytest.raises(_capi.HMError) as ei:
        api.basis_dim_query(*args)
    assert ei.value.code == code
    assert len(str(ei.value)) > 8


def test_bonds_check(lib):
    from paper_0706_3293_gb300 import api, _capi
    api.bonds_check(4, api.BondList.make([0, 1], [1, 3], [1.0, -0.5]))
    for u, v, J in [([0], [0], [1.0]), ([0], [4], [1.0]), ([-1], [1], [1.0]),
                    ([0], [1], [float("nan")])]:
        with pytest.raises(_capi.HMError) as ei:
            api.bonds_check(4, api.BondList.make(u, v, J))
        assert ei.value.code == _capi.HM_EINVAL
    big = api.BondList.make([0] * 513, [1] * 513, [1.0] * 513)
    with pytest.raises(_capi.HMError):
        api.bonds_check(4, big)


def test_last_error_is_per_call(lib):
    from paper_0706_3293_gb300 import _capi
    d = ctypes.c_int64()
    assert lib.basis_dim_query(16, 1, 3, ctypes.byref(d)) == _capi.HM_EPARITY
    assert b"magnetic" in lib.hm_last_error()


def test_sym_eigenvalues_host_solver():
    """The library's host Jacobi eigensolver (used by arnoldi_run on its Hessenberg
    matrix) against numpy's eigvalsh on symmetric parts of random and tridiagonal
    matrices; NULL and bad sizes are rejected.  No GPU involved."""
    from paper_0706_3293_gb300 import api, _capi
    rng = np.random.default_rng(4)
    for n in (1, 2, 5, 33, 90):
        a = rng.standard_normal((n, n))
        ref = np.linalg.eigvalsh(0.5 * (a + a.T))
        np.testing.assert_allclose(api.sym_eigenvalues(a), ref, rtol=0, atol=1e-12 * max(1.0, np.abs(ref).max()))
    t = np.diag(rng.standard_normal(40)) + np.diag(np.full(39, 0.5), 1) + np.diag(np.full(39, 0.5), -1)
    np.testing.assert_allclose(api.sym_eigenvalues(t), np.linalg.eigvalsh(t), rtol=0, atol=1e-13)
    L = _capi.load()
    assert L.sym_eigenvalues(0, None, None) == _capi.HM_EINVAL
