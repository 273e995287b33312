"""The C-ABI library loads and exports every entry point that include/wproj.h
declares (no compute calls: this runs without a GPU)."""
import os
import re
import ctypes

import pytest

from paper_1307_3424_gb300 import wproj

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "wproj.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wproj_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("wproj_build_kernels", "wproj_phi", "wproj_phi_adj", "wproj_solve_bpdn"):
        assert must in names


@pytest.fixture(scope="module")
def built_lib():
    if not os.path.exists(wproj.LIB_PATH):
        from paper_1307_3424_gb300 import _build
        _build.build()
    return ctypes.CDLL(wproj.LIB_PATH)


def test_library_exports_every_declared_symbol(built_lib):
    for name in declared_symbols():
        assert hasattr(built_lib, name), name


def test_binding_covers_the_header():
    assert set(declared_symbols()) <= set(wproj.EXPORTED)


def test_last_error_and_version_callable(built_lib):
    L = wproj.lib()
    assert b"sm_103a" in L.wproj_version()
    p = wproj.dr_defaults()
    assert p.iters == 50 and p.inner_iters == 10 and p.power_iters == 100
    assert abs(p.gamma_frac - 1e-2) < 1e-15 and p.lambda_ == 1.0


def test_invalid_plan_arguments_rejected_on_host(built_lib):
    # argument validation happens before any device work
    L = wproj.lib()
    h = ctypes.c_void_p()
    for d in (wproj.GridDesc(12, 4, 0.03, 0, 0, 0, 0),     # N not a power of two
              wproj.GridDesc(64, 5, 0.03, 0, 0, 0, 0),     # W
              wproj.GridDesc(64, 4, -1.0, 0, 0, 0, 0),     # fov
              wproj.GridDesc(64, 4, 0.03, 0, 0, 48, 0),    # box
              wproj.GridDesc(64, 4, 0.9, 0, 0, 0, 0)):     # 1 - 2L^2 < 0
        assert L.wproj_plan_create(ctypes.byref(h), ctypes.byref(d)) == wproj.ERR_INVALID_ARG
        assert L.wproj_last_error()


def test_daubechies_taps_on_the_host_match_oracle(built_lib):
    # the library's tap generator runs on the host (spectral factorisation in
    # double): its taps against the oracle's for every supported order
    import numpy as np
    from oracle import wavelet_oracle as W
    for p in range(1, 11):
        h = np.array(wproj.daubechies_taps(p))
        assert np.allclose(h, W.daubechies_taps(p), rtol=0, atol=1e-12), p
    for p in (0, 11):
        with pytest.raises(wproj.WprojError):
            wproj.daubechies_taps(p)


def test_dr_defaults_select_the_dirac_basis(built_lib):
    p = wproj.dr_defaults()
    assert p.psi == 0 and p.psi_levels == 4
