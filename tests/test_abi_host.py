"""CPU checks of the C-ABI library: it builds, loads, exports every entry point that
include/odwf.h declares, and its host-only logic (the optimal-weight generator and
argument validation) agrees with the oracle.  No GPU compute is called here."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1811_08095_gb300 as odwf
from oracle import zolotarev

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return odwf.load(build_if_missing=True)


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            txt = open(os.path.join(inc, fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w[\w\s\*]*?\b((?:odwf|serve)_\w+)\s*\(", txt, flags=re.M))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), "libodwf.so does not export %s" % n


def test_bounds_checked_build_exports_the_same_abi():
    """The debug variant (ODWF_BOUNDS_CHECK) is built beside the library and exports the same
    entry points; its version string says it is the checked build."""
    from paper_1811_08095_gb300 import build as b

    b.build(bounds_check=True)
    chk = ctypes.CDLL(b.LIB_CHECK)
    for n in declared_functions():
        assert hasattr(chk, n), "libodwf_check.so does not export %s" % n
    chk.odwf_version.restype = ctypes.c_char_p
    assert b"bounds-checked" in chk.odwf_version()


def test_library_is_in_tree(lib):
    assert os.path.dirname(odwf.lib_path()).startswith(ROOT)


@pytest.mark.parametrize("ns", [2, 4, 8, 16])
@pytest.mark.parametrize("variant,shifted", [(odwf.ODWF_OMEGA_SHIFTED_R5, True), (odwf.ODWF_OMEGA_PLAIN, False)])
def test_omega_matches_oracle(lib, ns, variant, shifted):
    for lmin, lmax in [(0.05, 6.0), (0.05, 6.2), (0.1, 2.5)]:
        w, dz = odwf.odwf_zolotarev_omega(ns, lmin, lmax, variant)
        wo, dzo = zolotarev.omega(ns, lmin, lmax, shifted)
        # the oracle finds the weights numerically; its accuracy falls with Ns (flat maxima)
        assert np.abs(w / wo - 1).max() < 1e-7
        assert abs(dz / dzo - 1) < 1e-6


@pytest.mark.parametrize("ns", [16, 32])
def test_omega_shifted_bound_large_ns(lib, ns):
    """Sec. 2: 0 <= 1 - S(lambda) <= 2 d_Z with R5-symmetric weights, checked directly."""
    lmin, lmax = 0.05, 6.2
    w, dz = odwf.odwf_zolotarev_omega(ns, lmin, lmax, odwf.ODWF_OMEGA_SHIFTED_R5)
    assert np.array_equal(w, w[::-1])
    lam = np.geomspace(lmin, lmax, 100001)
    T = np.ones_like(lam)
    for ws in w:
        T *= (1 - ws * lam) / (1 + ws * lam)
    one_minus_s = 1 - (1 - T) / (1 + T)
    assert one_minus_s.min() > -1e-12
    assert one_minus_s.max() <= 2 * dz * (1 + 1e-3) + 1e-14


def test_omega_invalid_arguments(lib):
    out = np.zeros(8)
    dz = ctypes.c_double()
    for args in [(7, 0.05, 6.0, 0), (0, 0.05, 6.0, 0), (8, 0.0, 6.0, 0), (8, 6.0, 0.05, 0), (8, 0.05, 6.0, 9)]:
        rc = lib.odwf_zolotarev_omega(args[0], args[1], args[2], args[3],
                                      out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(dz))
        assert rc == odwf._lib.ODWF_EINVAL
        assert lib.odwf_last_error()


def test_create_rejects_bad_sizes(lib):
    om = np.ones(8)
    h = ctypes.c_void_p()
    for dims, ns in [((3, 4, 4, 4), 8), ((4, 4, 4, 0), 8), ((4, 4, 4, 4), 6), ((4, 4, 4, 4), 64)]:
        lat = odwf._lib.odwf_lattice()
        for i in range(4):
            lat.dims[i] = dims[i]
        lat.t_antiperiodic = 1
        rc = lib.odwf_create(ctypes.byref(lat), ns, 1.3, 0.01, om.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h))
        assert rc == odwf._lib.ODWF_EINVAL, dims
    assert lib.odwf_create(None, 8, 1.3, 0.01, None, ctypes.byref(h)) == odwf._lib.ODWF_EINVAL


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without libodwf.so the binding raises instead of computing anything."""
    from paper_1811_08095_gb300 import _lib

    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "libodwf.so"))
    with pytest.raises(RuntimeError, match="no fallback"):
        _lib.load()


def test_hmc_entry_points_reject_a_null_handle(lib):
    """The HMC calls refuse a null handle with ODWF_EINVAL before touching a device."""
    E = odwf._lib.ODWF_EINVAL
    act = ctypes.c_double(0.0)
    prm = odwf._lib.odwf_solve_params()
    st = odwf._lib.odwf_solve_stats()
    en = np.zeros(2)
    assert lib.odwf_pf_force(None, None, 0.1, 0.5, ctypes.byref(prm), ctypes.byref(act), None, ctypes.byref(st),
                             None) == E
    assert b"null handle" in lib.odwf_last_error()
    assert lib.odwf_pf_heatbath(None, None, 0.1, 0.5, ctypes.byref(prm), None, ctypes.byref(st), None) == E
    assert lib.odwf_gauge_force(None, None, 6.2, ctypes.byref(act), None, None) == E
    assert lib.odwf_md_trajectory(None, None, None, 0, None, None, None, 6.2, 0.1, 1, 1, 0, ctypes.byref(prm),
                                  en.ctypes.data_as(ctypes.c_void_p), ctypes.byref(st), None) == E
    assert b"odwf_md_trajectory" in lib.odwf_last_error()
