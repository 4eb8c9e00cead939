"""Host-only parts of the flow ABI (no GPU compute): the t0 interpolation of odwf_flow_t0
agrees with the oracle's, and odwf_flow_create rejects bad extents before touching a device."""
import ctypes

import numpy as np
import pytest

import paper_1811_08095_gb300 as odwf
from oracle import flow as fl

L = odwf._lib


@pytest.fixture(scope="module")
def lib():
    return odwf.load(build_if_missing=True)


def _records(ts, es):
    return [{"t": t, "e_plaq": 0.0, "e_clover": e, "q_clover": 0.0, "plaq_min": 1.0, "plaq_mean": 1.0}
            for t, e in zip(ts, es)]


def test_t0_matches_the_oracle(lib):
    ts = np.round(np.arange(0.0, 8.0001, 0.1), 10)
    # a smooth E(t) whose t^2 E crosses 0.3 between two records
    es = 0.08 / (1.0 + ts) ** 1.2
    want = fl.t0_scale(ts, es)
    assert want is not None and 1 < want < 8
    got = odwf.odwf_flow_t0(_records(ts, es))
    assert abs(got - want) < 1e-12
    assert odwf.odwf_flow_t0(_records(ts, es), target=5.0) is None
    assert fl.t0_scale(ts, es, 5.0) is None


@pytest.mark.parametrize("dims", [(1, 4, 4, 4), (4, 4, 0, 4), (4, 4, 4, 5000)])
def test_create_rejects_bad_extents(lib, dims):
    d = (ctypes.c_int32 * 4)(*dims)
    h = ctypes.c_void_p()
    assert lib.odwf_flow_create(d, ctypes.byref(h)) == L.ODWF_EINVAL
    assert not h.value
