"""odwf_apply_m5_noalloc, the allocation-free variant of odwf_apply_m5.

It serves callers that must not let a library allocate device memory (their own pool
already holds the GPU's memory, or they cannot accept cudaMalloc's device-wide
synchronisation); it keeps its staging fields in a fixed device array instead.  This
test calls it through the C ABI on device buffers, twice in a row with different
operators and sizes (the array keeps the previous call's contents), and checks each
result against odwf_apply_m5 on the same input at the GPU tests' FP64 tolerance, and
directly against the FP64 oracle's M, M^dag, M^-1, M^-dag.  It also checks that further calls
leave the device's free memory unchanged, and that buffers of another GPU are refused.  The
file is collected last, so a run that stops at its first failure has run every other
test already; it also passes when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1811_08095_gb300 as odwf
from gpu_common import M0, assert_close_componentwise, torch_cuda
from oracle import zolotarev
from paper_1811_08095_gb300 import _lib

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _noalloc(lib, ns, mq, w, out, inp, n_sites, op, stream=None):
    return lib.odwf_apply_m5_noalloc(ns, M0, mq, w.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(inp.data_ptr()), n_sites, op, stream)


def test_noalloc_matches_apply_m5_twice():
    torch = torch_cuda()
    lib = odwf.load()
    rng = np.random.default_rng(77)
    calls = [(16, 0.002, 1000, 2), (8, 0.5, 8192, 3)]  # (Ns, m_q, n_sites, op): different sizes and ops
    for ns, mq, n_sites, op in calls:
        w, _ = zolotarev.omega(ns, 0.05, 6.2, True)
        w = np.ascontiguousarray(w)
        x = rng.standard_normal((ns, n_sites, 4, 3)) + 1j * rng.standard_normal((ns, n_sites, 4, 3))
        xd = torch.from_numpy(x).cuda()
        ref = torch.zeros_like(xd)
        h = odwf.Handle((2, 2, 2, 2), ns, M0, mq, w)
        h.apply_m5(ref, xd, n_sites, op)
        got = torch.full_like(xd, float("nan"))
        rc = _noalloc(lib, ns, mq, w, got, xd, n_sites, op)
        assert rc == _lib.ODWF_OK, lib.odwf_last_error()
        torch.cuda.synchronize()
        assert_close_componentwise(got.cpu().numpy(), ref.cpu().numpy(), TOL)
        # and directly against the FP64 oracle's site-local operator
        assert_close_componentwise(got.cpu().numpy(), oracle.m5(x, M0, mq, w, op), TOL)
        h.close()


def test_noalloc_allocates_no_device_memory():
    """After a first call on the device (which reserves the fixed array under lazy module
    loading), further calls with other sizes and operators leave the device's free memory
    unchanged: the entry point allocates nothing."""
    torch = torch_cuda()
    lib = odwf.load()
    rng = np.random.default_rng(5)
    bufs = []
    for ns, n_sites in [(16, 4096), (8, 100)]:
        x = rng.standard_normal((ns, n_sites, 4, 3)) + 1j * rng.standard_normal((ns, n_sites, 4, 3))
        xd = torch.from_numpy(x).cuda()
        bufs.append((ns, n_sites, xd, torch.zeros_like(xd)))
    w16 = np.ascontiguousarray(zolotarev.omega(16, 0.05, 6.2, True)[0])
    w8 = np.ascontiguousarray(zolotarev.omega(8, 0.05, 6.2, True)[0])
    ns, n_sites, xd, yd = bufs[0]
    assert _noalloc(lib, ns, 0.01, w16, yd, xd, n_sites, 0) == _lib.ODWF_OK  # warm: set-up of this device
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for (ns, n_sites, xd, yd), w, op in zip(bufs, (w16, w8), (3, 1)):
        assert _noalloc(lib, ns, 0.2, w, yd, xd, n_sites, op) == _lib.ODWF_OK, lib.odwf_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_memory_of_another_gpu():
    """Device buffers of a GPU other than the current one are refused before any kernel runs
    (the kernels would read another GPU's memory without peer access)."""
    torch = torch_cuda()
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two visible GPUs")
    lib = odwf.load()
    ns = 8
    w = np.ascontiguousarray(zolotarev.omega(ns, 0.05, 6.2, True)[0])
    x1 = torch.zeros((ns, 16, 4, 3), dtype=torch.complex128, device="cuda:1")
    y0 = torch.zeros((ns, 16, 4, 3), dtype=torch.complex128, device="cuda:0")
    with torch.cuda.device(0):
        assert _noalloc(lib, ns, 0.01, w, y0, x1, 16, 0) == _lib.ODWF_EINVAL


def test_noalloc_rejects_oversize_and_host_pointers():
    torch = torch_cuda()
    lib = odwf.load()
    ns = 16
    w = np.ascontiguousarray(zolotarev.omega(ns, 0.05, 6.2, True)[0])
    n_sites = 65536 // ns + 1  # one site over the fixed scratch capacity
    x = torch.zeros((ns, n_sites, 4, 3), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    assert _noalloc(lib, ns, 0.01, w, y, x, n_sites, 0) == _lib.ODWF_EINVAL
    assert b"65536" in lib.odwf_last_error()
    xh = np.zeros((ns, 4, 4, 3), dtype=np.complex128)
    rc = lib.odwf_apply_m5_noalloc(ns, M0, 0.01, w.ctypes.data_as(ctypes.c_void_p), ctypes.c_void_p(y.data_ptr()),
                                   xh.ctypes.data_as(ctypes.c_void_p), 4, 0, None)
    assert rc == _lib.ODWF_EINVAL
