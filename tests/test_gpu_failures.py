"""Failure paths, made on the host or by the inputs (no GPU fault, trap or hang):

* a right-hand side holding NaN is a CG breakdown (ODWF_EBREAKDOWN), through odwf_cg_solve (FP64
  and mixed precision), odwf_cg_solve_batched (the other systems of the batch still converge)
  and serve_submit;
* serve_cancel stops a running request between chunks (ODWF_ECANCELED) and a queued one at
  once, and the server keeps serving;
* the admission policy sheds requests that waited past the deadline (ODWF_ETIMEOUT) and refuses
  submissions beyond the queue cap (ODWF_EBUSY);
* an error inside a batch (injected on the host as a failing chunk launch, in a child process)
  fails that batch's requests with ODWF_ECUDA while the server stays usable.
"""
import os
import subprocess
import sys
import time

import numpy as np
import pytest

import odwf_synth as syn
import paper_1811_08095_gb300 as odwf
from gpu_common import M0, make_case, torch_cuda
from oracle import zolotarev

pytestmark = pytest.mark.gpu
L = odwf._lib


def _poll_done(srv, t, timeout_s=120):
    t_end = time.time() + timeout_s
    while time.time() < t_end:
        rc, res = srv.poll(t, 50)
        if rc != L.ODWF_PENDING:
            return rc, res
    raise AssertionError("request %d did not finish" % t)


@pytest.mark.parametrize("prec", ["f64", "f16"])
def test_nan_rhs_is_breakdown(prec):
    torch = torch_cuda()
    dims, ns, mq = (4, 4, 4, 4), 8, 0.1
    U, w = make_case(dims, ns, mq)
    h = odwf.Handle(dims, ns, M0, mq, w)
    h.set_gauge(torch.from_numpy(U).cuda())
    b = syn.gaussian_spinor_even(ns, dims, 1)
    b[3, 5, 1, 2] = np.nan
    x = np.zeros_like(b)
    st = h.cg_solve(x, b, tol=1e-10, max_iter=1000, prec=prec, raise_on_error=False)
    assert st["rc"] == L.ODWF_EBREAKDOWN and st["status"] == L.ODWF_EBREAKDOWN, st
    # batched: the NaN system breaks down, the others converge
    bs = [syn.gaussian_spinor_even(ns, dims, 2), b, syn.gaussian_spinor_even(ns, dims, 3)]
    xs = [np.zeros_like(v) for v in bs]
    sts = h.cg_solve_batched(xs, bs, [0.1, 0.1, 0.3], tol=1e-10, max_iter=1000, prec=prec, raise_on_error=False)
    assert [s["status"] for s in sts] == [0, L.ODWF_EBREAKDOWN, 0], sts
    assert sts[0]["true_resid"] <= 1e-10 and sts[2]["true_resid"] <= 1e-10
    h.close()


def test_nan_rhs_through_serving():
    torch_cuda()
    dims, ns = (4, 4, 4, 4), 8
    srv = odwf.Server(4 << 30)
    srv.register_gauge(0, dims, syn.gauge_field(dims, 0.3, 1))
    w, _ = zolotarev.omega(ns, 0.05, 6.2, True)
    bad = syn.gaussian_spinor_even(ns, dims, 4)
    bad[0, 0, 0, 0] = np.nan
    good = syn.gaussian_spinor_even(ns, dims, 5)
    xb, xg = np.zeros_like(bad), np.zeros_like(good)
    t1 = srv.submit(0, ns, M0, 0.1, w, [bad], [xb], tol=1e-10, prec="f16")
    t2 = srv.submit(0, ns, M0, 0.1, w, [good], [xg], tol=1e-10, prec="f16")
    rc1, _ = _poll_done(srv, t1)
    rc2, r2 = _poll_done(srv, t2)
    assert rc1 == L.ODWF_EBREAKDOWN
    assert rc2 == 0 and r2["true_resid"] <= 1e-10
    srv.close()


def _slow_request(srv, dims, ns, w, seed, nrhs=1):
    """A request that runs until it is cancelled: light mass and a tolerance below FP64 reach."""
    bs = [syn.gaussian_spinor_even(ns, dims, seed + k) for k in range(nrhs)]
    xs = [np.zeros_like(b) for b in bs]
    return srv.submit(0, ns, M0, 0.0005, w, bs, xs, tol=1e-17, prec="f16", max_iter=1000000), xs


def test_cancel_running_and_queued():
    torch_cuda()
    dims, ns = (16, 16, 16, 16), 8
    srv = odwf.Server(16 << 30)
    srv.register_gauge(0, dims, syn.gauge_field_torch(dims, 0.25, 11, device="cuda"))
    w, _ = zolotarev.omega(ns, 0.05, 6.2, True)
    t_run, xs = _slow_request(srv, dims, ns, w, 10, nrhs=16)  # fills the batch's 16 slots
    t_wait, _ = _slow_request(srv, dims, ns, w, 40)           # waits for a slot
    t_end = time.time() + 60
    while time.time() < t_end:  # until the first is admitted
        rc, res = srv.poll(t_run, 0)
        if res["queue_ms"] >= 0:
            break
        time.sleep(0.01)
    assert rc == L.ODWF_PENDING
    rc, res = srv.poll(t_wait, 0)
    assert rc == L.ODWF_PENDING and res["queue_ms"] < 0  # still queued
    srv.cancel(t_wait)
    assert srv.poll(t_wait, 0)[0] == L.ODWF_ECANCELED  # queued: at once
    t0 = time.time()
    srv.cancel(t_run)
    rc, _ = _poll_done(srv, t_run, 60)
    assert rc == L.ODWF_ECANCELED, rc
    assert time.time() - t0 < 30
    assert all(not np.any(x) for x in xs)  # a cancelled request writes no solution
    # the server keeps serving
    b = syn.gaussian_spinor_even(ns, dims, 99)
    x = np.zeros_like(b)
    t = srv.submit(0, ns, M0, 0.2, w, [b], [x], tol=1e-10, prec="f16")
    rc, r = _poll_done(srv, t)
    assert rc == 0 and r["true_resid"] <= 1e-10
    with pytest.raises(odwf.OdwfError):
        srv.cancel(123456789)  # unknown ticket
    srv.close()


def test_admission_deadline_and_queue_cap():
    torch_cuda()
    dims, ns = (16, 16, 16, 16), 8
    srv = odwf.Server(16 << 30)
    srv.register_gauge(0, dims, syn.gauge_field_torch(dims, 0.25, 12, device="cuda"))
    w, _ = zolotarev.omega(ns, 0.05, 6.2, True)
    srv.set_policy(admit_deadline_ms=0.0, max_queued=1)
    t_run, _ = _slow_request(srv, dims, ns, w, 10, nrhs=16)
    t_end = time.time() + 60
    while time.time() < t_end and srv.poll(t_run, 0)[1]["queue_ms"] < 0:
        time.sleep(0.01)
    t_q, _ = _slow_request(srv, dims, ns, w, 40)  # queued (the batch is full)
    ok, t_none = srv.try_submit(0, ns, M0, 0.1, w, [syn.gaussian_spinor_even(ns, dims, 41)],
                                [np.zeros_like(syn.gaussian_spinor_even(ns, dims, 41))])
    assert ok == L.ODWF_EBUSY and t_none is None
    # a 50 ms deadline sheds the queued request
    srv.set_policy(admit_deadline_ms=50.0, max_queued=0)
    rc, res = _poll_done(srv, t_q, 30)
    assert rc == L.ODWF_ETIMEOUT and res["queue_ms"] < 0, (rc, res)
    srv.cancel(t_run)
    assert _poll_done(srv, t_run, 60)[0] == L.ODWF_ECANCELED
    srv.close()


_CHILD = r"""
import sys, time
sys.path.insert(0, %r)
import numpy as np, torch
import odwf_synth as syn
import paper_1811_08095_gb300 as odwf
from oracle import zolotarev
L = odwf._lib
dims, ns = (4, 4, 4, 4), 8
srv = odwf.Server(4 << 30)
srv.register_gauge(0, dims, syn.gauge_field(dims, 0.3, 1))
w, _ = zolotarev.omega(ns, 0.05, 6.2, True)
def run(seed):
    b = syn.gaussian_spinor_even(ns, dims, seed)
    x = np.zeros_like(b)
    t = srv.submit(0, ns, M0, 0.1, w, [b], [x], tol=1e-10, prec="f16")
    t_end = time.time() + 60
    while time.time() < t_end:
        rc, r = srv.poll(t, 50)
        if rc != L.ODWF_PENDING:
            return rc, r
    return -1, None
M0 = 1.3
rc1, _ = run(1)   # its first chunk launch is the injected failure
rc2, r2 = run(2)  # a new batch after the failed one was dropped
print("RESULT", rc1, rc2, r2["true_resid"] if r2 else None)
srv.close()
"""


def test_error_inside_a_batch_fails_its_requests():
    torch_cuda()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, ODWF_SERVE_INJECT_ERROR="1")
    out = subprocess.run([sys.executable, "-c", _CHILD % root], env=env, capture_output=True, text=True, timeout=300)
    line = [ln for ln in out.stdout.splitlines() if ln.startswith("RESULT")]
    assert out.returncode == 0 and line, out.stdout + out.stderr
    _, rc1, rc2, resid = line[0].split()
    assert int(rc1) == L.ODWF_ECUDA
    assert int(rc2) == 0 and float(resid) <= 1e-10
