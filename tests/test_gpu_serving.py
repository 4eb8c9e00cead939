"""Serving loop (serve_* C ABI): requests on several resident fields, Ns and masses are
solved concurrently; every result meets the oracle's residual bar and equals the same
system solved alone (within the solver tolerance); a request submitted while another is
running joins the running batch before that one finishes (continuous batching); bad
requests fail with the documented codes."""
import time

import numpy as np
import pytest

import odwf_synth as syn
import oracle
import paper_1811_08095_gb300 as odwf
from gpu_common import M0, rel_norm, torch_cuda
from oracle import zolotarev

pytestmark = pytest.mark.gpu


def _wait(srv, tickets, timeout_s=120):
    out = {}
    t_end = time.time() + timeout_s
    while tickets and time.time() < t_end:
        for t in list(tickets):
            rc, res = srv.poll(t, 50)
            if rc != odwf._lib.ODWF_PENDING:
                out[t] = (rc, res)
                tickets.remove(t)
    assert not tickets, "requests did not finish"
    return out


def test_mixed_requests_match_alone_and_oracle():
    torch = torch_cuda()
    fields = {0: ((4, 4, 4, 4), 0.3, 1), 1: ((6, 4, 2, 4), 0.25, 2)}
    srv = odwf.Server(8 << 30)
    U = {}
    for fid, (dims, eps, seed) in fields.items():
        U[fid] = syn.gauge_field(dims, eps, seed)
        srv.register_gauge(fid, dims, U[fid])
    reqs = [  # field, Ns, m_q, nrhs, prec
        (0, 8, 0.01, 3, "f16"), (1, 16, 0.2, 2, "f16"), (0, 8, 0.5, 1, "f16"),
        (0, 4, 0.05, 2, "bf16"), (1, 8, 0.04, 2, "f64"),
    ]
    subs = []
    for i, (fid, ns, mq, nrhs, prec) in enumerate(reqs):
        dims = fields[fid][0]
        w, _ = zolotarev.omega(ns, 0.05, 6.2, True)
        bs = [syn.gaussian_spinor_even(ns, dims, 500 + 10 * i + k) for k in range(nrhs)]
        xs = [np.zeros_like(b) for b in bs]
        t = srv.submit(fid, ns, M0, mq, w, bs, xs, tol=1e-10, prec=prec)
        subs.append((t, fid, ns, mq, w, bs, xs, prec))
    res = _wait(srv, [s[0] for s in subs])
    for t, fid, ns, mq, w, bs, xs, prec in subs:
        rc, r = res[t]
        assert rc == 0 and r["true_resid"] <= 1e-10, r
        dims = fields[fid][0]
        h = odwf.Handle(dims, ns, M0, mq, w)
        h.set_gauge(U[fid])
        for b, x in zip(bs, xs):
            resid = np.linalg.norm(b - oracle.normal_op(U[fid], x, M0, mq, w)) / np.linalg.norm(b)
            assert resid <= 1e-10
            xa = np.zeros_like(b)
            h.cg_solve(xa, b, tol=1e-10, prec=prec)
            assert rel_norm(x, xa) <= 1e-8  # alone vs in the mix
        h.close()
    srv.close()


def test_continuous_batching_joins_running_batch():
    torch = torch_cuda()
    dims, ns = (16, 16, 16, 16), 16
    srv = odwf.Server(0)
    U = syn.gauge_field_torch(dims, 0.25, 3, device="cuda")
    srv.register_gauge(0, dims, U)
    w, _ = zolotarev.omega(ns, 0.05, 6.2, True)
    shape = (ns, dims[0] * dims[1] * dims[2] * dims[3] // 2, 4, 3)
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    b1 = [torch.randn(shape, dtype=torch.complex128, device="cuda", generator=g)]
    x1 = [torch.zeros_like(b1[0])]
    b2 = [torch.randn(shape, dtype=torch.complex128, device="cuda", generator=g)]
    x2 = [torch.zeros_like(b2[0])]
    torch.cuda.synchronize()
    t_sub1 = time.perf_counter()
    t1 = srv.submit(0, ns, M0, 0.002, w, b1, x1, tol=1e-10, prec="f16")
    time.sleep(0.05)
    t_sub2 = time.perf_counter()
    t2 = srv.submit(0, ns, M0, 0.3, w, b2, x2, tol=1e-10, prec="f16")
    res = _wait(srv, [t1, t2])
    (rc1, r1), (rc2, r2) = res[t1], res[t2]
    assert rc1 == 0 and rc2 == 0
    end1 = t_sub1 + r1["latency_ms"] / 1e3
    admit2 = t_sub2 + r2["queue_ms"] / 1e3
    assert r1["latency_ms"] / 1e3 > (t_sub2 - t_sub1) + 0.01, "first request finished too early to test"
    assert admit2 < end1, "the second request waited for the first batch to finish"
    srv.close()


def test_serving_errors():
    torch_cuda()
    srv = odwf.Server(256 << 20)
    dims = (4, 4, 4, 4)
    U = syn.gauge_field(dims, 0.3, 1)
    srv.register_gauge(0, dims, U)
    w, _ = zolotarev.omega(8, 0.05, 6.0, True)
    b = [syn.gaussian_spinor_even(8, dims, 1)]
    x = [np.zeros_like(b[0])]
    with pytest.raises(odwf.OdwfError) as e:
        srv.submit(9, 8, M0, 0.1, w, b, x)  # unknown field
    assert e.value.code == odwf._lib.ODWF_ENOTFOUND
    with pytest.raises(odwf.OdwfError) as e:
        srv.register_gauge(0, dims, U)  # duplicate id
    assert e.value.code == odwf._lib.ODWF_EINVAL
    big = (32, 32, 32, 32)
    with pytest.raises(odwf.OdwfError) as e:  # the 256 MiB budget cannot hold this 604 MB field
        srv.register_gauge(1, big, np.zeros((4, 32, 32, 32, 32, 3, 3), dtype=np.complex128))
    assert e.value.code == odwf._lib.ODWF_ENOMEM
    rc, _ = srv.poll(12345, 0)
    assert rc == odwf._lib.ODWF_ENOTFOUND
    srv.close()
