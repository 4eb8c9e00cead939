"""GPU solver parity against the FP64 oracle, through the C ABI.

* FP64 CG and mixed-precision CG (FP32 / FP16 / BF16 inner storage, FP32 arithmetic, FP64
  reliable updates) on S^dag S x = b: the true residual ||b - S^dag S x||/||b|| recomputed by
  the oracle is <= 1e-10, and the solution agrees with the oracle's CG (run to 1e-13) to
  1e-8 relative (the targets of the 4^4 x 8 and 16^3 x 32 x 16 workloads).
* batched multi-RHS / multi-mass solves agree with solving each system alone and with the
  oracle; full-lattice D x = eta and D^dag D x = b through the Schur system agree with dense
  LU on 2^4 x 4 and meet the residual bar on 4^4 x 8 (oracle residual).
* degenerate inputs: b = 0, a tiny max_iter, invalid parameters.
"""
import numpy as np
import pytest

import odwf_synth as syn
import oracle
import paper_1811_08095_gb300 as odwf
from gpu_common import M0, from_dev, make_case, rel_norm, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.fixture(scope="module")
def c1():
    """4^4 x 8, m0 = 1.3, m_q = 0.01, weights on [0.05, 6.0], links exp(0.3 i H) (seed 1)."""
    dims, ns, mq = (4, 4, 4, 4), 8, 0.01
    U, w = make_case(dims, ns, mq, eps=0.3, seed=1)
    b = syn.gaussian_spinor_even(ns, dims, 100)
    x_ref, it, res = oracle.cg(U, b, M0, mq, w, tol=1e-13)
    assert it > 0
    return dims, ns, mq, U, w, b, x_ref


def _true_resid(U, x, b, mq, w):
    Ax = oracle.normal_op(U, x, M0, mq, w)
    return rel_norm(Ax, b) if False else np.linalg.norm((b - Ax).reshape(-1)) / np.linalg.norm(b.reshape(-1))


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "bf16"])
def test_cg_c1(torch, c1, prec):
    dims, ns, mq, U, w, b, x_ref = c1
    h = odwf.Handle(dims, ns, M0, mq, w)
    h.set_gauge(to_dev(torch, U))
    x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
    st = h.cg_solve(x, to_dev(torch, b), tol=1e-10, max_iter=20000, prec=prec)
    torch.cuda.synchronize()
    xs = from_dev(x)
    assert st["status"] == 0 and st["true_resid"] <= 1e-10
    assert _true_resid(U, xs, b, mq, w) <= 1e-10
    assert rel_norm(xs, x_ref) <= 1e-8
    if prec != "f64":
        assert st["n_reliable"] >= 1
    h.close()


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_cg_ragged_ns16_host_pointers(torch, prec):
    dims, ns, mq = (6, 4, 4, 8), 16, 0.04
    U, w = make_case(dims, ns, mq, eps=0.25, seed=2)
    b = syn.gaussian_spinor_even(ns, dims, 101)
    h = odwf.Handle(dims, ns, M0, mq, w)
    h.set_gauge(U)
    x = np.zeros_like(b)
    st = h.cg_solve(x, b, tol=1e-10, max_iter=20000, prec=prec)
    assert st["status"] == 0
    assert _true_resid(U, x, b, mq, w) <= 1e-10
    x_ref, _, _ = oracle.cg(U, b, M0, mq, w, tol=1e-13)
    assert rel_norm(x, x_ref) <= 1e-8
    h.close()


@pytest.mark.parametrize("ns,prec", [(4, "f16"), (2, "bf16"), (32, "f32")])
def test_cg_generic_kernel_ns(torch, ns, prec):
    """Ns outside {8, 16} runs the generic mixed kernels; same bar."""
    dims, mq = (4, 2, 4, 4), 0.03
    U, w = make_case(dims, ns, mq, eps=0.3, seed=5)
    b = syn.gaussian_spinor_even(ns, dims, 102)
    h = odwf.Handle(dims, ns, M0, mq, w)
    h.set_gauge(U)
    x = np.zeros_like(b)
    st = h.cg_solve(x, b, tol=1e-10, max_iter=20000, prec=prec)
    assert st["status"] == 0
    assert _true_resid(U, x, b, mq, w) <= 1e-10
    x_ref, _, _ = oracle.cg(U, b, M0, mq, w, tol=1e-13)
    assert rel_norm(x, x_ref) <= 1e-8
    h.close()


def test_batched_multi_mass_multi_rhs(torch):
    dims, ns = (4, 4, 4, 8), 8
    U, w = make_case(dims, ns, 0.01, eps=0.25, seed=3)
    masses = [0.002, 0.04, 0.5]
    bs = [syn.gaussian_spinor_even(ns, dims, 200 + k) for k in range(2)]
    sys_b = [b for m in masses for b in bs]
    sys_m = [m for m in masses for b in bs]
    h = odwf.Handle(dims, ns, M0, 0.1, w)
    h.set_gauge(to_dev(torch, U))
    for prec in ("f16", "f64"):
        xs = [torch.zeros(b.shape, dtype=torch.complex128, device="cuda") for b in sys_b]
        stats = h.cg_solve_batched(xs, [to_dev(torch, b) for b in sys_b], sys_m, tol=1e-10, max_iter=50000,
                                   prec=prec)
        torch.cuda.synchronize()
        for k, (x, b, m) in enumerate(zip(xs, sys_b, sys_m)):
            xs_k = from_dev(x)
            assert stats[k]["status"] == 0
            assert _true_resid(U, xs_k, b, m, w) <= 1e-10
            # alone vs in the batch
            xa = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
            h.cg_solve(xa, to_dev(torch, b), tol=1e-10, max_iter=50000, prec=prec, mq=m)
            torch.cuda.synchronize()
            assert rel_norm(xs_k, from_dev(xa)) <= 1e-8
    h.close()


def test_full_dirac_and_full_normal_dense(torch):
    from oracle import dense

    dims, ns, mq = (2, 2, 2, 2), 4, 0.05
    U, w = make_case(dims, ns, mq, eps=0.5, seed=4)
    D = dense.dense_d5(U, ns, M0, mq, w)
    eta = syn.gaussian_spinor(ns, dims, 300)
    h = odwf.Handle(dims, ns, M0, mq, w)
    h.set_gauge(U)
    for system, A in [(odwf.ODWF_SYS_FULL_DIRAC, D), (odwf.ODWF_SYS_FULL_NORMAL, D.conj().T @ D)]:
        for prec in ("f64", "f16"):
            x = np.zeros_like(eta)
            st = h.cg_solve(x, eta, tol=1e-12, max_iter=20000, prec=prec, system=system)
            x_ref = np.linalg.solve(A, eta.reshape(-1)).reshape(eta.shape)
            assert rel_norm(x, x_ref) <= 1e-8, (system, prec)
            assert st["true_resid"] <= 1e-10
    h.close()


def test_full_systems_residual_c1(torch, c1):
    dims, ns, mq, U, w, _, _ = c1
    eta = syn.gaussian_spinor(ns, dims, 301)
    h = odwf.Handle(dims, ns, M0, mq, w)
    h.set_gauge(to_dev(torch, U))
    x = np.zeros_like(eta)
    st = h.cg_solve(x, eta, tol=1e-11, max_iter=20000, prec="f16", system=odwf.ODWF_SYS_FULL_DIRAC)
    r = eta - oracle.d5(U, x, M0, mq, w)
    assert np.linalg.norm(r) / np.linalg.norm(eta) <= 1e-10
    x = np.zeros_like(eta)
    st = h.cg_solve(x, eta, tol=1e-12, max_iter=40000, prec="f16", system=odwf.ODWF_SYS_FULL_NORMAL)
    r = eta - oracle.normal_op(U, x, M0, mq, w, True, oracle.FULL_NORMAL)
    assert np.linalg.norm(r) / np.linalg.norm(eta) <= 1e-10, st
    h.close()


def test_degenerate_inputs(torch, c1):
    dims, ns, mq, U, w, b, _ = c1
    h = odwf.Handle(dims, ns, M0, mq, w)
    h.set_gauge(U)
    z = np.zeros_like(b)
    x = np.ones_like(b)
    st = h.cg_solve(x, z, tol=1e-10, prec="f16")
    assert st["status"] == 0 and np.all(x == 0)
    x = np.zeros_like(b)
    st = h.cg_solve(x, b, tol=1e-10, max_iter=3, prec="f64", raise_on_error=False)
    assert st["rc"] == odwf._lib.ODWF_ENOCONV and st["iters"] <= 3 + 8
    assert st["true_resid"] > 1e-10
    with pytest.raises(odwf.OdwfError):
        h.cg_solve(x, b, tol=-1.0)
    with pytest.raises(odwf.OdwfError):
        h.cg_solve(x, b, tol=1e-10, prec=9)
    h.close()
