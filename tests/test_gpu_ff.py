"""Float-float reliable updates of the mixed-precision CG against the FP64 oracle, through the
C ABI.

The reliable update recomputes the true residual b - S^dag S x, in FP64 or in float-float
arithmetic (each real the unevaluated sum of two FP32 numbers, about 48 bits, on the FP32 pipe);
float-float by default.

* odwf_apply_normal_prec(prec = ODWF_FF), the update's operator with float-float fields, links
  and arithmetic, agrees with the oracle's FP64 S^dag S.  Bar: 1e-10 of the component scale
  (max(|ref|, 1e-3 ||ref||_inf)) per component and 1e-12 in norm: one float-float operation errs by
  at most about 2^-44 of its operands, and an output component sums about a hundred terms.
* Mixed solves with float-float updates meet the true-residual bar recomputed by the oracle,
  agree with the FP64-update solves and the oracle's solution to 1e-8, and take the same
  number of iterations to within two per restart; batched solves with float-float updates too.
"""
import numpy as np
import pytest

import odwf_synth as syn
import oracle
import paper_1811_08095_gb300 as odwf
from gpu_common import M0, assert_close_componentwise, from_dev, make_case, rel_norm, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [
    ((4, 4, 4, 4), 8, 0.01, True),
    ((2, 2, 2, 2), 4, 0.05, True),
    ((6, 4, 2, 10), 8, 0.2, True),
    ((4, 2, 6, 4), 2, 0.5, False),
    ((2, 4, 2, 4), 16, 0.002, True),
]


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.mark.parametrize("dims,ns,mq,tbc", CASES)
def test_ff_normal_operator_matches_oracle(torch, dims, ns, mq, tbc):
    U, w = make_case(dims, ns, mq, eps=0.6, seed=1)
    h = odwf.Handle(dims, ns, M0, mq, w, t_antiperiodic=tbc)
    h.set_gauge(to_dev(torch, U))
    pe = syn.gaussian_spinor_even(ns, dims, 11)
    ref = oracle.normal_op(U, pe, M0, mq, w, tbc, oracle.SCHUR_NORMAL)
    out = torch.empty(pe.shape, dtype=torch.complex128, device="cuda")
    h.apply_normal_prec(out, to_dev(torch, pe), "ff")
    got = from_dev(out)
    assert_close_componentwise(got, ref, 1e-10)
    assert rel_norm(got, ref) < 1e-12
    # and it is far more accurate than the FP32 operator of the inner iteration
    o32 = torch.empty_like(out)
    h.apply_normal_prec(o32, to_dev(torch, pe), "f32", 18)
    assert rel_norm(from_dev(o32), ref) > 1e3 * rel_norm(got, ref)
    h.close()


def _resid(U, x, b, mq, w):
    Ax = oracle.normal_op(U, x, M0, mq, w)
    return np.linalg.norm((b - Ax).reshape(-1)) / np.linalg.norm(b.reshape(-1))


@pytest.mark.parametrize("dims,ns,mq,prec", [((4, 4, 4, 4), 8, 0.01, "f16"), ((6, 4, 2, 10), 8, 0.2, "bf16"),
                                             ((4, 4, 4, 8), 16, 0.002, "f32")])
def test_ff_updates_against_f64_updates_and_oracle(torch, dims, ns, mq, prec):
    U, w = make_case(dims, ns, mq, eps=0.3, seed=2)
    b = syn.gaussian_spinor_even(ns, dims, 101)
    x_ref, _, _ = oracle.cg(U, b, M0, mq, w, tol=1e-13)
    h = odwf.Handle(dims, ns, M0, mq, w)
    h.set_gauge(to_dev(torch, U))
    out = {}
    for f64 in (False, True):
        x = torch.zeros(b.shape, dtype=torch.complex128, device="cuda")
        st = h.cg_solve(x, to_dev(torch, b), tol=1e-10, max_iter=40000, prec=prec, updates="f64" if f64 else "ff")
        torch.cuda.synchronize()
        xs = from_dev(x)
        assert st["status"] == 0 and st["true_resid"] <= 1e-10, st
        assert _resid(U, xs, b, mq, w) <= 1e-10
        assert rel_norm(xs, x_ref) <= 1e-8
        assert st["n_reliable"] >= 1
        out[f64] = (xs, st)
    (x_ff, s_ff), (x_64, s_64) = out[False], out[True]
    assert rel_norm(x_ff, x_64) <= 1e-8
    assert abs(s_ff["iters"] - s_64["iters"]) <= 2 * (s_64["n_reliable"] + 1), (s_ff, s_64)
    # the library's own final residual agrees with the oracle's
    assert abs(s_ff["true_resid"] - _resid(U, x_ff, b, mq, w)) <= 1e-3 * s_ff["true_resid"] + 1e-14
    h.close()


def test_ff_updates_batched_three_masses(torch):
    dims, ns = (8, 8, 8, 8), 16
    U, w = make_case(dims, ns, 0.04, eps=0.3, seed=3)
    masses = [0.002, 0.04, 0.5]
    bs = [syn.gaussian_spinor_even(ns, dims, 200 + k) for k in range(3)]
    h = odwf.Handle(dims, ns, M0, 0.04, w)
    h.set_gauge(to_dev(torch, U))
    xs = [torch.zeros(b.shape, dtype=torch.complex128, device="cuda") for b in bs]
    sts = h.cg_solve_batched(xs, [to_dev(torch, b) for b in bs], masses, tol=1e-10, max_iter=40000, prec="f16",
                             updates="ff")
    torch.cuda.synchronize()
    for x, b, mq, st in zip(xs, bs, masses, sts):
        assert st["status"] == 0 and st["true_resid"] <= 1e-10, st
        assert _resid(U, from_dev(x), b, mq, w) <= 1e-10
    h.close()
