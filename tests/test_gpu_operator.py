"""GPU parity of the FP64 operator kernels against the FP64 CPU oracle, element by element,
through the C ABI: D, D^dag (full lattice), S, S^dag (even sites), S^dag S, D^dag D and the
site-local M, M^dag, M^-1, M^-dag, on lattices that span several thread blocks with a
ragged tail, every supported Ns, both time boundaries and the minimal 2^4 lattice.
Bar: |gpu - oracle| <= 1e-12 max(|oracle|, 1e-3 ||oracle||_inf) per component."""
import numpy as np
import pytest

import odwf_synth as syn
import oracle
import paper_1811_08095_gb300 as odwf
from gpu_common import M0, assert_close_componentwise, from_dev, make_case, rel_norm, to_dev, torch_cuda

pytestmark = pytest.mark.gpu

TOL = 1e-12

CASES = [
    # dims, Ns, m_q, antiperiodic
    ((4, 4, 4, 4), 8, 0.01, True),     # the 4^4 x 8 workload
    ((2, 2, 2, 2), 4, 0.05, True),     # minimal lattice: x+mu and x-mu coincide
    ((6, 4, 2, 10), 8, 0.2, True),     # 1920 5D half sites: ragged last block
    ((4, 2, 6, 4), 2, 0.5, False),
    ((2, 4, 2, 4), 16, 0.002, True),
    ((4, 4, 2, 2), 32, 0.04, False),
]


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def _handle(dims, ns, mq, tbc, seed=1):
    U, w = make_case(dims, ns, mq, eps=0.6, seed=seed)
    h = odwf.Handle(dims, ns, M0, mq, w, t_antiperiodic=tbc)
    return h, U, w


@pytest.mark.parametrize("dims,ns,mq,tbc", CASES)
def test_full_operator_and_dagger(torch, dims, ns, mq, tbc):
    h, U, w = _handle(dims, ns, mq, tbc)
    h.set_gauge(to_dev(torch, U))
    psi = syn.gaussian_spinor(ns, dims, 7)
    for dag in (False, True):
        ref = oracle.d5(U, psi, M0, mq, w, tbc, dag)
        out = torch.zeros(psi.shape, dtype=torch.complex128, device="cuda")
        (h.apply_dagger if dag else h.apply)(out, to_dev(torch, psi), odwf.ODWF_MODE_FULL)
        torch.cuda.synchronize()
        assert_close_componentwise(from_dev(out), ref, TOL)
    h.close()


@pytest.mark.parametrize("dims,ns,mq,tbc", CASES)
def test_schur_operator_and_dagger(torch, dims, ns, mq, tbc):
    h, U, w = _handle(dims, ns, mq, tbc)
    h.set_gauge(U)  # host gauge field: staged by the library
    psi = syn.gaussian_spinor_even(ns, dims, 8)
    for dag in (False, True):
        ref = oracle.schur(U, psi, M0, mq, w, tbc, dag)
        out = np.zeros_like(psi)
        (h.apply_dagger if dag else h.apply)(out, psi, odwf.ODWF_MODE_SCHUR_EVEN)  # host fields
        assert_close_componentwise(out, ref, TOL)
    h.close()


@pytest.mark.parametrize("dims,ns,mq,tbc", CASES[:3])
def test_normal_operators(torch, dims, ns, mq, tbc):
    h, U, w = _handle(dims, ns, mq, tbc)
    h.set_gauge(to_dev(torch, U))
    pe = syn.gaussian_spinor_even(ns, dims, 9)
    ref = oracle.normal_op(U, pe, M0, mq, w, tbc, oracle.SCHUR_NORMAL)
    out = torch.zeros(pe.shape, dtype=torch.complex128, device="cuda")
    h.apply_normal(out, to_dev(torch, pe), odwf.ODWF_SYS_SCHUR_NORMAL)
    torch.cuda.synchronize()
    assert_close_componentwise(from_dev(out), ref, TOL)
    pf = syn.gaussian_spinor(ns, dims, 10)
    ref = oracle.normal_op(U, pf, M0, mq, w, tbc, oracle.FULL_NORMAL)
    out = np.zeros_like(pf)
    h.apply_normal(out, pf, odwf.ODWF_SYS_FULL_NORMAL)
    assert_close_componentwise(out, ref, TOL)
    h.close()


@pytest.mark.parametrize("ns", [2, 4, 8, 16, 32])
def test_site_local_ops(torch, ns):
    dims = (2, 2, 2, 2)
    _, w = make_case(dims, ns, 0.1)
    h = odwf.Handle(dims, ns, M0, 0.03, w)
    n_sites = 37  # any number of sites: a ragged lane-group count
    psi = np.random.default_rng(ns).standard_normal((ns, n_sites, 4, 3, 2)).view(np.complex128)[..., 0]
    psi = np.ascontiguousarray(psi)
    for op in range(4):
        ref = oracle.m5(psi, M0, 0.03, w, op)
        out = np.zeros_like(psi)
        h.apply_m5(out, psi, n_sites, op)
        assert_close_componentwise(out, ref, TOL)
    h.close()


@pytest.mark.parametrize("prec,tol", [("f32", 2e-6), ("f16", 5e-3), ("bf16", 4e-2)])
@pytest.mark.parametrize("recon", [12, 18])
def test_mixed_precision_normal_operator(torch, prec, tol, recon):
    """The inner operator S^dag S in FP32 arithmetic on FP32 / FP16 / BF16 storage: normwise
    relative error bounded by a few roundings of the storage format (2^-24, 2^-11, 2^-8)."""
    dims, ns, mq = (6, 4, 2, 10), 8, 0.01
    U, w = make_case(dims, ns, mq, eps=0.3)
    h = odwf.Handle(dims, ns, M0, mq, w)
    h.set_gauge(to_dev(torch, U))
    pe = syn.gaussian_spinor_even(ns, dims, 11)
    ref = oracle.normal_op(U, pe, M0, mq, w, True, oracle.SCHUR_NORMAL)
    out = np.zeros_like(pe)
    h.apply_normal_prec(out, pe, prec, recon)
    err = rel_norm(out, ref)
    assert err < tol, err
    h.close()


def test_invalid_arguments_on_gpu(torch):
    dims, ns = (4, 4, 4, 4), 8
    U, w = make_case(dims, ns, 0.01)
    h = odwf.Handle(dims, ns, M0, 0.01, w)
    psi = np.zeros((ns,) + (4, 4, 4, 4) + (4, 3), dtype=np.complex128)
    with pytest.raises(odwf.OdwfError):  # gauge field not set yet
        h.apply(np.zeros_like(psi), psi, odwf.ODWF_MODE_FULL)
    h.set_gauge(U)
    with pytest.raises(odwf.OdwfError):
        h.apply(np.zeros_like(psi), psi, 7)
    with pytest.raises(odwf.OdwfError):
        h.apply_m5(np.zeros_like(psi), psi, 0, 0)
    h.close()
