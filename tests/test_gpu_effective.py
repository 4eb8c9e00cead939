"""The 4D effective operator of Sec. 2 through the 5D solve (odwf_effective_solve) and the
residual mass read off it (odwf_residual_mass), against the FP64 oracle's dense 4D effective
operator (1 + r)/2 + (1 - r)/2 gamma_5 S(H_w) built by eigendecomposition of H_w (the dense
identity with the 5D route is pinned in tests/test_oracle_odwf.py).

Bars: FP64 solves to a full-system residual of 1e-12 reproduce D_eff^-1 b to 1e-9 (relative,
normwise) and m_res to 1e-10 absolute; the mixed-precision (FP16 inner) solve to 1e-10
reproduces D_eff^-1 b to 1e-7.
"""
import numpy as np
import pytest

import odwf_synth as syn
import paper_1811_08095_gb300 as odwf
from gpu_common import M0, rel_norm, torch_cuda
from oracle import dense, zolotarev

pytestmark = pytest.mark.gpu

LR = (0.05, 6.2)


def _case(dims, ns, mq, seed=1, eps=0.4):
    U = syn.gauge_field(dims, eps, seed)
    w, _ = zolotarev.omega(ns, LR[0], LR[1], True)
    h = odwf.Handle(dims, ns, M0, mq, w)
    h.set_gauge(U)
    return U, w, h


@pytest.mark.parametrize("dims,ns,mq", [((2, 2, 2, 2), 4, 0.1), ((2, 2, 2, 2), 8, 0.01), ((4, 4, 4, 4), 8, 0.05)])
def test_effective_solve_matches_dense_overlap(dims, ns, mq):
    torch_cuda()
    U, w, h = _case(dims, ns, mq)
    Deff = dense.effective_dense(U, ns, M0, mq, LR[0], LR[1])
    b4 = syn.gaussian_spinor(1, dims, 31)[0]
    ref = dense.effective_propagator(Deff, b4)
    x = np.zeros_like(b4)
    st = h.effective_solve(x, b4, tol=1e-12, max_iter=100000, prec="f64")
    assert st["rc"] == 0 and st["true_resid"] <= 1e-12, st
    assert rel_norm(x, ref) <= 1e-9, rel_norm(x, ref)
    # mixed precision inner solve
    xm = np.zeros_like(b4)
    st = h.effective_solve(xm, b4, tol=1e-10, max_iter=100000, prec="f16")
    assert st["rc"] == 0, st
    assert rel_norm(xm, ref) <= 1e-7, rel_norm(xm, ref)
    h.close()


@pytest.mark.parametrize("dims,ns,mq,site", [((2, 2, 2, 2), 4, 0.1, (1, 0, 1, 1)), ((4, 4, 4, 4), 8, 0.04, (2, 1, 3, 0))])
def test_residual_mass_matches_dense(dims, ns, mq, site):
    torch_cuda()
    U, w, h = _case(dims, ns, mq, seed=2)
    Deff = dense.effective_dense(U, ns, M0, mq, LR[0], LR[1])
    lx, ly, lz, lt = dims
    lex = site[0] + lx * (site[1] + ly * (site[2] + lz * site[3]))
    m_ref, num, den, per_site = dense.residual_mass(Deff, M0, mq, lex)
    mres, corr, st = h.residual_mass(site, tol=1e-12, prec="f64", mq=mq)
    assert st["status"] == 0, st
    assert abs(mres - m_ref) <= 1e-10, (mres, m_ref)
    # correlator: sum of tr(G^dag G) over each time slice, counted from the source time
    ct = per_site.reshape(lt, -1).sum(axis=1)
    ct = np.roll(ct, -site[3])
    assert np.allclose(corr, ct, rtol=1e-9, atol=1e-12 * ct.max())
    h.close()
