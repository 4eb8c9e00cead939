"""Element-wise parity of the production mixed-precision CG iteration (the p update and the
hops K1..K4 that the batched solver launches every iteration) against the FP64 oracle.

odwf_mixed_cg_step runs exactly those launches once and returns every field the iteration
stores.  Each stage is checked on the stored (rounded) inputs it actually read, so the only
differences left are the kernel's FP32 arithmetic and the rounding of its own output to the
storage format:

    |gpu - ref| <= c_store * max|ref over the 5D site| + c_arith * max|ref over the field|

with c_store = 2^-11 (FP16: twice the half-ulp 2^-12 of a value scaled into [-1, 1] by the
per-site scale), 2^-8 (BF16) or 2^-23 (FP32 storage), and c_arith = 1e-5 (FP32 arithmetic on
sums of ~100 terms).  A wrong sign, a dropped corner term (m_q = 0.5 makes r = 0.19) or a
transposed link is an O(1) error and fails.  The references are the oracle's own pinned
pieces: -1/2 W from the Wilson operator (oracle.hop_w), B and B^dag (oracle.b5), M^dag, M^-1
and M^-dag (oracle.m5); their composition is checked against oracle.normal_op (S^dag S).
"""
import numpy as np
import pytest

import odwf_synth as syn
import oracle
import paper_1811_08095_gb300 as odwf
from gpu_common import M0, make_case, torch_cuda

pytestmark = pytest.mark.gpu

C_STORE = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8, "f32": 2.0 ** -23, "acc": 2.0 ** -23}  # acc: FP32 r, x
C_ARITH = 1e-5
# normwise bound of the composed inner operator against S^dag S (roundings of the stored
# intermediates of four hops)
C_NORMAL = {"f16": 4e-3, "bf16": 3e-2, "f32": 2e-5}  # FP16 links add ~2^-12 per link entry

CASES = [
    # dims, Ns, m_q, antiperiodic, storage, link reals
    ((4, 4, 4, 4), 8, 0.5, True, "f16", 12),
    ((6, 4, 2, 10), 8, 0.04, True, "f16", 18),     # 960 half sites x 8: ragged last block
    ((6, 4, 2, 10), 16, 0.5, False, "bf16", 12),
    ((4, 2, 6, 4), 16, 0.002, True, "f32", 12),
    ((2, 2, 2, 2), 8, 0.5, True, "f16", 12),       # minimal lattice: x+mu and x-mu coincide
    ((4, 6, 2, 2), 16, 0.5, True, "f16", 12),
]


def _stored_check(got, ref, prec, what, c_arith=C_ARITH, field_scale=None):
    ns = ref.shape[0]
    site = np.abs(ref).reshape(ns, -1, 12).max(axis=2)[..., None, None]
    fs = np.abs(ref).max() if field_scale is None else field_scale
    bound = C_STORE[prec] * site + c_arith * fs
    err = np.abs(got - ref)
    worst = (err / bound).max()
    assert worst <= 1.0, "%s: error %.3e of its bound (max |err| %.3e)" % (what, worst, err.max())
    return worst


def _r32(a):
    return a.astype(np.complex64).astype(np.complex128)


def _links_as_stored_fp16(U):
    """The links an FP16 12-real kernel multiplies by: rows 0 and 1 rounded to FP16 (real and
    imaginary parts), row 2 = conj(row0 x row1) of the rounded rows."""
    V = U.copy()
    r = V[..., :2, :]
    r = r.real.astype(np.float16).astype(np.float64) + 1j * r.imag.astype(np.float16).astype(np.float64)
    V[..., :2, :] = r
    a, b = V[..., 0, :], V[..., 1, :]
    V[..., 2, :] = np.conj(np.cross(a, b))
    return V


def _step_and_check(torch, dims, ns, mq, tbc, prec, recon, seed=1, eps=0.4, link_prec="f32"):
    U0, w = make_case(dims, ns, mq, eps=eps, seed=seed, lrange=(0.05, 6.2))
    h = odwf.Handle(dims, ns, M0, mq, w, t_antiperiodic=tbc)
    h.set_gauge(torch.from_numpy(U0).cuda())
    U = _links_as_stored_fp16(U0) if link_prec == "f16" else U0
    p_prev = syn.gaussian_spinor_even(ns, dims, 200 + seed)
    r = syn.gaussian_spinor_even(ns, dims, 300 + seed)
    x = syn.gaussian_spinor_even(ns, dims, 400 + seed)
    beta = 0.7
    r32, x32 = _r32(r), _r32(x)
    rr = float(np.vdot(r32, r32).real)
    outs = [np.zeros_like(p_prev) for _ in range(8)]  # host outputs: the library stages them
    sc = h.mixed_cg_step(p_prev, r, x, outs, beta, rr, prec=prec, link_recon=recon, mq=mq, link_prec=link_prec)
    h.close()
    assert sc["status"] == 0, sc
    pps, p, chi_p, chi_t, a, c, r_new, x_new = outs
    worst = {}
    # the storage round trip of the input itself
    worst["p_prev"] = _stored_check(pps, p_prev, prec, "p_prev stored")
    # P: p = r + beta p_prev;  chi_p = B p
    worst["p"] = _stored_check(p, r32 + beta * pps, prec, "p")
    worst["chi_p"] = _stored_check(chi_p, oracle.b5(p, M0, mq, w), prec, "chi_p = B p")
    # K1: chi_t = B M^-1 (-1/2 W chi_p)   (odd sites)
    t = oracle.m5(oracle.hop_w(U, chi_p, 0, M0, tbc), M0, mq, w, oracle.MINV)
    worst["chi_t"] = _stored_check(chi_t, oracle.b5(t, M0, mq, w), prec, "K1 chi_t")
    # K2: s = p - M^-1 (-1/2 W chi_t);  a = M^-dag s;  pAp = |s|^2
    s = p - oracle.m5(oracle.hop_w(U, chi_t, 1, M0, tbc), M0, mq, w, oracle.MINV)
    worst["a"] = _stored_check(a, oracle.m5(s, M0, mq, w, oracle.MINVDAG), prec, "K2 a")
    pap = float(np.vdot(s, s).real)
    assert abs(sc["pAp"] - pap) <= 1e-5 * pap, (sc["pAp"], pap)
    assert abs(sc["alpha"] - rr / pap) <= 1e-5 * rr / pap, (sc["alpha"], rr / pap)
    # K3: c = M^-dag B^dag (-1/2 W^dag a)   (odd sites)
    cref = oracle.m5(oracle.b5(oracle.hop_w(U, a, 0, M0, tbc, dagger=True), M0, mq, w, dagger=True),
                     M0, mq, w, oracle.MINVDAG)
    worst["c"] = _stored_check(c, cref, prec, "K3 c")
    # K4: Ap = M^dag a - B^dag (-1/2 W^dag c);  r -= alpha Ap;  x += alpha p   (FP32 storage)
    ap = oracle.m5(a, M0, mq, w, oracle.MDAG) - oracle.b5(oracle.hop_w(U, c, 1, M0, tbc, dagger=True), M0, mq,
                                                          w, dagger=True)
    al = sc["alpha"]
    scale_r = max(np.abs(r32).max(), np.abs(al * ap).max())
    worst["r_new"] = _stored_check(r_new, r32 - al * ap, "acc", "K4 r", field_scale=scale_r)
    worst["x_new"] = _stored_check(x_new, x32 + al * p, "acc", "K4 x",
                                   field_scale=max(np.abs(x32).max(), np.abs(al * p).max()))
    rrn = float(np.vdot(r_new, r_new).real)
    assert abs(sc["rr_new"] - rrn) <= 1e-5 * rrn, (sc["rr_new"], rrn)
    # the stage references compose to the oracle's S^dag S on the stored p (exact links)
    an = oracle.normal_op(U0, p, M0, mq, w, tbc)
    rel = np.linalg.norm(ap - an) / np.linalg.norm(an)
    assert rel <= C_NORMAL[prec], (rel, prec)
    return worst


@pytest.mark.parametrize("dims,ns,mq,tbc,prec,recon", CASES)
def test_mixed_step_elementwise(dims, ns, mq, tbc, prec, recon):
    torch = torch_cuda()
    worst = _step_and_check(torch, dims, ns, mq, tbc, prec, recon)
    print("worst error / bound per field:", {k: round(v, 3) for k, v in worst.items()})


@pytest.mark.parametrize("dims,ns,mq,prec", [((4, 4, 4, 4), 8, 0.5, "f16"), ((6, 4, 2, 10), 16, 0.04, "bf16")])
def test_mixed_step_fp16_links(dims, ns, mq, prec):
    """FP16 links of 12 reals: the same per-stage bounds with the links as the kernel stores them
    (the composition check against S^dag S on exact links absorbs the link rounding)."""
    torch = torch_cuda()
    worst = _step_and_check(torch, dims, ns, mq, True, prec, 12, link_prec="f16")
    print("worst error / bound per field:", {k: round(v, 3) for k, v in worst.items()})


def test_mixed_step_full_size_16x16x16x32():
    """The benchmark's lattice and launch configuration (16^3 x 32, Ns = 16, FP16, 12-real links),
    heavy mass so the corner terms are visible; every component of every stored field."""
    torch = torch_cuda()
    worst = _step_and_check(torch, (16, 16, 16, 32), 16, 0.5, True, "f16", 12, seed=2, eps=0.25)
    print("worst error / bound per field:", {k: round(v, 3) for k, v in worst.items()})


def test_mixed_step_rejects_unsupported():
    torch = torch_cuda()
    dims, ns = (4, 4, 4, 4), 4
    U, w = make_case(dims, ns, 0.1)
    h = odwf.Handle(dims, ns, M0, 0.1, w)
    h.set_gauge(U)
    f = syn.gaussian_spinor_even(ns, dims, 1)
    with pytest.raises(odwf.OdwfError):  # the production kernels need Ns = 8 or 16
        h.mixed_cg_step(f, f, f, [None] * 8, 0.5, 1.0, prec="f16")
    h.close()
    h = odwf.Handle(dims, 8, M0, 0.1, make_case(dims, 8, 0.1)[1])
    h.set_gauge(U)
    f = syn.gaussian_spinor_even(8, dims, 1)
    with pytest.raises(odwf.OdwfError):  # rr must be positive
        h.mixed_cg_step(f, f, f, [None] * 8, 0.5, 0.0, prec="f16")
    with pytest.raises(odwf.OdwfError):  # FP64 is not an inner storage format
        h.mixed_cg_step(f, f, f, [None] * 8, 0.5, 1.0, prec="f64")
    h.close()


@pytest.mark.parametrize("prec,link_prec", [("f16", "f32"), ("bf16", "f32"), ("f16", "f16")])
def test_mixed_iterations_track_fp64_on_4x4x4x4(prec, link_prec):
    """An inner-operator defect would cost iterations that the FP64 reliable updates then hide.
    FP16 storage (unit roundoff 2^-11) must stay within 10% (+2) of the FP64 CG's iteration
    count; BF16 (2^-8, eight times coarser) loses more per restart and is held to 75% (+2)
    (measured: 158 against 99 on this system)."""
    torch = torch_cuda()
    dims, ns, mq = (4, 4, 4, 4), 8, 0.01
    U, w = make_case(dims, ns, mq, eps=0.3, seed=1)
    h = odwf.Handle(dims, ns, M0, mq, w)
    h.set_gauge(torch.from_numpy(U).cuda())
    b = torch.from_numpy(syn.gaussian_spinor_even(ns, dims, 100)).cuda()
    x = torch.zeros_like(b)
    s64 = h.cg_solve(x, b, tol=1e-10, max_iter=20000, prec="f64")
    smx = h.cg_solve(x, b, tol=1e-10, max_iter=20000, prec=prec, link_prec=link_prec)
    h.close()
    margin = 1.1 if prec == "f16" else 1.75
    assert smx["iters"] <= margin * s64["iters"] + 2, (smx, s64)
