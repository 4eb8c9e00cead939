"""GPU parity of the gradient flow and its observables (odwf_flow_*, Sec. 2-3) against the FP64
oracle in oracle/flow.py, through the C ABI.

Tolerances.  The kernels compute the force, the exponential and the observables in FP32
(unit roundoff u = 2^-24) and keep the links as float-float pairs, so the links drift from an
FP64 integration only through the FP32 rounding of each stage increment: per step at most about
64 u * eps * max|Z| in an entry (the force sums 36 products of O(1) matrices, each rounded, and the
three stage exponents weigh it by 1/4 + 8/9 + 3/4 + 17/36 + 1 < 4).  The bound used is
n * eps * max|Z| * 64 u + 8 u.  Site densities are FP32 sums of O(10) terms: relative 2e-6 of the
field's scale; lattice averages and the charge are summed in FP64 from them.
"""
import numpy as np
import pytest

import odwf_synth as syn
import paper_1811_08095_gb300 as odwf
from gpu_common import torch_cuda
from oracle import flow as fl

pytestmark = pytest.mark.gpu
L = odwf._lib
U32 = 2.0 ** -24
FULL = (64, 64, 64, 64)  # the flow benchmark's lattice (the paper's 64^4), eps = 0.01
FULL_EPS = 0.01


def _link_tol(nsteps, eps, zmax):
    return nsteps * eps * zmax * 64 * U32 + 8 * U32


def _gpu_flow(torch, U, eps, nsteps, every):
    f = odwf.Flow(fl.dims_of(U))
    f.set_gauge(torch.from_numpy(U).cuda())
    obs = f.run(eps, nsteps, measure_every=every)
    out = torch.empty(U.shape, dtype=torch.complex128, device="cuda")
    f.get_gauge(out)
    torch.cuda.synchronize()
    f.close()
    return out.cpu().numpy(), obs


@pytest.mark.parametrize("dims", [(6, 4, 8, 5), (5, 3, 4, 6), (4, 6, 4, 8), (2, 2, 2, 2)])
def test_flow_matches_oracle(dims):
    """Ten steps on small lattices (ragged last block, odd extents, time slabs of 1, 2 and 8, and
    the minimal 2^4 lattice, where x + mu and x - mu are the same site)."""
    torch = torch_cuda()
    U = syn.gauge_field(dims, 0.6, 101)
    eps, n, every = 0.02, 10, 5
    V_ref, obs_ref = fl.flow(U, eps, n, measure_every=every)
    V_gpu, obs = _gpu_flow(torch, U, eps, n, every)
    zmax = np.abs(fl.force(U)).max()
    err = np.abs(V_gpu - V_ref).max()
    assert err < _link_tol(n, eps, zmax), (err, _link_tol(n, eps, zmax))
    assert np.abs(V_gpu - U).max() > 100 * err  # the field moved
    assert len(obs) == len(obs_ref) == 3
    for o, r in zip(obs, obs_ref):
        assert abs(o["t"] - r["t"]) < 1e-12
        for k in ("e_plaq", "e_clover"):
            assert abs(o[k] - r[k]) < 2e-6 * abs(r[k]), (k, o[k], r[k])
        assert abs(o["q_clover"] - r["q"]) < 2e-6 * syn.volume(dims) * max(1e-3, abs(r["q"]) / syn.volume(dims))
        assert abs(o["plaq_min"] - r["plaq_min"]) < 1e-6
        assert abs(o["plaq_mean"] - r["plaq_mean"]) < 1e-6


def test_measure_densities_match_oracle():
    torch = torch_cuda()
    dims = (6, 4, 8, 5)
    U = syn.gauge_field(dims, 0.5, 103)
    s = fl.site_observables(U)
    f = odwf.Flow(dims)
    f.set_gauge(U)  # host pointer path
    V = syn.volume(dims)
    e_site = torch.empty(V, dtype=torch.float32, device="cuda")
    q_host = np.empty(V, dtype=np.float32)  # host pointer path
    o = f.measure(0.5, e_site, q_host)
    e = e_site.cpu().numpy()
    assert abs(o["t"] - 0.5) < 1e-15
    assert np.abs(e - s["e_clover"]).max() < 2e-6 * np.abs(s["e_clover"]).max()
    assert np.abs(q_host - s["q"]).max() < 2e-6 * np.abs(s["q"]).max()
    assert abs(o["e_clover"] - s["e_clover"].mean()) < 2e-6 * s["e_clover"].mean()
    assert abs(o["e_plaq"] - s["e_plaq"].mean()) < 2e-6 * s["e_plaq"].mean()
    assert abs(o["q_clover"] - s["q"].sum()) < 2e-6 * np.abs(s["q"]).sum()
    assert abs(o["plaq_min"] - s["plaq_min"].min()) < 1e-6
    # the host copy of the field comes back through the float-float pairs at FP64 precision
    back = np.empty_like(U)
    f.get_gauge(back)
    assert np.abs(back - U).max() < 1e-13
    f.close()


@pytest.mark.parametrize("charges", [(1, -1, 0), (2, -1, -1)])
def test_flux_field_closed_forms_and_stationarity(charges):
    torch = torch_cuda()
    dims = (4, 4, 6, 6)
    fluxes = {(0, 1): 1, (0, 2): 2, (0, 3): -1, (1, 2): 1, (1, 3): 3, (2, 3): 1}
    U = syn.flux_field(dims, fluxes, charges)
    q = np.array(charges, dtype=np.float64)
    th = {p: 2 * np.pi * fluxes[p] / (dims[p[0]] * dims[p[1]]) for p in fl.PLANES}
    fv = {}
    for p in fl.PLANES:
        d = np.sin(q * th[p])
        fv[p] = d - d.sum() / 3
    e_clov = sum(fv[p] @ fv[p] for p in fl.PLANES)
    e_plaq = 2 * sum(3 - np.cos(q * th[p]).sum() for p in fl.PLANES)
    qd = (fv[(0, 1)] @ fv[(2, 3)] - fv[(0, 2)] @ fv[(1, 3)] + fv[(0, 3)] @ fv[(1, 2)]) / (4 * np.pi ** 2)
    V_gpu, obs = _gpu_flow(torch, U, 0.02, 5, 5)
    o = obs[0]
    assert abs(o["e_clover"] - e_clov) < 2e-6 * e_clov
    assert abs(o["e_plaq"] - e_plaq) < 2e-6 * e_plaq
    assert abs(o["q_clover"] - syn.volume(dims) * qd) < 1e-5
    assert abs(o["plaq_min"] - min(np.cos(q * th[p]).sum() / 3 for p in fl.PLANES)) < 1e-6
    assert np.abs(V_gpu - U).max() < _link_tol(5, 0.02, 3.0)  # a stationary point: nothing moves
    assert abs(obs[1]["q_clover"] - o["q_clover"]) < 1e-5


def test_pure_gauge_is_a_fixed_point():
    torch = torch_cuda()
    dims = (4, 2, 4, 6)
    lx, ly, lz, lt = dims
    Om = syn.gauge_field(dims, 2.0, 105)[0]
    U = np.empty((4, lt, lz, ly, lx, 3, 3), dtype=np.complex128)
    ax = {0: 3, 1: 2, 2: 1, 3: 0}
    for mu in range(4):
        U[mu] = Om @ np.conj(np.swapaxes(np.roll(Om, -1, axis=ax[mu]), -1, -2))
    V_gpu, obs = _gpu_flow(torch, U, 0.05, 4, 4)
    for o in obs:
        assert abs(o["e_clover"]) < 1e-10 and abs(o["e_plaq"]) < 1e-5 and abs(o["q_clover"]) < 1e-10
        assert abs(o["plaq_min"] - 1.0) < 1e-6
    assert np.abs(V_gpu - U).max() < 1e-6


@pytest.mark.slow
def test_noisy_flux_flows_to_integer_charge_like_the_oracle():
    """Sec. 3: after flow the field is admissible and the clover charge sits at the integer."""
    torch = torch_cuda()
    dims = (8, 8, 8, 8)
    U = syn.gauge_field(dims, 0.35, 71) @ syn.flux_field(dims, {(0, 1): 1, (2, 3): 1})
    _, obs_ref = fl.flow(U, 0.02, 50, measure_every=25)
    _, obs = _gpu_flow(torch, U, 0.02, 50, 25)
    o, r = obs[-1], obs_ref[-1]
    assert o["plaq_min"] > 44 / 45 and abs(o["q_clover"] - 2.0) < 0.02
    assert abs(o["q_clover"] - r["q"]) < 1e-4
    assert abs(o["e_clover"] - r["e_clover"]) < 1e-5 * r["e_clover"] + 1e-9


def test_long_flow_keeps_links_special_unitary_and_is_deterministic():
    """6000 stages: the float-float links stay on SU(3) without reprojection, and two runs give
    bit-identical observables (fixed-order reductions)."""
    torch = torch_cuda()
    dims = (8, 8, 8, 8)
    U = syn.gauge_field(dims, 0.5, 107)
    runs = []
    for _ in range(2):
        V_gpu, obs = _gpu_flow(torch, U, 0.01, 2000, 500)
        runs.append(obs)
    W = V_gpu.reshape(-1, 3, 3)
    unit = np.abs(W @ np.conj(np.swapaxes(W, -1, -2)) - np.eye(3)).max()
    det = np.abs(np.linalg.det(W) - 1).max()
    assert unit < 1e-6 and det < 1e-6, (unit, det)
    assert runs[0] == runs[1]
    e = [o["e_clover"] for o in runs[0]]
    assert all(b < a for a, b in zip(e, e[1:]))  # the flow smooths: E falls monotonically


def test_errors_are_reported():
    torch = torch_cuda()
    f = odwf.Flow((4, 4, 4, 4))
    with pytest.raises(odwf.OdwfError) as ei:
        f.measure()
    assert ei.value.code == L.ODWF_EINVAL  # no gauge field yet
    f.set_gauge(syn.gauge_field((4, 4, 4, 4), 0.3, 1))
    n = __import__("ctypes").c_int(0)
    arr = (L.odwf_flow_obs * 1)()
    rc = L.load().odwf_flow_run(f._h, 0.01, 10, 5, 0.0, arr, 1, __import__("ctypes").byref(n), None)
    assert rc == L.ODWF_EINVAL and n.value == 0  # needs 3 records
    rc = L.load().odwf_flow_run(f._h, -0.01, 1, 0, 0.0, None, 0, None, None)
    assert rc == L.ODWF_EINVAL
    with pytest.raises(odwf.OdwfError):
        odwf.Flow((4, 1, 4, 4))
    f.close()
    del torch


def _box(torch, Udev, c, hw):
    """The (2 hw + 1)^4 neighbourhood of site c = (x, y, z, t), as a periodic oracle lattice."""
    lt, lz, ly, lx = Udev.shape[1:5]
    r = torch.arange(-hw, hw + 1, device=Udev.device)
    B = Udev.index_select(1, (c[3] + r) % lt).index_select(2, (c[2] + r) % lz)
    B = B.index_select(3, (c[1] + r) % ly).index_select(4, (c[0] + r) % lx)
    return B.cpu().numpy()


def test_full_size_sampled_step_and_densities():
    """64^4 at eps = 0.01, the flow benchmark's configuration.  One step on the GPU; at sampled
    sites the oracle flows the 7^4 neighbourhood (whose centre a step cannot reach from outside:
    each of the three stages reaches one site further) and measures the densities on the 5^4
    neighbourhood; the lattice record must equal the sums of the per-site densities."""
    torch = torch_cuda()
    dims = FULL
    V = syn.volume(dims)
    Udev = syn.gauge_field_torch(dims, 0.2, 3, device="cuda")
    f = odwf.Flow(dims)
    f.set_gauge(Udev)
    e_site = torch.empty(V, dtype=torch.float32, device="cuda")
    q_site = torch.empty(V, dtype=torch.float32, device="cuda")
    o = f.measure(0.0, e_site, q_site)
    rng = np.random.default_rng(5)
    sites = [tuple(int(rng.integers(0, n)) for n in dims) for _ in range(12)]
    sites += [(0, 0, 0, 0), (63, 63, 63, 63), (0, 63, 7, 56)]  # wrap-around corners, slab edges
    lx, ly, lz, lt = dims
    e_all = e_site.cpu().numpy()
    q_all = q_site.cpu().numpy()
    for c in sites:
        B = _box(torch, Udev, c, 2)
        s = fl.site_observables(B, np.array([[2, 2, 2, 2]]))
        idx = ((c[3] * lz + c[2]) * ly + c[1]) * lx + c[0]
        assert abs(e_all[idx] - s["e_clover"][0]) < 2e-6 * max(1.0, s["e_clover"][0])
        assert abs(q_all[idx] - s["q"][0]) < 2e-6 * max(1e-2, abs(s["q"][0])) + 1e-9
    assert abs(o["e_clover"] - e_all.astype(np.float64).mean()) < 1e-6 * o["e_clover"]
    assert abs(o["q_clover"] - q_all.astype(np.float64).sum()) < 1e-6 * np.abs(q_all).sum()
    del e_site, q_site
    f.run(FULL_EPS, 1)
    Vdev = torch.empty_like(Udev)
    f.get_gauge(Vdev)
    torch.cuda.synchronize()
    worst, tol = 0.0, 0.0
    for c in sites[:8]:
        B = _box(torch, Udev, c, 3)
        zmax = np.abs(fl.force(B)).max()
        ref = fl.rk3_step(B, FULL_EPS)[:, 3, 3, 3, 3]
        got = Vdev[:, c[3], c[2], c[1], c[0]].cpu().numpy()
        worst = max(worst, np.abs(got - ref).max())
        tol = max(tol, _link_tol(1, FULL_EPS, zmax))
    assert worst < tol, (worst, tol)
    f.close()
