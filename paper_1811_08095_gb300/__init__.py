"""GB300-native optimal domain-wall fermion (ODWF) operator and D^dag D solvers.

Thin Python layer over the C ABI in include/odwf.h (libodwf.so, built in-tree for
sm_103a).  Functions named like the C entry points take the same arguments; `Handle`
and `Server` wrap them for convenience.  Every computation runs in the library's CUDA
kernels; this module only marshals arguments.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _lib
from ._lib import (ODWF_BF16, ODWF_F16, ODWF_F32, ODWF_F64, ODWF_MODE_FULL, ODWF_MODE_SCHUR_EVEN,
                   ODWF_OMEGA_PLAIN, ODWF_OMEGA_SHIFTED_R5, ODWF_SYS_FULL_DIRAC, ODWF_SYS_FULL_NORMAL,
                   ODWF_SYS_SCHUR_NORMAL, OdwfError, check, ptr, stream_ptr)

__all__ = ["Handle", "Server", "Flow", "odwf_flow_t0", "odwf_zolotarev_omega", "OdwfError", "ODWF_F64", "ODWF_F32", "ODWF_F16",
           "ODWF_BF16", "ODWF_MODE_FULL", "ODWF_MODE_SCHUR_EVEN", "ODWF_SYS_SCHUR_NORMAL",
           "ODWF_SYS_FULL_NORMAL", "ODWF_SYS_FULL_DIRAC", "ODWF_OMEGA_SHIFTED_R5", "ODWF_OMEGA_PLAIN",
           "load", "lib_path"]

PREC = {"f64": ODWF_F64, "f32": ODWF_F32, "f16": ODWF_F16, "bf16": ODWF_BF16, "ff": _lib.ODWF_FF}


def load(build_if_missing: bool = False):
    return _lib.load(build_if_missing)


def lib_path() -> str:
    return _lib.LIB_PATH


def odwf_version() -> str:
    return _lib.load().odwf_version().decode()


def odwf_zolotarev_omega(ns: int, lmin: float, lmax: float, variant: int = ODWF_OMEGA_SHIFTED_R5):
    """Optimal weights omega_s (host computation).  Returns (omega[Ns], d_Z)."""
    out = np.zeros(ns, dtype=np.float64)
    dz = ctypes.c_double(0.0)
    check(_lib.load().odwf_zolotarev_omega(int(ns), float(lmin), float(lmax), int(variant), ptr(out),
                                           ctypes.byref(dz)))
    return out, dz.value


def _obs_dict(o):
    return {k: getattr(o, k) for k, _ in _lib.odwf_flow_obs._fields_}


def odwf_flow_t0(obs, target: float = 0.3):
    """Flow time where t^2 <E_clover> first reaches `target` (host interpolation between the two
    bracketing records of `obs`, a list of measurement dicts), or None when it is not reached."""
    arr = (_lib.odwf_flow_obs * max(1, len(obs)))()
    for i, o in enumerate(obs):
        for k, _ in _lib.odwf_flow_obs._fields_:
            setattr(arr[i], k, float(o[k]))
    t0 = ctypes.c_double(0.0)
    rc = _lib.load().odwf_flow_t0(arr, len(obs), float(target), ctypes.byref(t0))
    if rc == _lib.ODWF_ENOTFOUND:
        return None
    check(rc)
    return t0.value


class Flow:
    """Gradient flow of a gauge field and its observables (odwf_flow_create ... odwf_flow_destroy)."""

    def __init__(self, dims):
        self._lib = _lib.load()
        self.dims = tuple(int(d) for d in dims)
        d = (ctypes.c_int32 * 4)(*self.dims)
        h = ctypes.c_void_p()
        check(self._lib.odwf_flow_create(d, ctypes.byref(h)))
        self._h = h

    @property
    def volume(self):
        return math.prod(self.dims)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.odwf_flow_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_gauge(self, U, stream=None):
        check(self._lib.odwf_flow_set_gauge(self._h, ptr(U), stream_ptr(stream)))

    def get_gauge(self, U, stream=None):
        check(self._lib.odwf_flow_get_gauge(self._h, ptr(U), stream_ptr(stream)))
        return U

    def measure(self, t=0.0, e_site=None, q_site=None, stream=None):
        o = _lib.odwf_flow_obs()
        check(self._lib.odwf_flow_measure(self._h, float(t), ctypes.byref(o), ptr(e_site), ptr(q_site),
                                          stream_ptr(stream)))
        return _obs_dict(o)

    def run(self, eps, nsteps, measure_every=0, t_start=0.0, stream=None):
        """Integrate nsteps flow steps; returns the list of measurements (empty when
        measure_every is 0)."""
        need = 0
        if measure_every > 0:
            need = (nsteps - 1) // measure_every + 1 if nsteps > 0 else 0
            need += 1 if nsteps % measure_every == 0 else 0
        arr = (_lib.odwf_flow_obs * max(1, need))()
        n = ctypes.c_int(0)
        check(self._lib.odwf_flow_run(self._h, float(eps), int(nsteps), int(measure_every), float(t_start), arr,
                                      need, ctypes.byref(n), stream_ptr(stream)))
        return [_obs_dict(arr[i]) for i in range(n.value)]


def _lattice(dims, t_antiperiodic):
    lat = _lib.odwf_lattice()
    for i in range(4):
        lat.dims[i] = int(dims[i])
    lat.t_antiperiodic = 1 if t_antiperiodic else 0
    return lat


UPDATES = {"auto": _lib.ODWF_UPDATES_AUTO, "f64": _lib.ODWF_UPDATES_F64, "ff": _lib.ODWF_UPDATES_FF}


def _params(tol, max_iter, prec, delta, system, link_recon, mq, check_every, link_prec="f32", updates="auto"):
    p = _lib.odwf_solve_params()
    p.tol = float(tol)
    p.max_iter = int(max_iter)
    p.prec = PREC[prec] if isinstance(prec, str) else int(prec)
    p.delta = float(delta)
    p.system = int(system)
    p.link_recon = int(link_recon)
    p.mq = float("nan") if mq is None else float(mq)
    p.check_every = int(check_every)
    p.link_prec = PREC[link_prec] if isinstance(link_prec, str) else int(link_prec)
    p.update_arith = UPDATES[updates] if isinstance(updates, str) else int(updates)
    return p


def _stats_dict(s):
    return {"iters": s.iters, "n_reliable": s.n_reliable, "true_resid": s.true_resid, "time_ms": s.time_ms,
            "status": s.status}


class Handle:
    """One lattice / Ns / m0 / weights configuration (odwf_create ... odwf_destroy)."""

    def __init__(self, dims, ns, m0, mq, omega, t_antiperiodic=True):
        self._lib = _lib.load()
        self.dims = tuple(int(d) for d in dims)
        self.ns = int(ns)
        self.m0 = float(m0)
        self.mq = float(mq)
        self.omega = np.ascontiguousarray(omega, dtype=np.float64)
        lat = _lattice(dims, t_antiperiodic)
        h = ctypes.c_void_p()
        check(self._lib.odwf_create(ctypes.byref(lat), self.ns, self.m0, self.mq, ptr(self.omega), ctypes.byref(h)))
        self._h = h

    @property
    def volume(self):
        return math.prod(self.dims)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.odwf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_gauge(self, U, stream=None):
        check(self._lib.odwf_set_gauge(self._h, ptr(U), stream_ptr(stream)))

    def apply(self, out, inp, mode=ODWF_MODE_FULL, stream=None):
        check(self._lib.odwf_apply(self._h, ptr(out), ptr(inp), int(mode), stream_ptr(stream)))
        return out

    def apply_dagger(self, out, inp, mode=ODWF_MODE_FULL, stream=None):
        check(self._lib.odwf_apply_dagger(self._h, ptr(out), ptr(inp), int(mode), stream_ptr(stream)))
        return out

    def apply_normal(self, out, inp, system=ODWF_SYS_SCHUR_NORMAL, stream=None):
        check(self._lib.odwf_apply_normal(self._h, ptr(out), ptr(inp), int(system), stream_ptr(stream)))
        return out

    def apply_normal_prec(self, out, inp, prec="f16", link_recon=12, stream=None):
        p = PREC[prec] if isinstance(prec, str) else int(prec)
        check(self._lib.odwf_apply_normal_prec(self._h, ptr(out), ptr(inp), p, int(link_recon), stream_ptr(stream)))
        return out

    def apply_m5(self, out, inp, n_sites, op, stream=None):
        check(self._lib.odwf_apply_m5(self._h, ptr(out), ptr(inp), int(n_sites), int(op), stream_ptr(stream)))
        return out

    def mixed_cg_step(self, p_prev, r, x, outs, beta, rr, prec="f16", link_recon=12, mq=None, stream=None,
                      link_prec="f32"):
        """odwf_mixed_cg_step: one production mixed CG iteration; `outs` is a list of 8 fields
        (or None) receiving p_prev as stored, p, chi_p, chi_t, a, c, r_new, x_new.  Returns the
        scalars as a dict."""
        assert len(outs) == 8
        oa = (ctypes.c_void_p * 8)(*[(ptr(o).value if o is not None else None) for o in outs])
        sc = _lib.odwf_cg_step_scalars()
        sc.beta = float(beta)
        sc.rr = float(rr)
        pr = PREC[prec] if isinstance(prec, str) else int(prec)
        lp = PREC[link_prec] if isinstance(link_prec, str) else int(link_prec)
        check(self._lib.odwf_mixed_cg_step(self._h, pr, int(link_recon), lp, self.mq if mq is None else float(mq),
                                           ptr(p_prev), ptr(r), ptr(x), ctypes.cast(oa, ctypes.c_void_p),
                                           ctypes.byref(sc), stream_ptr(stream)))
        return {"pAp": sc.pAp, "alpha": sc.alpha, "rr_new": sc.rr_new, "status": sc.status}

    def time_kernel(self, kind, fill, prec="f16", link_recon=12, link_prec="f32", nsys=1, reps=10, stream=None):
        """odwf_time_kernel: CUDA-event time of `reps` launches of one production mixed kernel
        (kind 1..4 = K1..K4, 5 = p update).  Returns the odwf_kernel_prof fields as a dict."""
        out = _lib.odwf_kernel_prof()
        pr = PREC[prec] if isinstance(prec, str) else int(prec)
        lp = PREC[link_prec] if isinstance(link_prec, str) else int(link_prec)
        check(self._lib.odwf_time_kernel(self._h, int(kind), pr, int(link_recon), lp, int(nsys), int(reps), ptr(fill),
                                         ctypes.byref(out), stream_ptr(stream)))
        return {"name": out.name.decode(), "launches": out.launches, "system_launches": out.system_launches,
                "total_ms": out.total_ms, "bytes_per_system": out.bytes_per_system,
                "bytes_per_launch": out.bytes_per_launch}

    def effective_solve(self, x, b, tol=1e-10, max_iter=100000, prec="f64", mq=None, stream=None,
                        raise_on_error=True, link_prec="f32"):
        """odwf_effective_solve: x = D_eff(m_q)^-1 b on 4D fields (Lt, Lz, Ly, Lx, 4, 3)."""
        p = _params(tol, max_iter, prec, 0.01, ODWF_SYS_FULL_DIRAC, 12, mq, 8, link_prec)
        st = _lib.odwf_solve_stats()
        rc = self._lib.odwf_effective_solve(self._h, ptr(x), ptr(b), ctypes.byref(p), ctypes.byref(st),
                                            stream_ptr(stream))
        if raise_on_error:
            check(rc)
        d = _stats_dict(st)
        d["rc"] = rc
        return d

    def pf_force(self, phi, m1, m2, force=None, tol=1e-10, max_iter=100000, prec="f64", updates="auto",
                 stream=None):
        """odwf_pf_force: the two-flavour pseudofermion action phi^+ S2^+ (S1^+ S1)^-1 S2 phi and,
        when `force` (a complex128 buffer of the gauge field's shape) is given, its force.
        Returns (action, stats dict)."""
        p = _params(tol, max_iter, prec, 0.01, ODWF_SYS_SCHUR_NORMAL, 12, None, 8, "f32", updates)
        st = _lib.odwf_solve_stats()
        act = ctypes.c_double(0.0)
        check(self._lib.odwf_pf_force(self._h, ptr(phi), float(m1), float(m2), ctypes.byref(p), ctypes.byref(act),
                                      ptr(force), ctypes.byref(st), stream_ptr(stream)))
        return act.value, _stats_dict(st)

    def pf_heatbath(self, eta, m1, m2, phi, tol=1e-10, max_iter=100000, prec="f64", updates="auto", stream=None):
        """odwf_pf_heatbath: phi = S(m2)^-1 S(m1)^+ eta into `phi` (an even-site buffer); returns the
        solve's stats dict."""
        p = _params(tol, max_iter, prec, 0.01, ODWF_SYS_SCHUR_NORMAL, 12, None, 8, "f32", updates)
        st = _lib.odwf_solve_stats()
        check(self._lib.odwf_pf_heatbath(self._h, ptr(eta), float(m1), float(m2), ctypes.byref(p), ptr(phi),
                                         ctypes.byref(st), stream_ptr(stream)))
        return _stats_dict(st)

    def hmc_trajectory(self, U, P, etas, masses, beta, tau, nsteps, u, integrator="omelyan", n_inner=0, tol=1e-10,
                       prec="f16", stream=None):
        """One HMC trajectory (Sec. 2).  The caller draws the momenta P (device, traceless
        anti-Hermitian), one Gaussian even-site field per pseudofermion term in etas (device),
        and u uniform in [0, 1).  Heat bath phi_i = S(m2_i)^-1 S(m1_i)^+ eta_i for masses =
        [(m1_i, m2_i), ...], the molecular dynamics of odwf_md_trajectory, then the Metropolis
        test u < exp(-dH); a rejected trajectory leaves U as it was.  Returns (accepted, dH)."""
        import math

        self.set_gauge(U, stream=stream)
        phis = []
        for eta, (m1, m2) in zip(etas, masses):
            phi = eta.new_empty(eta.shape)
            self.pf_heatbath(eta, m1, m2, phi, tol=tol, prec=prec, stream=stream)
            phis.append(phi)
        U0 = U.clone()
        h0, h1, _ = self.md_trajectory(U, P, [(phi, m1, m2) for phi, (m1, m2) in zip(phis, masses)], beta, tau,
                                       nsteps, integrator, n_inner=n_inner, tol=tol, prec=prec, stream=stream)
        dH = h1 - h0
        accepted = dH <= 0.0 or u < math.exp(-dH)
        if not accepted:
            U.copy_(U0)
            self.set_gauge(U, stream=stream)
        return accepted, dH

    def gauge_force(self, U, beta, force=None, stream=None):
        """odwf_gauge_force: the Wilson plaquette action of U (host array or device tensor of the
        gauge field's shape) and, when `force` is given, its force Pi into it.  Returns the action."""
        act = ctypes.c_double(0.0)
        check(self._lib.odwf_gauge_force(self._h, ptr(U), float(beta), ctypes.byref(act), ptr(force),
                                         stream_ptr(stream)))
        return act.value

    def md_trajectory(self, U, P, terms, beta, tau, nsteps, integrator="omelyan", n_inner=0, tol=1e-10,
                      max_iter=100000, prec="f64", updates="auto", stream=None):
        """odwf_md_trajectory: integrate (U, P) (device tensors, updated in place) over time tau in
        nsteps steps; terms = [(phi, m1, m2), ...]; n_inner > 0: the gauge force on an inner time
        scale of n_inner steps per drift (Sexton-Weingarten).  Returns (H_start, H_end, stats
        dict of the trajectory's solves)."""
        n = len(terms)
        integ = {"leapfrog": 0, "omelyan": 1}[integrator]
        p = _params(tol, max_iter, prec, 0.01, ODWF_SYS_SCHUR_NORMAL, 12, None, 8, "f32", updates)
        phis = (ctypes.c_void_p * max(n, 1))(*[ptr(t[0]).value for t in terms])
        m1 = np.ascontiguousarray([t[1] for t in terms] or [0.0], dtype=np.float64)
        m2 = np.ascontiguousarray([t[2] for t in terms] or [0.0], dtype=np.float64)
        en = np.zeros(2, dtype=np.float64)
        st = _lib.odwf_solve_stats()
        check(self._lib.odwf_md_trajectory(self._h, ptr(U), ptr(P), n, ctypes.cast(phis, ctypes.c_void_p), ptr(m1),
                                           ptr(m2), float(beta), float(tau), int(nsteps), integ, int(n_inner),
                                           ctypes.byref(p), ptr(en), ctypes.byref(st), stream_ptr(stream)))
        return float(en[0]), float(en[1]), _stats_dict(st)

    def residual_mass(self, site, tol=1e-10, max_iter=100000, prec="f64", mq=None, stream=None):
        """odwf_residual_mass at site (x, y, z, t): returns (m_res, C(t) array, stats dict)."""
        p = _params(tol, max_iter, prec, 0.01, ODWF_SYS_FULL_DIRAC, 12, mq, 8)
        st = _lib.odwf_solve_stats()
        s4 = (ctypes.c_int32 * 4)(*[int(v) for v in site])
        mres = ctypes.c_double(0.0)
        corr = np.zeros(self.dims[3], dtype=np.float64)
        check(self._lib.odwf_residual_mass(self._h, ctypes.cast(s4, ctypes.c_void_p), ctypes.byref(p),
                                           ctypes.byref(mres), ptr(corr), ctypes.byref(st), stream_ptr(stream)))
        return mres.value, corr, _stats_dict(st)

    def cg_solve(self, x, b, tol=1e-10, max_iter=100000, prec="f64", delta=0.01, system=ODWF_SYS_SCHUR_NORMAL,
                 link_recon=12, mq=None, check_every=8, stream=None, raise_on_error=True, link_prec="f32",
                 updates="auto"):
        p = _params(tol, max_iter, prec, delta, system, link_recon, mq, check_every, link_prec, updates)
        st = _lib.odwf_solve_stats()
        rc = self._lib.odwf_cg_solve(self._h, ptr(x), ptr(b), ctypes.byref(p), ctypes.byref(st), stream_ptr(stream))
        if raise_on_error:
            check(rc)
        d = _stats_dict(st)
        d["rc"] = rc
        return d

    def cg_solve_batched(self, xs, bs, mqs=None, tol=1e-10, max_iter=100000, prec="f64", delta=0.01,
                         link_recon=12, check_every=8, stream=None, raise_on_error=True, link_prec="f32",
                         updates="auto"):
        n = len(xs)
        assert len(bs) == n
        xa = (ctypes.c_void_p * n)(*[ptr(x).value for x in xs])
        ba = (ctypes.c_void_p * n)(*[ptr(b).value for b in bs])
        mq_arr = None
        if mqs is not None:
            mq_np = np.ascontiguousarray(mqs, dtype=np.float64)
            assert mq_np.shape == (n,)
            mq_arr = ptr(mq_np)
        p = _params(tol, max_iter, prec, delta, ODWF_SYS_SCHUR_NORMAL, link_recon, None, check_every, link_prec,
                    updates)
        st = (_lib.odwf_solve_stats * n)()
        rc = self._lib.odwf_cg_solve_batched(self._h, n, ctypes.cast(xa, ctypes.c_void_p),
                                             ctypes.cast(ba, ctypes.c_void_p), mq_arr, ctypes.byref(p),
                                             ctypes.cast(st, ctypes.c_void_p), stream_ptr(stream))
        if raise_on_error:
            check(rc)
        out = [_stats_dict(s) for s in st]
        for d in out:
            d["rc"] = rc
        return out


class Server:
    """Serving loop (serve_create ... serve_destroy): resident gauge fields, continuous batching."""

    def __init__(self, hbm_budget_bytes=0):
        self._lib = _lib.load()
        h = ctypes.c_void_p()
        check(self._lib.serve_create(ctypes.c_size_t(int(hbm_budget_bytes)), ctypes.byref(h)))
        self._h = h
        self._keep = {}

    def register_gauge(self, field_id, dims, U, t_antiperiodic=True):
        lat = _lattice(dims, t_antiperiodic)
        check(self._lib.serve_register_gauge(self._h, int(field_id), ctypes.byref(lat), ptr(U)))

    def submit(self, field_id, ns, m0, mq, omega, bs, xs, tol=1e-10, prec="f16", max_iter=100000):
        n = len(bs)
        om = np.ascontiguousarray(omega, dtype=np.float64)
        ba = (ctypes.c_void_p * n)(*[ptr(b).value for b in bs])
        xa = (ctypes.c_void_p * n)(*[ptr(x).value for x in xs])
        req = _lib.odwf_request()
        req.field_id = int(field_id)
        req.Ns = int(ns)
        req.m0 = float(m0)
        req.mq = float(mq)
        req.omega = om.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        req.nrhs = n
        req.b = ctypes.cast(ba, ctypes.POINTER(ctypes.c_void_p))
        req.x = ctypes.cast(xa, ctypes.POINTER(ctypes.c_void_p))
        req.tol = float(tol)
        req.prec = PREC[prec] if isinstance(prec, str) else int(prec)
        req.max_iter = int(max_iter)
        t = ctypes.c_uint64(0)
        check(self._lib.serve_submit(self._h, ctypes.byref(req), ctypes.byref(t)))
        self._keep[t.value] = (om, ba, xa, bs, xs)
        return t.value

    def set_policy(self, admit_deadline_ms=0.0, max_queued=0, fair=False):
        check(self._lib.serve_set_policy(self._h, float(admit_deadline_ms), int(max_queued), 1 if fair else 0))

    def cancel(self, ticket):
        check(self._lib.serve_cancel(self._h, ctypes.c_uint64(ticket)))

    def try_submit(self, *a, **k):
        """submit(), returning (status, ticket) instead of raising (ODWF_EBUSY when the queue is full)."""
        try:
            return _lib.ODWF_OK, self.submit(*a, **k)
        except OdwfError as e:
            return e.code, None

    def poll(self, ticket, timeout_ms=0):
        r = _lib.odwf_result()
        rc = self._lib.serve_poll(self._h, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(r))
        return rc, {"status": r.status, "iters": r.iters, "true_resid": r.true_resid, "latency_ms": r.latency_ms,
                    "queue_ms": r.queue_ms}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.serve_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
