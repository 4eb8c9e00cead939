"""A short, fixed solver run for profiling the kernels (e.g. under ncu).

Runs the batched mixed-precision CG for a given number of iterations (it stops at
max_iter, so the run is short and its launch sequence is fixed) on a synthetic
workload, and exits 0:

    python -m paper_1811_08095_gb300.profile_case --dims 16 16 16 32 --ns 16 --nsys 3 --iters 4
"""
from __future__ import annotations

import argparse
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--dims", type=int, nargs=4, default=[16, 16, 16, 32])
    ap.add_argument("--ns", type=int, default=16)
    ap.add_argument("--nsys", type=int, default=3)
    ap.add_argument("--iters", type=int, default=4)
    ap.add_argument("--prec", default="f16")
    ap.add_argument("--eps", type=float, default=0.25)
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch

    import odwf_synth as syn
    import paper_1811_08095_gb300 as odwf

    dims = tuple(a.dims)
    w, _ = odwf.odwf_zolotarev_omega(a.ns, 0.05, 6.2)
    U = syn.gauge_field(dims, a.eps, 2)
    h = odwf.Handle(dims, a.ns, 1.3, 0.04, w)
    h.set_gauge(torch.from_numpy(U).cuda())
    masses = [0.002, 0.04, 0.5, 0.1, 0.01, 0.2][: a.nsys] + [0.05] * max(0, a.nsys - 6)
    bs = [torch.from_numpy(syn.gaussian_spinor_even(a.ns, dims, 100 + k)).cuda() for k in range(a.nsys)]
    xs = [torch.zeros_like(b) for b in bs]
    st = h.cg_solve_batched(xs, bs, masses, tol=1e-10, max_iter=a.iters, prec=a.prec, check_every=a.iters,
                            raise_on_error=False)
    torch.cuda.synchronize()
    print("profile_case: iters %s" % [s["iters"] for s in st])
    h.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
