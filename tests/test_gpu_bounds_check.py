"""The bounds-checked debug build (libodwf_check.so, ODWF_BOUNDS_CHECK) on a GPU: every gathered
index is checked in the kernels and an out-of-range one would be reported by the call as
ODWF_ECUDA.  A child process loads that build (ODWF_LIBRARY) and runs the production paths --
the FP64 operator, mixed-precision solves at Ns = 8 and 16 (one- and two-s-per-lane hops), a
batched solve over a ragged lattice and the effective operator -- and every call succeeds with
results that meet their residual bars."""
import os
import subprocess
import sys

import pytest

from gpu_common import torch_cuda

pytestmark = pytest.mark.gpu

_CHILD = r"""
import sys
sys.path.insert(0, %r)
import numpy as np
import odwf_synth as syn
import paper_1811_08095_gb300 as odwf
from oracle import zolotarev
lib = odwf.load()
assert b"bounds-checked" in lib.odwf_version(), lib.odwf_version()
M0 = 1.3
for dims, ns in [((4, 4, 4, 4), 8), ((6, 4, 2, 10), 16)]:
    U = syn.gauge_field(dims, 0.3, 1)
    w, _ = zolotarev.omega(ns, 0.05, 6.2, True)
    h = odwf.Handle(dims, ns, M0, 0.1, w)
    h.set_gauge(U)
    psi = syn.gaussian_spinor(ns, dims, 3)
    out = np.zeros_like(psi)
    h.apply(out, psi, odwf.ODWF_MODE_FULL)
    bs = [syn.gaussian_spinor_even(ns, dims, 10 + k) for k in range(3)]
    xs = [np.zeros_like(b) for b in bs]
    st = h.cg_solve_batched(xs, bs, [0.01, 0.1, 0.5], tol=1e-10, max_iter=20000, prec="f16")
    assert all(s["status"] == 0 and s["true_resid"] <= 1e-10 for s in st), st
    x4 = np.zeros((dims[3], dims[2], dims[1], dims[0], 4, 3), dtype=np.complex128)
    b4 = syn.gaussian_spinor(1, dims, 5)[0]
    st = h.effective_solve(x4, b4, tol=1e-10, prec="f16")
    assert st["rc"] == 0, st
    h.close()
print("CHECKED-OK")
"""


def test_bounds_checked_build_runs_clean():
    torch_cuda()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    from paper_1811_08095_gb300 import build as b

    b.build(bounds_check=True)
    env = dict(os.environ, ODWF_LIBRARY=b.LIB_CHECK)
    out = subprocess.run([sys.executable, "-c", _CHILD % root], env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0 and "CHECKED-OK" in out.stdout, out.stdout[-2000:] + out.stderr[-3000:]
