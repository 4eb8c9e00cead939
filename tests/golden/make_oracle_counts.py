"""Writes oracle_cg_16x16x16x32_ns16.json: the FP64 oracle's CG on the 16^3 x 32 x 16
workload (links exp(0.25 i H) seed 2, m0 = 1.3, shifted weights on [0.05, 6.2], Gaussian
right-hand sides seeds 100 + k for m_q = 0.002, 0.04, 0.5), calling only oracle/.

For each mass it records the oracle's iteration count to a relative residual of 1e-10
(capped at --cap iterations; a capped run records "capped": true and its count is a lower
bound), the recomputed true residual, seconds per iteration on this machine, and, for a
converged run, 512 sampled components of the solution with their flat indices, which the
GPU tests compare against at full size.

    python tests/golden/make_oracle_counts.py [--cap 400] [--masses 0.5,0.04,0.002]
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import odwf_synth as syn  # noqa: E402
import oracle  # noqa: E402
from oracle import zolotarev  # noqa: E402

DIMS = (16, 16, 16, 32)
NS = 16
M0 = 1.3
EPS = 0.25
SEED = 2
LRANGE = (0.05, 6.2)
MASSES = (0.002, 0.04, 0.5)
OUT = os.path.join(HERE, "oracle_cg_16x16x16x32_ns16.json")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--cap", type=int, default=400)
    ap.add_argument("--masses", default="0.5,0.04,0.002")
    a = ap.parse_args()
    U = syn.gauge_field(DIMS, EPS, SEED)
    w, _ = zolotarev.omega(NS, LRANGE[0], LRANGE[1], True)
    data = {"workload": "16^3x32, Ns=16, m0=1.3, eps=0.25 seed 2, shifted omega on [0.05, 6.2]",
            "threads": oracle.num_threads(), "systems": []}
    if os.path.exists(OUT):
        data = json.load(open(OUT))
    done = {s["mq"] for s in data["systems"]}
    for mq in [float(m) for m in a.masses.split(",")]:
        if mq in done:
            continue
        k = MASSES.index(mq)
        b = syn.gaussian_spinor_even(NS, DIMS, 100 + k)
        t = time.time()
        x, it, res = oracle.cg(U, b, M0, mq, w, tol=1e-10, max_iter=a.cap)
        dt = time.time() - t
        n_it = it if it >= 0 else a.cap
        rec = {"mq": mq, "rhs_seed": 100 + k, "iters": n_it, "capped": it < 0, "true_resid": res,
               "seconds_per_iter": dt / (n_it + 2), "threads": oracle.num_threads()}
        if it >= 0:
            rng = np.random.default_rng(12345 + k)
            flat = x.reshape(-1)
            idx = np.sort(rng.choice(flat.size, 512, replace=False))
            rec["sample_index"] = [int(i) for i in idx]
            rec["sample_re"] = [float(v) for v in flat[idx].real]
            rec["sample_im"] = [float(v) for v in flat[idx].imag]
        data["systems"].append(rec)
        with open(OUT, "w") as f:
            json.dump(data, f)
        print("m_q=%g iters=%d capped=%s resid=%.2e %.1fs" % (mq, n_it, it < 0, res, dt), flush=True)


if __name__ == "__main__":
    main()
