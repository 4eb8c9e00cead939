"""Writes zolotarev_weights.json from the oracle's Zolotarev generator (oracle/ only).

The fixture records the weights of the workloads used in the tests and benchmark, so
that a change in the generator shows up as a diff.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import zolotarev  # noqa: E402

CASES = [
    # (Ns, lambda_min, lambda_max, shifted)
    (4, 0.05, 6.0, True),
    (8, 0.05, 6.0, True),
    (8, 0.05, 6.0, False),
    (16, 0.05, 6.0, True),
    (16, 0.05, 6.2, True),  # the paper's lambda_max/lambda_min = 6.20/0.05 (Sec. 2)
    (16, 0.05, 6.2, False),
]


def main():
    out = {"source": "oracle.zolotarev.omega", "cases": []}
    for ns, lmin, lmax, shifted in CASES:
        w, dz = zolotarev.omega(ns, lmin, lmax, shifted)
        out["cases"].append({"Ns": ns, "lmin": lmin, "lmax": lmax, "shifted": shifted,
                             "omega": [float(v) for v in w], "d_Z": float(dz)})
    with open(os.path.join(HERE, "zolotarev_weights.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
