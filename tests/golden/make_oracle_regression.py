"""Writes oracle_regression.json: the FP64 oracle's outputs for a few fixed
tracks (p2z and p2r, both charges, forward and backward paths, a strongly
curved one).  The paper prints no worked example, so these values come from
the oracle itself (this script calls only oracle/): they pin the oracle
against unnoticed change, while test_oracle_pins.py pins it against closed
forms, an independent integration and invariants.  Re-run only for a change
of the oracle's arithmetic that a cited passage justifies.

    python tests/golden/make_oracle_regression.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

BZ = 3.8
# covariance: diag(1e-4, 1e-4, 2.5e-3, 1e-4 k^2, 1e-6, 1e-6) plus small correlations
def cov21(k):
    c = [0.0] * 21
    diag = [1e-4, 1e-4, 2.5e-3, 1e-4 * k * k, 1e-6, 1e-6]
    idx = lambda i, j: i * (i + 1) // 2 + j
    for i, v in enumerate(diag):
        c[idx(i, i)] = v
    c[idx(1, 0)] = 2e-5
    c[idx(4, 0)] = -3e-6
    c[idx(5, 2)] = 1e-5
    c[idx(4, 3)] = 1e-7 * k
    return c

CASES = [
    # kind, state (x, y, z, k, phi, theta), q, surface, hit offset; the hit is
    # the oracle's crossing moved by the offset (x, y for a plane; r*phi and z
    # on a cylinder), V_hit as in the single-step workloads
    ("p2z", [0.01, -0.02, 1.5, 1 / 2.0, 0.7, 0.3], 1, 50.0, (0.012, -0.007)),
    ("p2z", [0.0, 0.01, -3.0, 1 / 0.6, -2.5, 0.25], -1, 40.0, (-0.004, 0.015)),
    ("p2z", [0.02, 0.0, 60.0, 1 / 5.0, 1.2, 2.8], 1, 30.0, (0.009, 0.003)),  # plane behind
    ("p2r", [0.01, 0.0, 0.5, 1 / 3.0, 0.4, 1.2], 1, 30.0, (0.011, -0.04)),
    ("p2r", [-0.01, 0.01, -2.0, 1 / 0.7, 2.9, 1.9], -1, 30.0, (-0.006, 0.07)),
    ("p2r", [0.0, 0.0, 0.0, 1 / 0.45, -1.0, 1.5707], 1, 30.0, (0.008, 0.02)),  # strongly curved
]
HC_Z = [1e-4, 0.0, 1e-4, 0.0, 0.0, 1e-4]


def hit_for(kind, p, q, surf, off):
    import math
    if kind == "p2z":
        pp, _, st = oracle.propagate_to_z(p, q, BZ, surf)
        return [pp[0] + off[0], pp[1] + off[1], surf], HC_Z
    pp, _, st = oracle.propagate_to_r(p, q, BZ, surf)
    a = math.atan2(pp[1], pp[0]) + off[0] / surf
    u = (-math.sin(a), math.cos(a))
    hc = [1e-4 * u[0] * u[0], 1e-4 * u[0] * u[1], 1e-4 * u[1] * u[1], 0.0, 0.0, 2.5e-3]
    return [surf * math.cos(a), surf * math.sin(a), pp[2] + off[1]], hc


def main():
    out = []
    for kind, p, q, surf, off in CASES:
        k = oracle.P2Z if kind == "p2z" else oracle.P2R
        hit, hc = hit_for(kind, p, q, surf, off)
        c = cov21(p[3])
        p2, c2, chi2, st = oracle.step(k, p, c, q, hit, hc, BZ, surf)
        out.append({"kind": kind, "state": p, "cov": c, "q": q, "hit": hit, "hit_cov": hc,
                    "surf": surf, "bz": BZ, "state_out": [float(v) for v in p2],
                    "cov_out": [float(v) for v in c2], "chi2": chi2, "status": st})
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {len(out)} cases")


if __name__ == "__main__":
    main()
