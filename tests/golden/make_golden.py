"""Writes tests/golden/oracle_small.json from the CPU oracle only.

The file pins the oracle build across hosts: the oracle is compiled without
FMA contraction and uses only correctly rounded operations (+, -, *, /, sqrt),
so an x86 and an Arm build must reproduce these values bit for bit.
Inputs come from the seeded generators in bfsynth.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import bfsynth  # noqa: E402
import oracle  # noqa: E402


def hexlist(a):
    return [float(v).hex() for v in a.reshape(-1)]


def main():
    n, batch = 5, 3
    A = bfsynth.randn_batch(batch, n, n, n + 1, seed=11, pad=0.0).numpy()
    B = bfsynth.randn_batch(batch, n, n, n + 1, seed=12, pad=0.0).numpy()
    C = bfsynth.randn_batch(batch, n, n, n + 1, seed=13, pad=0.0).numpy()
    S = bfsynth.spd_batch(batch, n, n, seed=14).numpy()
    out = {
        "inputs": {"A": hexlist(A), "B": hexlist(B), "C": hexlist(C), "S": hexlist(S),
                   "shape_gemm": [batch, n, n + 1], "shape_spd": [batch, n, n]},
        "dgemm_nt": hexlist(oracle.dgemm("N", "T", n, n, n, 1.0, A, B, 1.0, C)),
        "dgemm_tn": hexlist(oracle.dgemm("T", "N", n, n, n, -0.5, A, B, 2.0, C)),
    }
    L, info = oracle.dpotrf_l(S)
    out["dpotrf_l"] = hexlist(L)
    out["dpotrf_info"] = info.tolist()
    out["dtrsm_rltn"] = hexlist(oracle.dtrsm("R", "L", "T", "N", n, n, 1.0, L, A[:, :, :n].copy()))
    with open(os.path.join(HERE, "oracle_small.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
