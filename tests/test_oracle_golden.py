"""The oracle rebuilt on this host reproduces the stored values bit for bit.

tests/golden/oracle_small.json is written by tests/golden/make_golden.py,
which calls only the oracle; the oracle uses correctly rounded operations
and no FMA contraction, so every host must give the same bits.
"""
import json
import os

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def unhex(v, shape):
    return np.array([float.fromhex(x) for x in v]).reshape(shape)


def same_bits(a, b):
    a, b = np.asarray(a).reshape(-1), np.asarray(b).reshape(-1)
    both_nan = np.isnan(a) & np.isnan(b)
    return bool(np.all(both_nan | (a.view(np.int64) == b.view(np.int64))))


def test_oracle_matches_golden(oracle):
    g = json.load(open(os.path.join(HERE, "oracle_small.json")))
    sg, ss = g["inputs"]["shape_gemm"], g["inputs"]["shape_spd"]
    A, B, C = (unhex(g["inputs"][k], sg) for k in "ABC")
    S = unhex(g["inputs"]["S"], ss)
    n = ss[1]
    assert same_bits(oracle.dgemm("N", "T", n, n, n, 1.0, A, B, 1.0, C), unhex(g["dgemm_nt"], sg))
    assert same_bits(oracle.dgemm("T", "N", n, n, n, -0.5, A, B, 2.0, C), unhex(g["dgemm_tn"], sg))
    L, info = oracle.dpotrf_l(S)
    assert same_bits(L, unhex(g["dpotrf_l"], ss))
    assert info.tolist() == g["dpotrf_info"]
    X = oracle.dtrsm("R", "L", "T", "N", n, n, 1.0, L, A[:, :, :n].copy())
    assert same_bits(X, unhex(g["dtrsm_rltn"], ss))


def test_flop_table_is_the_papers():
    rows = [l.split() for l in open(os.path.join(HERE, "flops_appendix_d.txt"))
            if l.strip() and not l.startswith("#")]
    table = dict(rows)
    assert table["dgemm_nt"] == "2*n^3" and table["dpotrf_l"] == "1/3*n^3"
