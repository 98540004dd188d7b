"""Autotuner for the size switch.

The paper sets each routine's switch point between algorithmic variants by
measurement on the target architecture (section 2.4, section 3.1).  This tool
does the same on the GPU it runs on: for every routine, transpose form and
order of the size sweep it times each candidate kernel variant and tiling
with CUDA events on a uniform batch of about 1 GiB of operands, keeps the
fastest, and writes the table to tuned/<gpu name>.json.  The binding loads
that table at import (bf_tune_set), so every later call uses the measured
switch; entries cover the order range from one tuned order up to the next.
On the GPU the batch size takes part in the switch too: for dpotrf the tool
also times the small-batch forms (one problem per CTA, teams of 4 and 2 lanes
per problem) against the table's variant over batches of 152 to 38,912
problems and stores the measured bounds (bf_tune_set_batch_rule).

    python -m paper_1902_08115_gb300.autotune [--quick] [--out PATH]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

ORDERS = (4, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256)
BUDGET = 1 << 30


def table_path(gpu_name: str) -> str:
    safe = "".join(c if c.isalnum() else "_" for c in gpu_name)
    return os.path.join(HERE, "tuned", safe + ".json")


def _time(torch, fn, reps=3):
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def _install(bf, entries):
    """Replace the size-switch table by the given entries."""
    bf.tune_clear()
    for e in entries:
        p = list(e["p"]) + [0] * (4 - len(e["p"]))
        bf.tune_set(e["routine"], e["code"], e["lo"], e["hi"], e["variant"], *p[:4])


def _gemm_candidates(n):
    cands = [(3, 0, 0, 0, 0)] if n <= 4 else []  # tiny: one thread per problem via shared memory
    tiles = [(0, 0)] if n <= 64 else [(0, 0), (32, 32), (48, 48), (64, 64), (n // 2 // 4 * 4, 64)]
    for variant in (0, 1):
        for TM, TN in tiles:
            for threads in (128, 256, 384, 512):
                tm = TM if TM else ((n + 3) // 4 * 4 if n <= 64 else 64)
                tn = TN if TN else ((n + 3) // 4 * 4 if n <= 64 else 64)
                tpp = (tm // 4) * (tn // 4)
                P = max(1, threads // tpp)
                if P * tpp > 512:
                    continue
                for KC in ((0,) if variant == 0 else ((0, 16) if n > 64 else (0,))):
                    c = (variant, TM, TN, KC, P)
                    if c not in cands:
                        cands.append(c)
    return cands


def tune(quick=False, out=None, log=print):
    import torch

    import bfsynth
    import paper_1902_08115_gb300 as bf

    dev = torch.device("cuda")
    name = torch.cuda.get_device_name(dev)
    bf.tune_clear()
    entries = []
    orders = ORDERS[::2] if quick else ORDERS
    t_start = time.time()
    for idx, n in enumerate(orders):
        hi = orders[idx + 1] - 1 if idx + 1 < len(orders) else 1 << 20
        lo = n if idx else 1
        # ---- dgemm, four forms
        b = bfsynth.sweep_batch(n, n, 3)  # the sweep's batch (2 GiB of operands)
        A = bfsynth.randn_batch(b, n, n, n, 1, device=dev)
        B = bfsynth.randn_batch(b, n, n, n, 2, device=dev)
        C = bfsynth.randn_batch(b, n, n, n, 3, device=dev)
        for code, (ta, tb) in enumerate((("N", "N"), ("N", "T"), ("T", "N"), ("T", "T"))):
            best = None
            for cand in _gemm_candidates(n):
                bf.tune_clear()
                bf.tune_set(bf.ROUTINE_DGEMM, code, 0, 1 << 30, *cand)
                ms = _time(torch, lambda: bf.dgemm(ta, tb, 1.0, A, B, 1.0, C, m=n, n=n, k=n))
                if best is None or ms < best[0]:
                    best = (ms, cand)
            gf = b * 2.0 * n ** 3 / (best[0] * 1e-3) / 1e9
            entries.append(dict(routine=bf.ROUTINE_DGEMM, code=code, lo=lo, hi=hi, variant=best[1][0],
                                p=list(best[1][1:]), gflops=round(gf, 1), n=n))
            log(f"dgemm {ta}{tb} n={n}: {best[1]} {gf:.0f} GFLOP/s")
        del A, B, C
        # ---- dtrsm: right-lower-T unit/non-unit, and the left-lower N/T of dpotrs
        b = bfsynth.sweep_batch(n, n, 2)  # wave quantization depends on the batch: tune at 2 GiB
        L = bfsynth.spd_batch(b, n, n, 4, device=dev)
        bf.tune_clear()
        bf.dpotrf(L, n=n)
        X = bfsynth.randn_batch(b, n, n, n, 5, device=dev)
        for code, args in ((11, ("R", "L", "T", "U")), (10, ("R", "L", "T", "N")),
                           (0, ("L", "L", "N", "N")), (2, ("L", "L", "T", "N"))):
            best = None
            for variant in ((0, 1, 3) if n <= 8 else ((0, 1, 2) if n >= 64 else (0, 1))):
                for MR in ((4,) if variant == 3 else (4, 8)):
                    for P, minb in (((0, 1), (0, 2)) if variant in (0, 2) else
                                    (((0, 1),) if variant == 3 else ((0, 1), (8, 1), (16, 1), (32, 1)))):
                        # the blocked form's updates are dgemm calls: time it with the dgemm
                        # entries measured so far installed
                        bf.tune_clear()
                        _install(bf, [e for e in entries if e["routine"] == bf.ROUTINE_DGEMM])
                        bf.tune_set(bf.ROUTINE_DTRSM, code, 0, 1 << 30, variant | bf.TUNE_FORCE, MR, P, minb)
                        cfg = bf.tune_query(bf.ROUTINE_DTRSM, code, n, n, 0, b)
                        if cfg[0] != variant:
                            continue  # not launchable in this form at this order
                        ms = _time(torch, lambda: bf.dtrsm(*args, 1.0, L, X, m=n, n=n))
                        if best is None or ms < best[0]:
                            best = (ms, (variant, MR, P, minb))
            fl = b * n * n * (n - 1 if args[3] == "U" else n)  # unit diagonal: n^2 (n - 1)
            entries.append(dict(routine=bf.ROUTINE_DTRSM, code=code, lo=lo, hi=hi, variant=best[1][0],
                                p=[best[1][1], best[1][2], best[1][3], 0], gflops=round(fl / best[0] / 1e6, 1),
                                n=n))
            log(f"dtrsm {''.join(args)} n={n}: {best[1]} {fl / best[0] / 1e6:.0f} GFLOP/s")
        del L, X
        # ---- dpotrf, per leading-dimension parity (table code lda & 1)
        for code, ld in ((0, n + (n & 1)), (1, n + 1 - (n & 1))):
            b = bfsynth.sweep_batch(n, ld, 1)  # the lane/blocked switch depends on the batch: tune at 2 GiB
            S0 = bfsynth.spd_batch(b, n, ld, 6, device=dev)
            S = S0.clone()
            best = None
            cands = [(0, T, 0, R, 2) for T in (64, 128, 256) for R in (4, 8) if R == 4 or n >= 8]
            cands += [(0, 64, 0, R, 1) for R in (4, 8) if R == 4 or n >= 8]
            if n <= 16:
                cands += [(1, T, 0, 0, 0) for T in (32, 64, 128)]
            if n >= 16:
                cands += [(2, 128, NB, 0, 0) for NB in (8, 16, 32, 64) if NB < n]
            if 16 <= n <= 256:
                cands += [(4, 0, 0, 0, 0)]  # one problem per CTA
            ms_copy = _time(torch, lambda: S.copy_(S0))
            for variant, T, NB, R, U in cands:
                # the blocked form calls dtrsm and dgemm: time it with the entries measured so
                # far installed, as every later call will run it
                _install(bf, entries)
                bf.tune_set(bf.ROUTINE_DPOTRF, code, 0, 1 << 30, variant | bf.TUNE_FORCE, T, NB, R, U)

                def run():
                    S.copy_(S0)
                    bf.dpotrf(S, n=n)

                ms = _time(torch, run) - ms_copy
                if best is None or ms < best[0]:
                    best = (max(ms, 1e-6), (variant, T, NB, R, U))
            fl = b * (n ** 3 / 3 + n ** 2 / 2 + n / 6)
            entries.append(dict(routine=bf.ROUTINE_DPOTRF, code=code, lo=lo, hi=hi, variant=best[1][0],
                                p=list(best[1][1:]), gflops=round(fl / best[0] / 1e6, 1), n=n, lda=ld))
            log(f"dpotrf n={n} lda={ld}: {best[1]} {fl / best[0] / 1e6:.0f} GFLOP/s")
            del S, S0
        torch.cuda.empty_cache()
    bf.tune_clear()
    rules = tune_batch_rules(torch, bf, dev, entries, log, orders=RULE_ORDERS[::2] if quick else RULE_ORDERS)
    bf.tune_clear()
    ragged = tune_ragged(torch, bf, dev, log, count=50000 if quick else 200000)
    doc = {"gpu": name, "ragged": ragged, "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
           "seconds": round(time.time() - t_start, 1), "entries": entries, "batch_rules": rules}
    path = out or table_path(name)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
    bf.load_table(path)
    return path


# ---------------------------------------------------------------------------- batch-size side
RULE_ORDERS = (12, 16, 24, 32, 48, 64, 96, 128, 192, 256)
RULE_BATCHES = tuple(152 * 2 ** k for k in range(9))  # 152 .. 38,912 problems
FORMS = ("cta", "team4", "team2", "table")


def derive_batch_rule(rows):
    """The batch-size schedule of dpotrf's forms from measured times.

    rows: [(batch, {form: ms})] in ascending batch, forms among FORMS ("table" = the size
    table's variant at every batch).  Returns (cta_max, team4_max, team2_max): the schedule
    cta -> team4 -> team2 -> table, bounds taken among the measured batches (0 = never), that
    minimises the summed ratio of the scheduled form's time to the best form's time over the
    measured batches.  Equal sums keep the smaller bounds (the table's variant)."""
    cuts = [0] + [b for b, _ in rows]
    best = None
    for i in range(len(cuts)):
        for j in range(i, len(cuts)):
            for k in range(j, len(cuts)):
                t = (cuts[i], cuts[j], cuts[k])
                cost = 0.0
                for b, ms in rows:
                    form = "cta" if b <= t[0] else "team4" if b <= t[1] else "team2" if b <= t[2] else "table"
                    if form not in ms:
                        cost = float("inf")
                        break
                    cost += ms[form] / min(ms.values())
                if best is None or cost < best[0] - 1e-9:
                    best = (cost, t)
    if best is None or best[0] == float("inf"):
        return 0, 0, 0
    return best[1]


def tune_batch_rules(torch, bf, dev, entries, log, orders=RULE_ORDERS, batches=RULE_BATCHES,
                     budget=2 << 30):
    """Time dpotrf's small-batch forms against the size table's variant over a range of batch
    sizes, per order and lda parity, and derive each order range's bounds (bf_tune_set_batch_rule).
    The tuned entries are installed while timing, as every later call will run them."""
    import bfsynth
    rules = []
    for idx, n in enumerate(orders):
        # from this order up to the next (orders outside the measured range keep the built-in
        # bounds)
        lo, hi = n, (orders[idx + 1] - 1 if idx + 1 < len(orders) else n)
        for code, ld in ((0, n + (n & 1)), (1, n + 1 - (n & 1))):
            table = [e for e in entries if e["routine"] == bf.ROUTINE_DPOTRF and e["code"] == code
                     and e["lo"] <= n <= e["hi"]]
            forms = {"team4": (5, 64, 0, 4, 0), "team2": (5, 64, 0, 2, 0)}
            if 16 <= n <= 256:
                forms["cta"] = (4, 0, 0, 0, 0)
            if table:
                forms["table"] = tuple([table[-1]["variant"]] + list(table[-1]["p"]))
            else:
                forms["table"] = (0, 0, 0, 0, 0)
            rows = []
            for b in batches:
                if b * n * ld * 8 > budget:
                    break
                S0 = bfsynth.spd_batch(b, n, ld, 7, device=dev)
                S = S0.clone()
                ms_copy = _time(torch, lambda: S.copy_(S0))
                times = {}
                for name, (variant, T, NB, R, U) in forms.items():
                    _install(bf, entries)
                    bf.tune_set(bf.ROUTINE_DPOTRF, code, 0, 1 << 30, variant | bf.TUNE_FORCE, T, NB, R, U)

                    def run():
                        S.copy_(S0)
                        bf.dpotrf(S, n=n)

                    times[name] = max(_time(torch, run) - ms_copy, 1e-6)
                rows.append((b, times))
                del S, S0
            cta_max, team4_max, team2_max = derive_batch_rule(rows)
            rules.append(dict(routine=bf.ROUTINE_DPOTRF, code=code, lo=lo, hi=hi, cta_max=cta_max,
                              team4_max=team4_max, team2_max=team2_max, n=n, lda=ld))
            log(f"dpotrf batch rule n={n} lda={ld}: cta <= {cta_max}, team4 <= {team4_max}, "
                f"team2 <= {team2_max}")
    bf.tune_clear()
    return rules


def tune_ragged(torch, bf, dev, log, count=200000, nrhs=4):
    """Threshold between the per-thread and per-CTA ragged forms, and the CTA size."""
    import numpy as np

    import bfsynth
    ns_t = bfsynth.ragged_orders(count, 2, 200, 99)
    S0, offS, B0, offB = bfsynth.ragged_spd(ns_t, nrhs, 100, device=dev)
    S, B = S0.clone(), B0.clone()
    best = None
    for lane_max in (16, 24, 32, 48, 64):
        for threads in (64, 128, 256):
            plan = bf.RaggedPlan(ns_t.numpy(), S, offS.numpy(), B, offB.numpy(), nrhs, lane_max=lane_max,
                                 threads=threads)
            ts = []
            for _ in range(3):
                S.copy_(S0)
                B.copy_(B0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                plan.launch()
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = min(ts)
            log(f"ragged lane_max={lane_max} threads={threads}: {ms:.3f} ms")
            if best is None or ms < best[0]:
                best = (ms, lane_max, threads)
            del plan
    return {"lane_max": best[1], "threads": best[2], "ms": round(best[0], 3), "problems": count}


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--out")
    a = ap.parse_args()
    print(tune(quick=a.quick, out=a.out))
