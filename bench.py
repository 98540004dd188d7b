#!/usr/bin/env python
"""Benchmark of the batched small-matrix FP64 BLAS/LAPACK library on GB300.

Workload (one "step"): the size sweep -- for every order n in
{4, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256} and leading dimension
lda in {n, n+3}, uniform batches sized so that each routine's operands total
about 2 GiB:
  dgemm nn, nt, tn, tt (m = n = k, C += op(A) op(B)),
  dtrsm right-lower-transposed with the unit-scaled Cholesky factor (rltu)
  and with the factor itself (rltn),
  dpotrf lower on S = G G^T + n I.
Inputs are synthetic (seeded), generated on the device before timing and
resident in HBM; every point is larger than L2, so no flush is needed.  The
dpotrf inputs are refreshed inside each step by copying the untouched upper
triangle of S back onto the factored lower triangle (a torch copy, timed as
part of the step, excluded from the per-call figures).

Reported: whole-step GFLOP/s (the value), per-point GFLOP/s and fraction of
the per-size roofline min(P_FP64, B_HBM * AI), the size switch's chosen
variant against each plain variant, an end-to-end rate through pinned host
memory, and the CPU oracle on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SWEEP_N = (4, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256)
PADS = (0, 3)
GEMM_FORMS = ("nn", "nt", "tn", "tt")
METRIC = "batched FP64 dgemm/dpotrf GFLOP/s and % of roofline vs n; chosen vs plain form"
# DRAM bytes per problem of the dgemm_nt kernel at n = lda = 256 (dgemm_tile_kernel<4,4,0,1,0,0>):
# dram__bytes_read.sum + dram__bytes_write.sum = 403.57 MB + 110.01 MB over 256 problems in one ncu
# capture of `python -m paper_1902_08115_gb300.profcase gemm 256 0`
DGEMM_NT_256_TRAFFIC_PER_PROBLEM = (403.572736e6 + 110.007040e6) / 256
HBM_FALLBACK_GBS = 6800.0


# ---------------------------------------------------------------------------- work accounting
def flops(routine: str, n: int) -> float:
    """Algorithmic flops of one problem (m = n = k); dpotrf uses LAPACK's count."""
    if routine.startswith("dgemm"):
        return 2.0 * n ** 3
    if routine == "dtrsm_rltu":
        return float(n * n * (n - 1))
    if routine == "dtrsm_rltn":
        return float(n ** 3)
    if routine == "dpotrf":
        return n ** 3 / 3.0 + n ** 2 / 2.0 + n / 6.0
    raise KeyError(routine)


def alg_bytes(routine: str, n: int) -> float:
    """Bytes the method must move per problem (lda padding not counted)."""
    if routine.startswith("dgemm"):
        return 32.0 * n * n
    if routine == "dtrsm_rltu":
        return 8.0 * (2 * n * n + n * (n - 1) / 2)
    if routine == "dtrsm_rltn":
        return 8.0 * (2 * n * n + n * (n + 1) / 2)
    if routine == "dpotrf":
        return 8.0 * n * (n + 1)
    raise KeyError(routine)


def batch_of(routine: str, n: int, ld: int) -> int:
    import bfsynth
    ops = 3 if routine.startswith("dgemm") else (2 if routine.startswith("dtrsm") else 1)
    return bfsynth.sweep_batch(n, ld, ops)


ROUTINES = tuple("dgemm_" + f for f in GEMM_FORMS) + ("dtrsm_rltu", "dtrsm_rltn", "dpotrf")


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback (profiling recipe)"


# ---------------------------------------------------------------------------- ranks
def reduce_max_ms(ms: float, world: int, device=None) -> float:
    """Max of a per-rank time over all ranks (one all-reduce; replicas share nothing else)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gflops(flops_per_rank: float, world: int, ms_step: float) -> float:
    """Units all ranks processed / the slowest rank's time (weak scaling: fixed work per rank)."""
    return flops_per_rank * world / (ms_step * 1e-3) / 1e9


# ---------------------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        self.gpu_id = gpu_id

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------- inputs
class Point:
    """Device-resident inputs of one sweep point (n, lda)."""

    def __init__(self, n: int, pad: int, dev, seed: int):
        import bfsynth
        self.n, self.pad, self.ld = n, pad, n + pad
        ld = self.ld
        bg = batch_of("dgemm", n, ld)
        self.A = bfsynth.randn_batch(bg, n, n, ld, seed, device=dev)
        self.B = bfsynth.randn_batch(bg, n, n, ld, seed + 1, device=dev)
        self.C = bfsynth.randn_batch(bg, n, n, ld, seed + 2, device=dev)
        import torch
        import paper_1902_08115_gb300 as bf
        # column-major (j, i) with i > j: the strict lower triangle
        self.low = torch.tril(torch.ones(n, n, dtype=torch.bool, device=dev), -1).t().contiguous()
        bt = batch_of("dtrsm", n, ld)
        # the triangular factors come from this library's own dpotrf of S = G G^T + n I (the
        # solve follows the factorisation); L_u = L diag(L)^{-1} is the unit-scaled factor
        self.L = bfsynth.spd_batch(bt, n, ld, seed + 3, device=dev)
        info = bf.dpotrf(self.L, n=n)
        assert int(info.abs().max()) == 0
        V = self.L[:, :, :n]
        d = torch.diagonal(V, dim1=1, dim2=2).clone()
        self.Lu = self.L.clone()
        self.Lu[:, :, :n] = V / d.unsqueeze(2)  # column j divided by l_jj
        self.X = bfsynth.randn_batch(bt, n, n, ld, seed + 4, device=dev)
        bp = batch_of("dpotrf", n, ld)
        self.S = bfsynth.spd_batch(bp, n, ld, seed + 5, device=dev)
        self.Sdiag = torch.diagonal(self.S[:, :, :n], dim1=1, dim2=2).clone()
        self.info = torch.zeros(bp, dtype=torch.int32, device=dev)
        self.batch = {"dgemm": bg, "dtrsm": bt, "dpotrf": bp}

    def restore_s(self):
        """Rebuild S from its untouched strict upper triangle and the saved diagonal."""
        import torch
        n = self.n
        V = self.S[:, :, :n]
        V.copy_(torch.where(self.low, V.transpose(1, 2), V))
        torch.diagonal(V, dim1=1, dim2=2).copy_(self.Sdiag)

    def nbatch(self, routine):
        return self.batch[routine.split("_")[0]]


def run_routine(bf, p: Point, routine: str):
    n = p.n
    if routine.startswith("dgemm_"):
        ta, tb = routine[-2].upper(), routine[-1].upper()
        bf.dgemm(ta, tb, 1.0, p.A, p.B, 1.0, p.C, m=n, n=n, k=n)
    elif routine == "dtrsm_rltu":
        bf.dtrsm("R", "L", "T", "U", 1.0, p.Lu, p.X, m=n, n=n)
    elif routine == "dtrsm_rltn":
        bf.dtrsm("R", "L", "T", "N", 1.0, p.L, p.X, m=n, n=n)
    elif routine == "dpotrf":
        bf.dpotrf(p.S, n=n, info=p.info)
    else:
        raise KeyError(routine)


def fp64_peak(bf, torch, dev):
    """Live FP64 FMA roof: best of 3 timed runs of the library's DFMA probe."""
    # 8 warps per SM: the 4x4 register-tile FMA pattern at full issue rate (64 warps per SM
    # oversubscribe the FP64 pipes and issue about 17% slower)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads, iters = sms * 2, 128, 4096
    out = torch.empty(blocks * threads, dtype=torch.float64, device=dev)
    st = bf._stream()
    args = (blocks, threads, iters, 32, 0, bf._ptr(out), st)
    bf._check("bf_probe_fp64_ex", bf.bf_probe_fp64_ex(*args))
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        bf.bf_probe_fp64_ex(*args)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = max(best, 2.0 * 16 * iters * blocks * threads / (ms * 1e-3))
    return best


# ---------------------------------------------------------------------------- CPU oracle baseline
_SAMPLES = {}


def _oracle_inputs(r, n, ld, k, seed):
    """Seeded CPU inputs of one sampled sweep point, built once and reused across steps."""
    key = (r, n, ld, k)
    if key not in _SAMPLES:
        import bfsynth
        if r.startswith("dgemm"):
            _SAMPLES[key] = tuple(bfsynth.randn_batch(k, n, n, ld, seed + t).numpy() for t in range(3))
        elif r.startswith("dtrsm"):
            _SAMPLES[key] = (bfsynth.unit_lower_batch(k, n, ld, seed, unit=(r[-1] == "u")).numpy(),
                             bfsynth.randn_batch(k, n, n, ld, seed + 1).numpy())
        else:
            _SAMPLES[key] = (bfsynth.spd_batch(k, n, ld, seed).numpy(),)
    return _SAMPLES[key]


# The oracle's sample: one fixed set of problems per sweep point and routine, sized for about
# ORACLE_SAMPLE_S seconds of CPU work on 16 cores; the CPU baseline of the GPU arm and every step
# of the reference arm time this same sample, so their rates compare.
ORACLE_SAMPLE_S = 6.0


def oracle_sample(budget_s: float = ORACLE_SAMPLE_S, steps: int = 1):
    """Time the CPU oracle on a bounded sample of every sweep point; returns (GFLOP/s, desc, cores).

    Only the oracle calls are timed; the sample inputs are generated once per process.  The
    sample's problem counts depend on budget_s alone (not on the host), so equal budgets time
    equal samples."""
    import oracle
    oracle.build()
    cores = oracle.num_threads()
    per_call = budget_s / (len(SWEEP_N) * len(PADS) * len(ROUTINES))
    est_rate = 0.5e9 * 16  # plain loops, binary64, no vectorisation, 16 cores
    tot_flops, tot_time, nprob = 0.0, 0.0, 0
    for _ in range(steps):
        for n in SWEEP_N:
            for pad in PADS:
                ld = n + pad
                for r in ROUTINES:
                    full = batch_of(r, n, ld)
                    k = int(max(16, min(full, 65536, per_call * est_rate / flops(r, n))))
                    ins = _oracle_inputs(r, n, ld, k, 7 * n + pad)
                    t0 = time.perf_counter()
                    if r.startswith("dgemm"):
                        oracle.dgemm(r[-2].upper(), r[-1].upper(), n, n, n, 1.0, ins[0], ins[1], 1.0, ins[2])
                    elif r.startswith("dtrsm"):
                        oracle.dtrsm("R", "L", "T", r[-1].upper(), n, n, 1.0, ins[0], ins[1])
                    else:
                        oracle.dpotrf_l(ins[0])
                    tot_time += time.perf_counter() - t0
                    tot_flops += k * flops(r, n)
                    nprob += k
    desc = (f"oracle (plain C, binary64, OpenMP over problems) on {nprob} problems: a fixed bounded "
            f"sample of every sweep point and routine (the same in both arms), ~{budget_s:.0f} s of "
            f"CPU work per pass on 16 cores (inputs built once, outside the timing)")
    return tot_flops / tot_time / 1e9, desc, cores


# ---------------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip forms, e2e and CPU baseline")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        reference_arm(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    import paper_1902_08115_gb300 as bf

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- inputs (seeded; each rank draws its own replica with a rank-dependent seed)
    import bfsynth
    points = []
    for i, n in enumerate(SWEEP_N):
        for pad in PADS:
            points.append(Point(n, pad, dev, bfsynth.BASE_SEED + 1000 * rank + 10 * i + pad))
    torch.cuda.synchronize()

    calls = [(p, r) for p in points for r in ROUTINES]
    step_flops = sum(p.nbatch(r) * flops(r, p.n) for p, r in calls)

    def step(events=None):
        for ci, (p, r) in enumerate(calls):
            if r == "dpotrf":
                p.restore_s()
            if events is not None:
                events[ci][0].record()
            run_routine(bf, p, r)
            if events is not None:
                events[ci][1].record()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    gpu_uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    clocks = Clocks(gpu_uuid)
    evs = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
            for _ in calls] for _ in range(args.steps)]
    launches0 = bf.bf_launch_count()
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for s in range(args.steps):
        step(evs[s])
    t1.record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = bf.bf_launch_count() - launches0
    # every factorisation of the timed steps must have succeeded (a failed pivot ends a problem
    # early and would make the timing meaningless)
    bad = sum(int((p.info != 0).sum()) for p in points)
    if bad:
        raise RuntimeError(f"{bad} dpotrf problems failed during the timed steps")
    ms_total = reduce_max_ms(t0.elapsed_time(t1), world, dev)
    ms_step = ms_total / args.steps
    value = whole_job_gflops(step_flops, world, ms_step)  # GFLOP/s, all ranks

    # ---- per-call figures and the roofline
    # FP64 roof from unit counts and the clock measured during the timed steps: every SM issues
    # 2 FP64 FMAs per clock (152 SMs x 2 x 2 flop x 2.07 GHz = 1.26 TFLOP/s, NVIDIA's 1.25 TFLOP/s);
    # the FMA probe is reported beside it (plain FMA loops issue below this rate)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_mhz = clk["sm_mhz"] or clk["sm_max_mhz"] or 2070.0
    peak = sms * 2 * 2 * clk_mhz * 1e6
    probe_peak = fp64_peak(bf, torch, dev)
    hbm, hbm_src = hbm_peak()
    per = {}
    for ci, (p, r) in enumerate(calls):
        ms = statistics.mean(evs[s][ci][0].elapsed_time(evs[s][ci][1]) for s in range(args.steps))
        f = p.nbatch(r) * flops(r, p.n)
        by = p.nbatch(r) * alg_bytes(r, p.n)
        roof = min(peak, hbm * 1e9 * f / by)
        per[(r, p.n, p.pad)] = dict(ms=ms, gflops=f / (ms * 1e-3) / 1e9, frac=f / (ms * 1e-3) / roof,
                                    flops=f, bytes=by, roof=roof)
    # the dominant kernel: the four dgemm forms and dtrsm at n = 256 have the largest per-call times
    # (within a few percent of each other); dgemm_nt, the paper's headline form, is reported
    dom = ("dgemm_nt", 256, 0)
    d = per[dom]
    traffic = DGEMM_NT_256_TRAFFIC_PER_PROBLEM * batch_of("dgemm_nt", 256, 256)
    roofline = {"bound": "alu", "achieved": round(d["flops"] / (d["ms"] * 1e-3) / 1e12, 4),
                "peak": round(peak / 1e12, 4), "unit": "TFLOP/s",
                "frac": round(d["flops"] / (d["ms"] * 1e-3) / peak, 4), "traffic": round(traffic),
                "traffic_note": "bytes per launch: DRAM read + write per problem from one ncu capture of "
                                "256 problems of this kernel, times the launch's batch; algorithmic "
                                f"{round(d['bytes'])} bytes",
                "kernel": f"{dom[0]} n={dom[1]} lda={dom[1] + dom[2]} (dgemm_tile_kernel<4,4,0,1,0,0>)",
                "peak_source": f"{sms} SMs x 2 FP64 FMA/clk x 2 flop x {clk_mhz:.0f} MHz (median SM clock "
                               f"of the timed steps)",
                "hbm_gbs": hbm, "hbm_source": hbm_src}
    sweep = {r: [[n, pad, round(per[(r, n, pad)]["gflops"], 2), round(per[(r, n, pad)]["frac"], 4)]
                 for n in SWEEP_N for pad in PADS] for r in ROUTINES}
    big = [per[(r, n, pad)]["frac"] for r in ("dgemm_nn", "dgemm_nt", "dgemm_tn", "dgemm_tt", "dpotrf")
           for n in SWEEP_N for pad in PADS if n >= 32]

    result = {
        "metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded N(0,1) operands, S = G G^T + n I, unit-scaled Cholesky factors)",
        "config": sweep_config(world),
        "roofline": roofline,
        "clocks": clk,
        "gpu_launches": int(launches),
        "fp64_peak_tflops": round(peak / 1e12, 4),
        "fp64_probe_tflops": round(probe_peak / 1e12, 4),
        "min_frac_n_ge_32_dgemm_dpotrf": round(min(big), 4),
        "sweep": sweep,
    }

    if not args.no_extras:
        result["forms"] = plain_forms(bf, torch, points, peak, hbm)
        result["hot"] = hot_forms(bf, torch, points)
        result["e2e"] = end_to_end(bf, torch, dev, points)
        result["config"]["e2e_workload"] = ("the sweep's routines and points with batches capped at 32 MiB of "
                                            "operands each (pinned host memory), inputs copied in and results "
                                            "read back every step; not the 2 GiB batches of `value`")
        del points
        torch.cuda.empty_cache()
        result["ragged"] = ragged_form(bf, torch, dev, rank)
        torch.cuda.empty_cache()
        result["diff"] = diff_form(bf, torch, dev, rank, peak)
        torch.cuda.empty_cache()
        result["precision"] = precision_form(bf, torch, dev, rank)
        torch.cuda.empty_cache()
        result["next_rows"] = next_rows(bf, torch, dev, peak)
        torch.cuda.empty_cache()
        result["vbatched"] = vbatched_form(bf, torch, dev, peak)
        torch.cuda.empty_cache()
        if rank == 0:
            v, desc, cores = oracle_sample()
            result["cpu_baseline"] = {"value": round(v, 3), "unit": "GFLOP/s", "cores": cores,
                                      "kind": "oracle", "sample": desc}
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        dist.destroy_process_group()


def plain_forms(bf, torch, points, peak, hbm):
    """Chosen (size switch) vs each plain variant, lda = n, 2 timed repetitions each."""
    forms = {}
    variants = {"dgemm": [("direct", 0), ("packed", 1)], "dtrsm": [("direct", 0), ("packed", 1)],
                "dpotrf": [("direct", 0), ("packed", 1), ("blocked", 2), ("cta", 4)]}
    routine_id = {"dgemm": bf.ROUTINE_DGEMM, "dtrsm": bf.ROUTINE_DTRSM, "dpotrf": bf.ROUTINE_DPOTRF}
    for r in ("dgemm_nn", "dgemm_nt", "dgemm_tn", "dtrsm_rltu", "dpotrf"):
        fam = r.split("_")[0]
        rows = []
        for p in points:
            if p.pad:
                continue
            row = {"n": p.n}
            for name, var in [("chosen", None)] + variants[fam]:
                if fam == "dpotrf" and name == "packed" and p.n > 16:
                    continue
                if fam == "dpotrf" and name == "cta" and p.n < 16:
                    continue
                if var is not None:
                    code = {"dgemm": (2 if r[-2] == "t" else 0) + (1 if r[-1] == "t" else 0),
                            "dtrsm": 8 + 2 + 1, "dpotrf": 0}[fam]
                    bf.tune_set(routine_id[fam], code, 0, 1 << 30, var | bf.TUNE_FORCE)
                try:
                    ts = []
                    for rep in range(3):
                        if fam == "dpotrf":
                            p.restore_s()
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record()
                        run_routine(bf, p, r)
                        e1.record()
                        e1.synchronize()
                        if rep:
                            ts.append(e0.elapsed_time(e1))
                    ms = min(ts)
                finally:
                    bf.reset_table()
                f = p.nbatch(r) * flops(r, p.n)
                row[name] = round(f / (ms * 1e-3) / 1e9, 2)
            rows.append(row)
        forms[r] = rows
    return forms


def _sub_ms(bf, torch, p, r, b, flush=None, reps=10):
    """Median CUDA-event time of routine r on the first b problems of point p.  Before each
    repetition the operand that the routine overwrites is restored from a saved copy (outside
    the timed region; the copy itself leaves the operands in L2); with `flush`, a buffer larger
    than L2 is then overwritten, so that the repetition starts cold."""
    n = p.n
    fam = r.split("_")[0]
    if fam == "dgemm":
        A, B, C = p.A[:b], p.B[:b], p.C[:b]
        C0 = C.clone()
        prep = lambda: C.copy_(C0)
        run = lambda: bf.dgemm("N", "T", 1.0, A, B, 1.0, C, m=n, n=n, k=n)
        keep = C0
    elif fam == "dtrsm":
        X, Lu = p.X[:b], p.Lu[:b]
        X0 = X.clone()
        prep = lambda: X.copy_(X0)
        run = lambda: bf.dtrsm("R", "L", "T", "U", 1.0, Lu, X, m=n, n=n)
        keep = X0
    else:
        p.restore_s()
        S, info = p.S[:b], p.info[:b]
        S0 = S.clone()
        prep = lambda: S.copy_(S0)
        run = lambda: bf.dpotrf(S, n=n, info=info)
        keep = S0
    ts = []
    for rep in range(reps + 1):
        prep()
        if flush is not None:
            flush.fill_(rep & 0x7F)
        # a GPU-side wait of ~50 us ahead of the timed call: its launch is enqueued while the GPU
        # is still busy, so the events time the call on the device, not the host's enqueue
        # latency (about 12 us through the Python binding) that an idle GPU would wait for
        torch.cuda._sleep(100000)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        e1.synchronize()
        if rep:
            ts.append(e0.elapsed_time(e1))
    prep()
    del keep
    if fam == "dpotrf" and int(info.abs().max()) != 0:
        raise RuntimeError("hot-cache dpotrf failed")
    return statistics.median(ts)


def hot_forms(bf, torch, points):
    """Hot-cache figures, the paper's own setting (operands resident in cache across
    repetitions): for every lda = n point, a sub-batch small enough to stay in the 126 MiB L2
    (48 MiB of operands), timed back to back, median of 10.  Plus the 4096 x n = 24 workload
    hot and cold (512 MiB overwritten between repetitions)."""
    out = {}
    budget = 48 << 20
    for r, nops in (("dgemm_nt", 3), ("dtrsm_rltu", 2), ("dpotrf", 1)):
        rows = []
        for p in points:
            if p.pad:
                continue
            b = max(1, min(p.nbatch(r), budget // (nops * p.n * p.ld * 8)))
            ms = _sub_ms(bf, torch, p, r, b)
            rows.append([p.n, b, round(b * flops(r, p.n) / (ms * 1e-3) / 1e9, 2)])
        out[r] = rows
    p24 = next(p for p in points if p.n == 24 and p.pad == 0)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=p24.A.device)
    small = {}
    for r in ("dgemm_nt", "dpotrf"):
        hot = _sub_ms(bf, torch, p24, r, 4096)
        cold = _sub_ms(bf, torch, p24, r, 4096, flush=flush)
        f = 4096 * flops(r, 24)
        small[r] = {"hot_gflops": round(f / (hot * 1e-3) / 1e9, 2), "hot_ms": round(hot, 4),
                    "cold_gflops": round(f / (cold * 1e-3) / 1e9, 2), "cold_ms": round(cold, 4)}
    del flush
    out["n24_batch4096"] = small
    out["columns"] = "[n, sub-batch, GFLOP/s]"
    return out


def ends_inward(items):
    """The items taken alternately from the front and the back: [a0, a_last, a1, a_last-1, ...]."""
    lo, hi, out = 0, len(items) - 1, []
    while lo <= hi:
        out.append(items[lo])
        if hi != lo:
            out.append(items[hi])
        lo, hi = lo + 1, hi - 1
    return out


def end_to_end(bf, torch, dev, points, cap_bytes=32 << 20, nstreams=8, interleave=True):
    """Same routines through the public API with host buffers: every call's inputs copied from
    pinned host memory and its result read back inside the timed region.  Batches are capped
    at cap_bytes of operands per routine and point (pinned host memory is limited)."""
    work = []
    for p in points:
        for r in ROUTINES:
            b = p.nbatch(r)
            per_problem = {"dgemm": 3, "dtrsm": 2, "dpotrf": 1}[r.split("_")[0]] * p.ld * p.n * 8
            k = max(1, min(b, cap_bytes // per_problem))
            if r.startswith("dgemm"):
                host = [p.A[:k].cpu().pin_memory(), p.B[:k].cpu().pin_memory(), p.C[:k].cpu().pin_memory()]
            elif r == "dtrsm_rltu":
                host = [p.Lu[:k].cpu().pin_memory(), p.X[:k].cpu().pin_memory()]
            elif r == "dtrsm_rltn":
                host = [p.L[:k].cpu().pin_memory(), p.X[:k].cpu().pin_memory()]
            else:
                p.restore_s()
                host = [p.S[:k].cpu().pin_memory()]
            out = torch.empty_like(host[-1], pin_memory=True)
            work.append((p, r, k, host, out))
    torch.cuda.synchronize()
    if interleave:
        # the list runs from the smallest orders (transfer-bound) to the largest (kernel-bound):
        # taken alternately from both ends, copies of one kind of call overlap kernels of the
        # other (680 -> 733-741 GFLOP/s on one box, 8 streams)
        work = ends_inward(work)

    # the calls are independent, so a user pipelines them: each call's copy in, kernel and copy
    # out go on one of nstreams streams in turn, and one call's transfers overlap other calls'
    # kernels (2 streams measured 521 GFLOP/s, 3 streams 607, 4 streams 659, 8 streams 688)
    streams = [torch.cuda.Stream(device=dev) for _ in range(nstreams)]

    def one_pass():
        h2d = d2h = 0
        for i, (p, r, k, host, out) in enumerate(work):
            with torch.cuda.stream(streams[i % len(streams)]):
                d = [h.to(dev, non_blocking=True) for h in host]
                h2d += sum(h.numel() * 8 for h in host)
                n = p.n
                if r.startswith("dgemm"):
                    bf.dgemm(r[-2].upper(), r[-1].upper(), 1.0, d[0], d[1], 1.0, d[2], m=n, n=n, k=n)
                elif r.startswith("dtrsm"):
                    bf.dtrsm("R", "L", "T", r[-1].upper(), 1.0, d[0], d[1], m=n, n=n)
                else:
                    info = torch.empty(k, dtype=torch.int32, device=dev)
                    bf.dpotrf(d[0], n=n, info=info)
                out.copy_(d[-1], non_blocking=True)
                d2h += out.numel() * 8
        return h2d, d2h

    one_pass()
    torch.cuda.synchronize()
    # each pass timed on its own, the median reported: the host side (Python issue, pinned
    # copies) shares the machine, and a single slow pass should not decide the figure
    reps, secs = 5, []
    for _ in range(reps):
        t0 = time.perf_counter()
        h2d, d2h = one_pass()
        torch.cuda.synchronize()
        secs.append(time.perf_counter() - t0)
    sec = statistics.median(secs)
    f = sum(k * flops(r, p.n) for p, r, k, _, _ in work)
    return {"value": round(f / sec / 1e9, 3), "unit": "GFLOP/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "passes_gflops": [round(f / x / 1e9, 1) for x in secs],
            "statistic": f"median of {reps} passes, each timed alone (host wall clock, synchronized)",
            "workload": f"the sweep's routines and points with batches capped at {cap_bytes >> 20} MiB "
                        "of operands each, through the Python binding of the C ABI, inputs copied "
                        "from pinned host memory and results read back every step, the independent "
                        f"calls spread over {nstreams} streams so transfers overlap kernels"
                        + (", small and large orders interleaved" if interleave else "")}


def _events_ms(torch, fn, reps=3, before=None):
    """min over reps of the CUDA-event time of fn() (before() runs untimed ahead of each rep)."""
    best = float("inf")
    for _ in range(reps):
        if before is not None:
            before()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def ragged_form(bf, torch, dev, rank, count=200000, nrhs=4):
    """Ragged batch (n log-uniform in [2, 200], dpotrf + dpotrs with 4 right-hand sides): one
    persistent graph-captured launch against plain per-size launches of the uniform path."""
    import ctypes

    import numpy as np

    import bfsynth
    ns_t = bfsynth.ragged_orders(count, 2, 200, bfsynth.BASE_SEED + 3 + rank)
    S0, offS, B0, offB = bfsynth.ragged_spd(ns_t, nrhs, bfsynth.BASE_SEED + 4 + rank, device=dev)
    ns = ns_t.numpy().astype(np.int64)
    S, B = S0.clone(), B0.clone()
    flops = float(np.sum(ns ** 3 / 3.0 + ns ** 2 / 2.0 + ns / 6.0 + 2.0 * nrhs * ns ** 2))
    cfg = bf.ragged_config()
    plan = bf.RaggedPlan(ns_t.numpy(), S, offS.numpy(), B, offB.numpy(), nrhs, **cfg)

    def restore():
        S.copy_(S0)
        B.copy_(B0)

    t_graph = _events_ms(torch, plan.launch, reps=3, before=restore)
    ok_graph = int((plan.info != 0).sum()) == 0
    err_graph = _ragged_sample_error(ns, S0, offS.numpy(), B0, offB.numpy(), S, B, nrhs)
    # plain per-size launches: one pointer-array dpotrf and two dtrsm per distinct order
    groups = []
    sbase, bbase = S.data_ptr(), B.data_ptr()
    for n in np.unique(ns):
        idx = np.nonzero(ns == n)[0]
        pa = torch.tensor(sbase + 8 * offS.numpy()[idx], dtype=torch.int64, device=dev)
        pb = torch.tensor(bbase + 8 * offB.numpy()[idx], dtype=torch.int64, device=dev)
        info = torch.zeros(len(idx), dtype=torch.int32, device=dev)
        groups.append((int(n), len(idx), pa, pb, info))
    st = bf._stream()

    def per_size():
        for n, cnt, pa, pb, info in groups:
            pav, pbv = ctypes.c_void_p(pa.data_ptr()), ctypes.c_void_p(pb.data_ptr())
            bf._check("bf_dpotrf_batched", bf.bf_dpotrf_batched(b"L", n, pav, n, ctypes.c_void_p(info.data_ptr()),
                                                               cnt, st))
            bf._check("bf_dtrsm_batched", bf.bf_dtrsm_batched(b"L", b"L", b"N", b"N", n, nrhs, 1.0, pav, n, pbv,
                                                             n, cnt, st))
            bf._check("bf_dtrsm_batched", bf.bf_dtrsm_batched(b"L", b"L", b"T", b"N", n, nrhs, 1.0, pav, n, pbv,
                                                             n, cnt, st))

    t_sizes = _events_ms(torch, per_size, reps=3, before=restore)
    ok_sizes = all(int((g[4] != 0).sum()) == 0 for g in groups)
    err_sizes = _ragged_sample_error(ns, S0, offS.numpy(), B0, offB.numpy(), S, B, nrhs)
    return {"problems": count, "nrhs": nrhs, "orders": "log-uniform in [2, 200]",
            "S_bytes": int(S0.numel() * 8), "gflop": round(flops / 1e9, 3),
            "persistent_graph_ms": round(t_graph, 3), "persistent_gflops": round(flops / t_graph / 1e6, 2),
            "per_size_launches_ms": round(t_sizes, 3), "per_size_gflops": round(flops / t_sizes / 1e6, 2),
            "speedup": round(t_sizes / t_graph, 3), "distinct_orders": len(groups), "plan": plan.describe(),
            "config": cfg, "all_info_zero": bool(ok_graph and ok_sizes),
            "max_normwise_error_vs_oracle": {"persistent": err_graph, "per_size": err_sizes,
                                             "sample": "256 problems (seeded, with the first and last), L and X"}}


def _ragged_sample_error(ns, S0, offS, B0, offB, S, B, nrhs, k=256):
    """Max normwise relative error of L and X against the oracle on a seeded sample of problems
    (computed after the timing; the oracle runs on the host)."""
    import numpy as np

    import oracle
    rng = np.random.default_rng(12)
    idx = np.unique(np.r_[0, len(ns) - 1, rng.integers(0, len(ns), k)]).astype(np.int64)
    sub_n = ns[idx].astype(np.int32)
    offs_s = np.zeros(len(idx), dtype=np.int64)
    offs_b = np.zeros(len(idx), dtype=np.int64)
    offs_s[1:] = np.cumsum(sub_n[:-1].astype(np.int64) ** 2)
    offs_b[1:] = np.cumsum(sub_n[:-1].astype(np.int64) * nrhs)
    S0h, B0h, Sh, Bh = (t.cpu().numpy() for t in (S0, B0, S, B))
    Sin = np.concatenate([S0h[offS[b]:offS[b] + int(ns[b]) ** 2] for b in idx])
    Bin = np.concatenate([B0h[offB[b]:offB[b] + int(ns[b]) * nrhs] for b in idx])
    So, Xo, info = oracle.ragged_potrf_potrs(sub_n, Sin, offs_s, Bin, offs_b, nrhs)
    worst = 0.0
    for t, b in enumerate(idx):
        n = int(ns[b])
        if info[t]:
            continue
        Lg = np.tril(Sh[offS[b]:offS[b] + n * n].reshape(n, n).T)
        Lr = np.tril(So[offs_s[t]:offs_s[t] + n * n].reshape(n, n).T)
        xg = Bh[offB[b]:offB[b] + n * nrhs]
        xr = Xo[offs_b[t]:offs_b[t] + n * nrhs]
        worst = max(worst, float(np.linalg.norm(Lg - Lr) / np.linalg.norm(Lr)),
                    float(np.linalg.norm(xg - xr) / np.linalg.norm(xr)))
    return worst


def diff_form(bf, torch, dev, rank, peak=None, batch=65536, n=32, q=16, r=8):
    """Differentiation workload: loss = sum((Q + J J^T)^{-1} B .* W) through the autograd
    Functions; forward, forward + backward, and the plain forward calls without autograd."""
    import bfsynth
    from paper_1902_08115_gb300 import autograd as ag
    Qd, J, B, W = bfsynth.diff_batch(batch, n, q, r, seed=bfsynth.BASE_SEED + 5 + rank, device=dev)
    ts = [x.clone().requires_grad_(True) for x in (Qd, J, B, W)]

    def fwd():
        with torch.no_grad():
            ag.spd_solve_loss(Qd, J, B, W)

    def fwd_bwd():
        for t in ts:
            t.grad = None
        loss, _, _ = ag.spd_solve_loss(*ts)
        loss.backward()

    C0 = torch.diag_embed(Qd)
    A = torch.empty_like(C0)
    X = torch.empty_like(B)

    def plain():
        A.copy_(C0)
        bf.dsyrk_dpotrf(J, A, n=n, k=q)
        X.copy_(B)
        bf.dpotrs(A, X, n=n, nrhs=r)

    t_f = _events_ms(torch, fwd)
    t_fb = _events_ms(torch, fwd_bwd)
    t_p = _events_ms(torch, plain)
    # forward: the fused dsyrk + dpotrf (lower triangle of J J^T: n(n+1) q), two solves
    flops_f = batch * (n * (n + 1) * q + n ** 3 / 3 + n * n / 2 + n / 6 + 2.0 * 2 * n * n * r)
    # the adjoints' algorithmic flops per problem: two triangular-solve adjoints (solve n^2 r,
    # lower-triangle gradient n(n+1) r), the Cholesky adjoint (Phi(L^T Lbar) n^3/3, two n x n
    # triangular solves 2 n^3), Jbar = 2 Cbar J (2 n^2 q)
    flops_b = batch * (2.0 * (n * n * r + n * (n + 1) * r) + n ** 3 / 3 + 2.0 * n ** 3 + 2.0 * n * n * q)
    t_b = t_fb - t_f
    # gradient accuracy: the last fwd_bwd's gradients against the oracle's closed form, sampled
    import numpy as np

    import oracle
    idx = np.unique(np.r_[0, batch - 1, np.random.default_rng(13).integers(0, batch, 256)]).astype(np.int64)
    sel = torch.as_tensor(idx, device=dev)
    ref = oracle.spd_solve_loss_grad(*(x[sel].cpu().numpy() for x in (Qd, J, B, W)))
    worst = 0.0
    for t, key in zip(ts, ("Qbar", "Jbar", "Bbar", "Wbar")):
        g = t.grad[sel].cpu().numpy().reshape(len(idx), -1)
        rr = ref[key].reshape(len(idx), -1)
        worst = max(worst, float(np.max(np.linalg.norm(g - rr, axis=1) / np.linalg.norm(rr, axis=1))))
    return {"batch": batch, "n": n, "q": q, "r": r, "forward_ms": round(t_f, 3),
            "forward_backward_ms": round(t_fb, 3), "plain_forward_ms": round(t_p, 3),
            "backward_over_forward": round(t_b / t_f, 3),
            "forward_gflops": round(flops_f / t_f / 1e6, 2),
            "backward_gflop": round(flops_b / 1e9, 3), "backward_gflops": round(flops_b / t_b / 1e6, 2),
            "backward_frac_of_fp64_peak": round(flops_b / (t_b * 1e-3) / peak, 4) if peak else None,
            "max_gradient_error_vs_oracle": worst,
            "gradient_sample": "256 problems (seeded, with the first and last), per-problem normwise "
                               "relative error of Qbar, Jbar, Bbar, Wbar against the closed form"}


def precision_form(bf, torch, dev, rank, batch=16384, n=128):
    """Mixed-precision SPD solve (binary32 factor + binary64 refinement) against the all-binary64
    dpotrf + dpotrs, cond(A) in {1e2, 1e4, 1e6} (one third each); accuracy by the oracle."""
    import numpy as np

    import bfsynth
    import oracle
    kappas = (1e2, 1e4, 1e6)
    A, b, kap = bfsynth.precision_batch(batch, n, kappas, seed=bfsynth.BASE_SEED + 6 + rank, device=dev)
    Bm = b.unsqueeze(1).contiguous()
    X = torch.empty_like(Bm)
    it = torch.empty(batch, dtype=torch.int32, device=dev)
    info = torch.empty(batch, dtype=torch.int32, device=dev)
    t_mixed = _events_ms(torch, lambda: bf.dsposv(A, Bm, X=X, iter=it, info=info))
    L = torch.empty_like(A)
    X64 = torch.empty_like(Bm)

    def fp64():
        L.copy_(A)
        bf.dpotrf(L)
        X64.copy_(Bm)
        bf.dpotrs(L, X64)

    t_copy = _events_ms(torch, lambda: (L.copy_(A), X64.copy_(Bm)))
    t_fp64 = _events_ms(torch, fp64) - t_copy
    itn, kapn = it.cpu().numpy(), kap.numpy()
    # accuracy, per result: backward error of every solution, computed by the oracle in binary64
    An, xn, bn = A.cpu().numpy(), X[:, 0, :].cpu().numpy(), b.cpu().numpy()
    eta = oracle.backward_error(An, xn, bn)
    eta64 = oracle.backward_error(An, X64[:, 0, :].cpu().numpy(), bn)
    x64 = X64[:, 0, :].cpu().numpy()
    fwd = np.abs(xn - x64).max(1) / np.abs(x64).max(1)
    per = {}
    for k in kappas:
        m = kapn == k
        per[f"{k:.0e}"] = {"iters_mean": round(float(itn[m].mean()), 3), "iters_max": int(itn[m].max()),
                           "fallbacks": int((itn[m] < 0).sum()), "eta_max": float(eta[m].max()),
                           "eta_fp64_max": float(eta64[m].max()), "fwd_diff_max": float(fwd[m].max())}
    return {"batch": batch, "n": n, "mixed_ms": round(t_mixed, 3), "fp64_ms": round(t_fp64, 3),
            "speedup": round(t_fp64 / t_mixed, 3), "eta_max": float(eta.max()),
            "all_info_zero": int((info != 0).sum()) == 0, "per_kappa": per}


def vbatched_form(bf, torch, dev, peak):
    """The variable-size entry points on mixed sizes: dpotrf on the ragged workload's 200,000
    orders (log-uniform in [2, 200], factor only), dgemm_nn and dtrsm_rltu on 100,000 problems
    with m, n, k uniform in [1, 64]; every problem's sizes and pointers in device arrays."""
    import ctypes

    import bfsynth
    ip = lambda t: ctypes.c_void_p(t.data_ptr())
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = {}
    ns = bfsynth.ragged_orders(200000, 2, 200, bfsynth.BASE_SEED + 3)
    S0, offS, _, _ = bfsynth.ragged_spd(ns, 1, bfsynth.BASE_SEED + 4, device=dev)
    S = S0.clone()
    n_d = ns.to(dev)
    ptr = (S.data_ptr() + 8 * offS.to(dev, torch.int64)).contiguous()
    info = torch.empty(len(ns), dtype=torch.int32, device=dev)

    def potrf():
        _ok(bf.bf_dpotrf_vbatched(b"L", ip(n_d), ip(ptr), ip(n_d), ip(info), len(ns), 200, st))
    ms = _events_ms(torch, potrf, before=lambda: S.copy_(S0))
    nf = ns.to(torch.float64)
    f = float((nf ** 3 / 3 + nf ** 2 / 2 + nf / 6).sum())
    out["dpotrf_ragged_200k"] = {"ms": round(ms, 3), "gflops": round(f / ms / 1e6, 1),
                                 "frac": round(f / ms * 1e3 / peak, 4), "all_info_zero": int(info.abs().max()) == 0}
    del S0, S, ptr
    g = torch.Generator().manual_seed(bfsynth.BASE_SEED + 7)
    cnt = 100000
    mm, nn, kk = (torch.randint(1, 65, (cnt,), generator=g) for _ in range(3))

    def offsets(sz):
        o = torch.zeros(cnt, dtype=torch.int64)
        o[1:] = torch.cumsum(sz, 0)[:-1]
        return o, int(sz.sum())
    (oa, na), (ob, nb), (oc, nc), (ol, nl) = (offsets(x) for x in (mm * kk, kk * nn, mm * nn, nn * nn))
    A = torch.randn(na, dtype=torch.float64, device=dev)
    B = torch.randn(nb, dtype=torch.float64, device=dev)
    C = torch.randn(nc, dtype=torch.float64, device=dev)
    L = torch.randn(nl, dtype=torch.float64, device=dev) * 0.01  # unit lower: the strict part is read
    m_d, n_d, k_d = (x.to(dev, torch.int32) for x in (mm, nn, kk))
    pa, pb, pc, pl = ((X.data_ptr() + 8 * o).to(dev) for X, o in ((A, oa), (B, ob), (C, oc), (L, ol)))
    dinfo = torch.empty(cnt, dtype=torch.int32, device=dev)

    def gemm():
        _ok(bf.bf_dgemm_vbatched(b"N", b"N", ip(m_d), ip(n_d), ip(k_d), 1.0, ip(pa), ip(m_d), ip(pb), ip(k_d), 1.0,
                                 ip(pc), ip(m_d), cnt, 64, 64, 64, ip(dinfo), st))
    ms = _events_ms(torch, gemm)
    f = float((2 * mm * nn * kk).to(torch.float64).sum())
    out["dgemm_nn_100k_mnk_1_64"] = {"ms": round(ms, 3), "gflops": round(f / ms / 1e6, 1),
                                     "frac": round(f / ms * 1e3 / peak, 4), "dinfo_zero": int(dinfo.abs().max()) == 0}

    def trsm():
        _ok(bf.bf_dtrsm_vbatched(b"R", b"L", b"T", b"U", ip(m_d), ip(n_d), 1.0, ip(pl), ip(n_d), ip(pc), ip(m_d),
                                 cnt, 64, 64, ip(dinfo), st))
    ms = _events_ms(torch, trsm)
    f = float((mm * nn * (nn - 1)).to(torch.float64).sum())
    out["dtrsm_rltu_100k_mn_1_64"] = {"ms": round(ms, 3), "gflops": round(f / ms / 1e6, 1),
                                      "frac": round(f / ms * 1e3 / peak, 4), "dinfo_zero": int(dinfo.abs().max()) == 0}
    return out


def _ok(status):
    if status != 0:
        raise RuntimeError(f"library call returned {status}")


def next_rows(bf, torch, dev, peak):
    """The routines beyond the sweep: dsyrk (ln, ut), dtrmm (rlnn, llnn), dpotrf 'U', dgetrf, skinny
    dgemm_nt, the fused
    dsyrk + dpotrf against its two calls, and the square-root Riccati recursion (section 5) with the
    fused routine against dsyrk + dpotrf; GFLOP/s and the fraction of the FP64 peak."""
    import bfsynth

    def rate(fl, ms):
        return {"ms": round(ms, 3), "gflops": round(fl / ms / 1e6, 1), "frac": round(fl / (ms * 1e-3) / peak, 4)}

    out = {"peak_tflops": round(peak / 1e12, 4)}
    for n in (16, 64, 256):
        b = bfsynth.sweep_batch(n, n, 2)
        A = bfsynth.randn_batch(b, n, n, n, 31, device=dev)
        C = bfsynth.randn_batch(b, n, n, n, 32, device=dev)
        fl = b * n * (n + 1) * n
        row = {"batch": b}
        for uplo, tr in (("L", "N"), ("U", "T")):
            row[f"dsyrk_{uplo.lower()}{tr.lower()}"] = rate(fl, _events_ms(
                torch, lambda: bf.dsyrk(uplo, tr, 1.0, A, 1.0, C, n=n, k=n)))
        L = bfsynth.spd_batch(b, n, n, 33, device=dev)
        bf.dpotrf(L)
        for side in "RL":
            row[f"dtrmm_{side.lower()}lnn"] = rate(b * n * n * (n + 1), _events_ms(
                torch, lambda: bf.dtrmm(side, "L", "N", "N", 1.0, L, C)))
        del A, C, L
        b1 = bfsynth.sweep_batch(n, n, 1)
        S0 = bfsynth.spd_batch(b1, n, n, 34, device=dev)
        S = S0.clone()
        ms = _events_ms(torch, lambda: bf.dpotrf(S, uplo="U"), before=lambda: S.copy_(S0))
        row["dpotrf_u"] = rate(b1 * (n ** 3 / 3 + n ** 2 / 2 + n / 6), ms)
        # dgetrf on the same batch (LAPACK's flop count 2n^3/3 - n^2/2 + 5n/6)
        ipiv = torch.empty(b1, n, dtype=torch.int32, device=dev)
        info = torch.empty(b1, dtype=torch.int32, device=dev)
        ms = _events_ms(torch, lambda: bf.dgetrf(S, ipiv=ipiv, info=info), before=lambda: S.copy_(S0))
        row["dgetrf"] = rate(b1 * (2 * n ** 3 / 3 - n ** 2 / 2 + 5 * n / 6), ms)
        del ipiv, info
        del S, S0
        torch.cuda.empty_cache()
        out[f"n{n}"] = row
    # skinny dgemm_nt (one dimension 4): C (m x n) += A (m x k) B^T (B n x k), ~2 GiB of operands
    for m, n, k in ((4, 256, 256), (256, 4, 256)):
        b = (1 << 31) // (8 * (m * k + n * k + m * n))
        A = bfsynth.randn_batch(b, m, k, m, 38, device=dev)
        B = bfsynth.randn_batch(b, n, k, n, 39, device=dev)
        C = bfsynth.randn_batch(b, m, n, m, 40, device=dev)
        out[f"dgemm_nt_m{m}_n{n}_k{k}"] = dict(batch=b, **rate(2.0 * b * m * n * k, _events_ms(
            torch, lambda: bf.dgemm("N", "T", 1.0, A, B, 1.0, C, m=m, n=n, k=k))))
        del A, B, C
    for n in (8, 32):
        b = bfsynth.sweep_batch(n, n, 1) // 2
        k = n // 2
        Y = bfsynth.randn_batch(b, n, k, n, 35, device=dev)
        S0 = bfsynth.spd_batch(b, n, n, 36, device=dev)
        S = S0.clone()
        fl = b * (n * (n + 1) * k + n ** 3 / 3 + n ** 2 / 2 + n / 6)

        def two_calls():
            bf.dsyrk("L", "N", 1.0, Y, 1.0, S, n=n, k=k)
            bf.dpotrf(S)

        out[f"dsyrk_dpotrf_n{n}"] = {
            "batch": b, "k": k,
            "fused_routine": rate(fl, _events_ms(torch, lambda: bf.dsyrk_dpotrf(Y, S, n=n, k=k),
                                                 before=lambda: S.copy_(S0))),
            "dsyrk_then_dpotrf": rate(fl, _events_ms(torch, two_calls, before=lambda: S.copy_(S0)))}
        del Y, S, S0
    # Riccati recursion, N = 10 stages; batches of ~16 GB of stage data (up to 64k problems)
    N = 10
    for nx, nu in ((8, 4), (24, 12), (40, 20), (64, 32)):
        m = nx + nu
        per = 8 * (N * m * nx + 2 * (N + 1) * m * m + nx * nx)
        batch = int(min(65536, 16e9 // per))
        BAt, RSQ, QN = bfsynth.riccati_batch(batch, N, nx, nu, 37 + nx, device=dev)
        F = torch.empty(batch, N + 1, m, m, dtype=torch.float64, device=dev)
        info = torch.empty(batch, dtype=torch.int32, device=dev)
        work = torch.empty(bf.bf_riccati_workspace_bytes(nx, nu, batch), dtype=torch.uint8, device=dev)
        fl = batch * (nx ** 3 / 3 + N * (m * nx * (nx + 1) + m * (m + 1) * nx + m ** 3 / 3 + m ** 2 / 2 + m / 6))
        row = {"batch": batch, "N": N}
        for fused in (True, False):
            ms = _events_ms(torch, lambda: bf.riccati(BAt, RSQ, QN, nx, nu, F=F, info=info, fused=fused, work=work))
            r = rate(fl, ms)
            r["us_per_recursion"] = round(ms * 1e3 / batch, 4)
            row["fused_routine" if fused else "dsyrk_then_dpotrf"] = r
        row["all_info_zero"] = int((info != 0).sum()) == 0
        out[f"riccati_nx{nx}_nu{nu}"] = row
        del BAt, RSQ, QN, F, work
        torch.cuda.empty_cache()
    return out


def sweep_config(world):
    """The workload both arms report: the size sweep of every routine and point."""
    return {"workload": "size sweep: n in {4,8,12,16,24,32,48,64,96,128,192,256} x lda in "
                        "{n, n+3}, ~2 GiB of operands per routine and point; dgemm nn/nt/tn/tt "
                        "(m=n=k, C += op(A)op(B)), dtrsm rltu + rltn, dpotrf_l",
            "l2": "no flush: every point's inputs (~2 GiB) exceed the 126 MiB L2",
            "dpotrf_inputs": "refreshed in-step from S's untouched upper triangle (torch copy)",
            "parallelism": f"replicas x{world} (no collective on the data path)"}


def reference_arm(args, rank, world):
    """The oracle timed as it stands on the host cores (rank 0 only)."""
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample()
    t = []
    rates = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        v, desc, cores = oracle_sample()
        t.append(time.perf_counter() - t0)
        rates.append(v)
    v = statistics.mean(rates)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "GFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1000 * statistics.mean(t), 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": sweep_config(world),
        "cpu_baseline": {"value": round(v, 3), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": round(v, 3), "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


if __name__ == "__main__":
    main()
