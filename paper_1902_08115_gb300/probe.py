"""FP64 machine model of the GPU this runs on (the measurements behind the kernel design).

Times the library's probes and prints one JSON object:
  * FP64 FMA throughput (bf_probe_fp64_ex) with all lanes, with 16/8/1 active lanes per
    warp (cost of a masked FP64 instruction), with 1/2/4/8 warps per SM (whether the FP64
    unit is per SM sub-partition), and with one dependent chain per thread instead of the
    4x4 register-tile pattern;
  * FP64 tensor-core MMA (mma.sync m8n8k4 and m16n8k4, bf_probe_kind 0 and 1) against it;
  * the cost of FP64 sqrt, 1/x and rsqrt in FMA issue slots, and binary32 FMA throughput.

    python -m paper_1902_08115_gb300.probe
"""
from __future__ import annotations

import json
import os
import sys

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def _best_seconds(launch, reps=3):
    import torch
    launch()
    best = None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        launch()
        e1.record()
        e1.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        best = t if best is None else min(best, t)
    return best


def measure():
    import torch

    import paper_1902_08115_gb300 as bf
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = torch.empty(sms * 8 * 1024, dtype=torch.float64, device="cuda")
    st = bf._stream()

    def rate(blocks, threads, iters, active=32, chains=0):
        args = (blocks, threads, iters, active, chains, bf._ptr(out), st)
        bf._check("bf_probe_fp64_ex", bf.bf_probe_fp64_ex(*args))
        t = _best_seconds(lambda: bf.bf_probe_fp64_ex(*args))
        flops = 2.0 * 16 * iters * blocks * threads  # full-warp equivalent
        return round(flops / t / 1e12, 4)

    def kind_seconds(kind, blocks, threads, iters):
        args = (kind, blocks, threads, iters, bf._ptr(out), st)
        bf._check("bf_probe_kind", bf.bf_probe_kind(*args))
        return _best_seconds(lambda: bf.bf_probe_kind(*args))

    res = {"gpu": torch.cuda.get_device_name(), "sms": sms, "unit": "TFLOP/s (full-warp equivalent)"}
    res["tile_all_lanes_8_warps_per_sm"] = dfma = rate(sms * 2, 128, 2048)
    res["chain_all_lanes_8_warps_per_sm"] = rate(sms * 2, 128, 2048, chains=1)
    for a in (16, 8, 1):
        res[f"tile_{a}_active_lanes"] = rate(sms * 2, 128, 2048, active=a)
    for w in (1, 2, 4, 8):
        res[f"tile_{w}_warps_per_sm"] = rate(sms, 32 * w, 2048)
    # one FP64 unit per SM or per sub-partition: 4 busy warps of a 16-warp CTA (indices 0, 4, 8,
    # 12: one sub-partition if warps are dealt by index modulo 4) against 4 warps per SM above
    t = kind_seconds(6, sms, 512, 2048)
    res["tile_4_warps_one_subpartition"] = round(2.0 * 16 * 2048 * sms * 4 * 32 / t / 1e12, 4)
    # FP64 tensor cores: 4 MMAs per iteration and warp, at 4 and 8 warps per SM
    for kind, name, flops_per_mma in ((0, "dmma_m8n8k4", 512), (1, "dmma_m16n8k4", 1024)):
        for w in (4, 8):
            iters = 1024
            t = kind_seconds(kind, sms * 2, 16 * w, iters)
            warps = sms * 2 * (16 * w) // 32
            res[f"{name}_{w}_warps_per_sm"] = round(4 * flops_per_mma * iters * warps / t / 1e12, 4)
    # special functions: per thread 4 x (op + 1 FMA) per iteration; slots = FMA-equivalents - 1
    fma_per_s = dfma * 1e12 / 2.0
    for kind, name in ((2, "sqrt"), (3, "rcp"), (4, "rsqrt")):
        iters = 512
        blocks, threads = sms * 2, 128
        t = kind_seconds(kind, blocks, threads, iters)
        slots = t * fma_per_s / (4.0 * iters * blocks * threads)
        res[f"fp64_{name}_fma_slots"] = round(slots - 1.0, 2)
    iters = 8192
    t = kind_seconds(5, sms * 4, 256, iters)
    res["ffma_tflops"] = round(2.0 * 16 * iters * sms * 4 * 256 / t / 1e12, 2)
    res["dmma_over_dfma"] = round(max(res[k] for k in res if k.startswith("dmma_")) / dfma, 3)
    return res


if __name__ == "__main__":
    print(json.dumps(measure()))
