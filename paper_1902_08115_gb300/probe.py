"""FP64 machine model of the GPU this runs on (the measurements behind the kernel design).

Times the library's FP64 FMA probe (bf_probe_fp64_ex) in several forms and
prints one JSON object: FMA throughput with all lanes, with 16/8/1 active
lanes per warp (cost of a masked FP64 instruction), with 1/2/4/8 warps per SM
(whether the FP64 unit is per SM sub-partition), and with a single dependent
chain per thread instead of the 4x4 register-tile pattern.

    python -m paper_1902_08115_gb300.probe
"""
from __future__ import annotations

import json
import os
import sys

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def measure():
    import torch

    import paper_1902_08115_gb300 as bf
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = torch.empty(sms * 8 * 1024, dtype=torch.float64, device="cuda")
    st = bf._stream()

    def rate(blocks, threads, iters, active=32, chains=0):
        args = (blocks, threads, iters, active, chains, bf._ptr(out), st)
        bf._check("bf_probe_fp64_ex", bf.bf_probe_fp64_ex(*args))
        best = 0.0
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            bf.bf_probe_fp64_ex(*args)
            e1.record()
            e1.synchronize()
            flops = 2.0 * 16 * iters * blocks * threads  # full-warp equivalent
            best = max(best, flops / (e0.elapsed_time(e1) * 1e-3))
        return round(best / 1e12, 4)

    res = {"gpu": torch.cuda.get_device_name(), "sms": sms, "unit": "TFLOP/s (full-warp equivalent)"}
    res["tile_all_lanes_8_warps_per_sm"] = rate(sms * 2, 128, 2048)
    res["chain_all_lanes_8_warps_per_sm"] = rate(sms * 2, 128, 2048, chains=1)
    for a in (16, 8, 1):
        res[f"tile_{a}_active_lanes"] = rate(sms * 2, 128, 2048, active=a)
    for w in (1, 2, 4, 8):
        res[f"tile_{w}_warps_per_sm"] = rate(sms, 32 * w, 2048)
    return res


if __name__ == "__main__":
    print(json.dumps(measure()))
