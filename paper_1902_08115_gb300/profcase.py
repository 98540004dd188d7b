"""One routine on a batch larger than L2 (256-384 MiB of operands), run three times: a
small, self-contained case for kernel profilers.  dpotrf also takes a batch size (the size
switch then picks the form that batch gets).

    python -m paper_1902_08115_gb300.profcase {potrf|gemm|trsm|getrf} N [PAD [BATCH]]
    python -m paper_1902_08115_gb300.profcase dsposv      (2048 SPD systems of order 128)
    python -m paper_1902_08115_gb300.profcase ragged      (3000 orders in [100, 200], 4 RHS)
    python -m paper_1902_08115_gb300.profcase vbatched    (dgemm_nn, 40,000 problems, m, n, k in [1, 64])
    python -m paper_1902_08115_gb300.profcase diff        (the differentiation workload's forward and
                                                           backward, 16,384 problems of order 32)
"""
from __future__ import annotations

import os
import sys

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main(argv):
    import torch

    import bfsynth
    import paper_1902_08115_gb300 as bf
    which = argv[0]
    if which == "dsposv":
        A = bfsynth.spd_batch(2048, 128, 128, 3, device="cuda")
        b = torch.randn(2048, 1, 128, dtype=torch.float64, device="cuda")
        for _ in range(3):
            bf.dsposv(A, b)
        torch.cuda.synchronize()
        print("ok dsposv")
        return
    if which == "diff":
        from paper_1902_08115_gb300 import autograd as ag
        Qd, J, B, W = bfsynth.diff_batch(16384, 32, 16, 8, seed=bfsynth.BASE_SEED, device="cuda")
        ts = [x.clone().requires_grad_(True) for x in (Qd, J, B, W)]
        for _ in range(3):
            for t in ts:
                t.grad = None
            loss, _, _ = ag.spd_solve_loss(*ts)
            loss.backward()
        torch.cuda.synchronize()
        print("ok diff")
        return
    if which == "vbatched":
        import ctypes
        g = torch.Generator().manual_seed(5)
        cnt = 40000
        mm, nn, kk = (torch.randint(1, 65, (cnt,), generator=g) for _ in range(3))

        def offsets(sz):
            o = torch.zeros(cnt, dtype=torch.int64)
            o[1:] = torch.cumsum(sz, 0)[:-1]
            return o, int(sz.sum())
        (oa, na), (ob, nb), (oc, nc) = (offsets(x) for x in (mm * kk, kk * nn, mm * nn))
        A, B, C = (torch.randn(x, dtype=torch.float64, device="cuda") for x in (na, nb, nc))
        m_d, n_d, k_d = (x.to("cuda", torch.int32) for x in (mm, nn, kk))
        pa, pb, pc = ((X.data_ptr() + 8 * o).to("cuda") for X, o in ((A, oa), (B, ob), (C, oc)))
        ip = lambda t: ctypes.c_void_p(t.data_ptr())
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for _ in range(3):
            assert bf.bf_dgemm_vbatched(b"N", b"N", ip(m_d), ip(n_d), ip(k_d), 1.0, ip(pa), ip(m_d), ip(pb), ip(k_d),
                                        1.0, ip(pc), ip(m_d), cnt, 64, 64, 64, None, st) == 0
        torch.cuda.synchronize()
        print("ok vbatched")
        return
    if which == "ragged":
        ns = bfsynth.ragged_orders(3000, 100, 200, 5)
        S0, offS, B0, offB = bfsynth.ragged_spd(ns, 4, 6, device="cuda")
        S, B = S0.clone(), B0.clone()
        plan = bf.RaggedPlan(ns.numpy(), S, offS.numpy(), B, offB.numpy(), 4, **bf.ragged_config())
        for _ in range(3):
            S.copy_(S0)
            B.copy_(B0)
            plan.launch()
        torch.cuda.synchronize()
        print("ok ragged")
        return
    n = int(argv[1])
    pad = int(argv[2]) if len(argv) > 2 else 0
    ld, dev = n + pad, "cuda"
    if which == "potrf":
        b = int(argv[3]) if len(argv) > 3 else max(1, (256 << 20) // (ld * n * 8))
        S0 = bfsynth.spd_batch(b, n, ld, 1, device=dev)
        S = S0.clone()
        for _ in range(3):
            S.copy_(S0)
            info = bf.dpotrf(S, n=n)
        torch.cuda.synchronize()
        assert int(info.abs().max()) == 0
    elif which == "gemm":
        b = max(1, (384 << 20) // (3 * ld * n * 8))
        A, B, C = (bfsynth.randn_batch(b, n, n, ld, s, device=dev) for s in (1, 2, 3))
        for _ in range(3):
            bf.dgemm("N", "T", 1.0, A, B, 1.0, C, m=n, n=n, k=n)
    elif which == "trsm":
        b = max(1, (256 << 20) // (2 * ld * n * 8))
        L = bfsynth.spd_batch(b, n, ld, 1, device=dev)
        bf.dpotrf(L, n=n)
        X = bfsynth.randn_batch(b, n, n, ld, 2, device=dev)
        for _ in range(3):
            bf.dtrsm("R", "L", "T", "U", 1.0, L, X, m=n, n=n)
    elif which == "getrf":
        b = max(1, (256 << 20) // (ld * n * 8))
        A0 = bfsynth.randn_batch(b, n, n, ld, 3, device=dev)
        A = A0.clone()
        for _ in range(3):
            A.copy_(A0)
            bf.dgetrf(A, n=n)
    else:
        raise SystemExit("routine must be potrf, gemm, trsm or getrf")
    torch.cuda.synchronize()
    print("ok", which, n, pad, b)


if __name__ == "__main__":
    main(sys.argv[1:])
