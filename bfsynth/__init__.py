"""Seeded synthetic inputs for the batched small-matrix FP64 workloads.

This module only draws random numbers and assembles test matrices from them;
it contains none of the library's arithmetic (no gemm, trsm or Cholesky of
its own).  It is the one module that both the CPU oracle's tests and the GPU
tests/benchmark use, so that both sides see the same bytes.

Layout: a batch of column-major matrices with ``ncols`` columns and leading
dimension ``ld`` is a contiguous torch tensor of shape ``(batch, ncols, ld)``;
element (i, j) of problem b is ``X[b, j, i]``.  Rows ``n..ld-1`` (the leading
dimension padding) are filled with NaN so that a kernel that reads or writes
them is caught.

Workload recipes (the paper's experiments use square matrices of order up to
300 with random entries, sections 4 and Appendix B; the configurations below
fix the distributions):

* dense operands: entries i.i.d. N(0, 1);
* SPD matrices: S = G G^T + n I with G i.i.d. N(0, 1) (n x n);
* unit-scaled triangular factors for the triangular-solve sweep:
  L_u = L diag(L)^{-1} with L the Cholesky factor of such an S (the factor is
  produced with torch.linalg.cholesky, a library routine used only to build
  inputs);
* ragged orders: n = clamp(round(exp(U(ln lo, ln hi))), lo, hi);
* conditioned SPD matrices: A = Q diag(s) Q^T, Q Haar-orthogonal (QR of a
  Gaussian matrix with the signs of R's diagonal folded into Q), s_i =
  kappa^{-i/(n-1)}, symmetrised;
* differentiation inputs: Q = diag(U(1, 2)), J, B, W i.i.d. N(0, 1).

Every generator takes a seed and a device; the generator state is local
(``torch.Generator``), so results do not depend on global RNG state.
"""
from __future__ import annotations

import math

import torch

BASE_SEED = 20190221


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=torch.device(device))
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    return g


def padded(batch: int, rows: int, ncols: int, ld: int, device="cpu", fill=float("nan")):
    """An uninitialised-looking batch: NaN everywhere (rows >= `rows` stay NaN)."""
    if ld < max(1, rows):
        raise ValueError("leading dimension smaller than the row count")
    return torch.full((batch, ncols, ld), fill, dtype=torch.float64, device=device)


def randn_batch(batch: int, rows: int, ncols: int, ld: int, seed: int, device="cpu",
                pad=float("nan")) -> torch.Tensor:
    """i.i.d. N(0,1) entries in rows < `rows`; padding rows hold `pad`."""
    g = _gen(seed, device)
    x = torch.randn((batch, ncols, rows), generator=g, dtype=torch.float64, device=device)
    if ld == rows:
        return x
    out = padded(batch, rows, ncols, ld, device, pad)
    out[:, :, :rows] = x
    return out


def randint_batch(batch: int, rows: int, ncols: int, ld: int, seed: int, lo=-3, hi=3,
                  device="cpu", pad=float("nan")) -> torch.Tensor:
    """Integer-valued entries in [lo, hi] (exact in binary64 under any summation order)."""
    g = _gen(seed, device)
    x = torch.randint(lo, hi + 1, (batch, ncols, rows), generator=g, device=device).to(torch.float64)
    if ld == rows:
        return x
    out = padded(batch, rows, ncols, ld, device, pad)
    out[:, :, :rows] = x
    return out


def spd_batch(batch: int, n: int, ld: int, seed: int, device="cpu", pad=float("nan"),
              chunk: int = 65536) -> torch.Tensor:
    """S = G G^T + n I, G i.i.d. N(0,1); column-major with leading dimension ld.

    Formed in chunks with torch.bmm (a library product used only to build inputs).
    """
    out = padded(batch, n, n, ld, device, pad) if ld != n else torch.empty(
        (batch, n, n), dtype=torch.float64, device=device)
    g = _gen(seed, device)
    eye = torch.eye(n, dtype=torch.float64, device=device) * n
    for s in range(0, batch, chunk):
        e = min(batch, s + chunk)
        G = torch.randn((e - s, n, n), generator=g, dtype=torch.float64, device=device)
        S = torch.bmm(G, G.transpose(1, 2)) + eye
        S = 0.5 * (S + S.transpose(1, 2))  # exact symmetry
        out[s:e, :, :n] = S
    return out


def unit_lower_batch(batch: int, n: int, ld: int, seed: int, device="cpu",
                     pad=float("nan"), unit=True, chunk: int = 65536) -> torch.Tensor:
    """Lower-triangular factor of an SPD S = G G^T + n I, optionally unit-scaled.

    unit=True returns L_u = L diag(L)^{-1} (unit diagonal stored explicitly);
    unit=False returns the Cholesky factor L itself.  The strict upper
    triangle is filled with NaN (a triangular solve must not read it).
    """
    out = padded(batch, n, n, ld, device, pad)
    g = _gen(seed, device)
    eye = torch.eye(n, dtype=torch.float64, device=device) * n
    upper = torch.triu(torch.ones(n, n, dtype=torch.bool, device=device), diagonal=1)
    for s in range(0, batch, chunk):
        e = min(batch, s + chunk)
        G = torch.randn((e - s, n, n), generator=g, dtype=torch.float64, device=device)
        S = torch.bmm(G, G.transpose(1, 2)) + eye
        S = 0.5 * (S + S.transpose(1, 2))
        L = torch.linalg.cholesky(S)  # row-major (i, j) = L_ij
        if unit:
            L = L / torch.diagonal(L, dim1=1, dim2=2).unsqueeze(1)
        Lc = L.transpose(1, 2).clone()  # Lc[b, j, i] = L_ij (column-major)
        Lc.masked_fill_(upper.t().unsqueeze(0), float("nan"))  # Lc[b, j, i] with i < j
        out[s:e, :, :n] = Lc
    return out


def ragged_orders(count: int, lo: int, hi: int, seed: int) -> torch.Tensor:
    """n = clamp(round(exp(U(ln lo, ln hi))), lo, hi), int32 on the CPU."""
    g = _gen(seed, "cpu")
    u = torch.rand(count, generator=g, dtype=torch.float64)
    n = torch.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
    return torch.clamp(torch.round(n), lo, hi).to(torch.int32)


def ragged_spd(ns: torch.Tensor, nrhs: int, seed: int, device="cpu"):
    """Ragged batch of S_b = G_b G_b^T + n_b I (leading dimension n_b) and RHS.

    Returns (S_flat, offS, B_flat, offB): flat float64 tensors and int64 element
    offsets; problem b's matrix starts at offS[b], its n_b x nrhs right-hand
    sides (N(0,1), leading dimension n_b) at offB[b].  Offsets are rounded up to
    an even element count so that every problem starts on a 16-byte boundary.
    """
    ns_cpu = ns.to("cpu", torch.int64)
    sizesS = ns_cpu * ns_cpu
    sizesB = ns_cpu * nrhs
    sizesS = sizesS + (sizesS & 1)
    sizesB = sizesB + (sizesB & 1)
    offS = torch.zeros_like(ns_cpu)
    offB = torch.zeros_like(ns_cpu)
    offS[1:] = torch.cumsum(sizesS, 0)[:-1]
    offB[1:] = torch.cumsum(sizesB, 0)[:-1]
    totS = int(sizesS.sum())
    totB = int(sizesB.sum())
    S = torch.zeros(totS, dtype=torch.float64, device=device)
    Bf = torch.zeros(totB, dtype=torch.float64, device=device)
    g = _gen(seed, device)
    # group problems by order so that each group is built with one batched product
    order = torch.argsort(ns_cpu, stable=True)
    sorted_n = ns_cpu[order]
    uniq, counts = torch.unique_consecutive(sorted_n, return_counts=True)
    start = 0
    for n, c in zip(uniq.tolist(), counts.tolist()):
        idx = order[start:start + c]
        start += c
        G = torch.randn((c, n, n), generator=g, dtype=torch.float64, device=device)
        Sm = torch.bmm(G, G.transpose(1, 2)) + n * torch.eye(n, dtype=torch.float64, device=device)
        Sm = 0.5 * (Sm + Sm.transpose(1, 2))
        Rm = torch.randn((c, nrhs, n), generator=g, dtype=torch.float64, device=device)
        # scatter: column-major of a symmetric matrix equals its row-major flattening
        posS = (offS[idx].unsqueeze(1) + torch.arange(n * n).unsqueeze(0)).to(device)
        S.index_put_((posS.reshape(-1),), Sm.reshape(-1))
        posB = (offB[idx].unsqueeze(1) + torch.arange(n * nrhs).unsqueeze(0)).to(device)
        Bf.index_put_((posB.reshape(-1),), Rm.reshape(-1))
    return S, offS, Bf, offB


def haar_orthogonal(batch: int, n: int, seed: int, device="cpu") -> torch.Tensor:
    """Haar-distributed orthogonal matrices (row-major (batch, n, n))."""
    g = _gen(seed, device)
    Z = torch.randn((batch, n, n), generator=g, dtype=torch.float64, device=device)
    Q, R = torch.linalg.qr(Z)
    d = torch.sign(torch.diagonal(R, dim1=1, dim2=2))
    d = torch.where(d == 0, torch.ones_like(d), d)
    return Q * d.unsqueeze(1)


def conditioned_spd(batch: int, n: int, kappa: float, seed: int, device="cpu",
                    chunk: int = 4096) -> torch.Tensor:
    """A = Q diag(s) Q^T with s_i = kappa^{-i/(n-1)}: cond_2(A) = kappa (column-major)."""
    out = torch.empty((batch, n, n), dtype=torch.float64, device=device)
    i = torch.arange(n, dtype=torch.float64, device=device)
    s = torch.pow(torch.tensor(float(kappa), dtype=torch.float64, device=device),
                  -i / max(1, n - 1))
    for c0 in range(0, batch, chunk):
        c1 = min(batch, c0 + chunk)
        Q = haar_orthogonal(c1 - c0, n, seed * 1000003 + c0, device)
        A = torch.bmm(Q * s.unsqueeze(0).unsqueeze(0), Q.transpose(1, 2))
        A = 0.5 * (A + A.transpose(1, 2))
        out[c0:c1] = A
    return out


def precision_batch(batch: int, n: int, kappas, seed: int, device="cpu"):
    """Equal thirds (first gets the remainder) of conditioned SPD systems + N(0,1) RHS.

    Returns (A (batch, n, n) column-major, b (batch, n), kappa_of_problem (batch,)).
    """
    kappas = list(kappas)
    parts = [batch // len(kappas)] * len(kappas)
    for t in range(batch - sum(parts)):
        parts[t] += 1
    As, ks = [], []
    for t, (kap, cnt) in enumerate(zip(kappas, parts)):
        As.append(conditioned_spd(cnt, n, kap, seed + 17 * t, device))
        ks.append(torch.full((cnt,), float(kap), dtype=torch.float64))
    g = _gen(seed + 99991, device)
    b = torch.randn((batch, n), generator=g, dtype=torch.float64, device=device)
    return torch.cat(As, 0), b, torch.cat(ks, 0)


def diff_batch(batch: int, n: int, q: int, r: int, seed: int, device="cpu"):
    """Differentiation workload: Qd ~ U(1,2) (batch, n); J (batch, q, n); B, W (batch, r, n)."""
    g = _gen(seed, device)
    Qd = 1.0 + torch.rand((batch, n), generator=g, dtype=torch.float64, device=device)
    J = torch.randn((batch, q, n), generator=g, dtype=torch.float64, device=device)
    B = torch.randn((batch, r, n), generator=g, dtype=torch.float64, device=device)
    W = torch.randn((batch, r, n), generator=g, dtype=torch.float64, device=device)
    return Qd, J, B, W


# ---------------------------------------------------------------------------
# Workload shapes of the size sweep: square problems of these orders, each
# point's batch chosen so that its operands total about 2 GiB.
SWEEP_N = (4, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256)
SWEEP_BYTES = 2 ** 31


def sweep_batch(n: int, ld: int, operands: int) -> int:
    """Problems per sweep point: floor(2 GiB / (operands * ld * n * 8 bytes))."""
    return SWEEP_BYTES // (operands * ld * n * 8)


def riccati_batch(batch: int, N: int, nx: int, nu: int, seed: int, device="cpu"):
    """Inputs of the square-root Riccati recursion (section 5), m = nu + nx, per problem:
    N stages of BAt = [B^T; A^T] (m x nx) with A ~ N(0, 1/nx) (nx x nx) and B ~ N(0, 1/nx)
    (nx x nu), and of RSQ = [R S; S^T Q] = G G^T + m I with G ~ N(0, 1) (m x m); the terminal
    Q_N = H H^T + nx I, H ~ N(0, 1).  Column-major layouts: BAt (batch, N, nx, m), RSQ
    (batch, N, m, m), QN (batch, nx, nx)."""
    g = _gen(seed, device)
    m = nx + nu
    f = dict(generator=g, dtype=torch.float64, device=device)
    A = torch.randn(batch, N, nx, nx, **f) / nx ** 0.5
    B = torch.randn(batch, N, nx, nu, **f) / nx ** 0.5
    BAt = torch.cat([B.transpose(-1, -2), A.transpose(-1, -2)], dim=-2).transpose(-1, -2).contiguous()
    del A, B
    G = torch.randn(batch, N, m, m, **f)
    RSQ = G @ G.transpose(-1, -2)
    del G
    RSQ = 0.5 * (RSQ + RSQ.transpose(-1, -2)) + m * torch.eye(m, dtype=torch.float64, device=device)
    H = torch.randn(batch, nx, nx, **f)
    QN = H @ H.transpose(-1, -2) + nx * torch.eye(nx, dtype=torch.float64, device=device)
    return BAt, RSQ.contiguous(), QN.contiguous()
