// bf_tune.cu -- the size switch: which kernel variant and tiling a call uses.
//
// The paper switches by matrix size between algorithmic variants, with a
// switch point that depends on the routine and the architecture and is found
// by measurement (section 2.4; section 3.1 gives 64..400 on its CPUs).  Here
// the switch is a table: built-in defaults below, overridden entry by entry
// through bf_tune_set() by the autotuner, which measures every candidate on
// the GPU it runs on.
#include <mutex>
#include <vector>

#include "bf_internal.h"
#include "../../include/bfgpu.h"

namespace bf {

struct TuneEntry {
    int routine, code, lo, hi;
    int variant, p0, p1, p2, p3;
    bool force;  // holds at every batch size (the small-batch switch is not applied)
};

static std::mutex g_mu;
static std::vector<TuneEntry> g_table;

static bool lookup(int routine, int code, int n, TuneEntry* out) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_table.rbegin(); it != g_table.rend(); ++it) {
        if (it->routine == routine && (it->code == code || it->code < 0) && n >= it->lo && n <= it->hi) {
            *out = *it;
            return true;
        }
    }
    return false;
}

// Measured batch-size bounds of dpotrf's small-batch forms (bf_tune_set_batch_rule); a
// negative bound keeps the built-in value.
struct BatchRule {
    int code, lo, hi;
    long long cta_max, team4_max, team2_max;
};

static std::vector<BatchRule> g_rules;

static bool lookup_rule(int code, int n, BatchRule* out) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_rules.rbegin(); it != g_rules.rend(); ++it) {
        if ((it->code == code || it->code < 0) && n >= it->lo && n <= it->hi) {
            *out = *it;
            return true;
        }
    }
    return false;
}

static int ceil4(int x) { return x < 4 ? 4 : (x + 3) / 4 * 4; }

static const size_t kSmemBudget = 200 * 1024;  // per CTA, below the 227 KB opt-in limit

// Make a dgemm configuration launchable: tiles are multiples of 4 no larger
// than the (rounded) problem, at most 512 threads per CTA (the kernel's launch
// bound), and the packed k-slice fits in shared memory.
static void sanitize_gemm(GemmConfig& c, int m, int n, int k) {
    if (c.variant == VAR_TINY && (m > 4 || n > 4 || k > 4)) c.variant = VAR_DIRECT;  // tiny: m, n, k <= 4
    if (c.variant == VAR_TINY) return;
    if (c.variant != VAR_DIRECT && c.variant != VAR_PACKED) c.variant = VAR_PACKED;
    c.TM = ceil4(c.TM < ceil4(m) ? c.TM : ceil4(m));
    c.TN = ceil4(c.TN < ceil4(n) ? c.TN : ceil4(n));
    while ((c.TM / 4) * (c.TN / 4) > 512) {
        if (c.TM >= c.TN) c.TM = ceil4(c.TM / 2);
        else c.TN = ceil4(c.TN / 2);
    }
    const int tpp = (c.TM / 4) * (c.TN / 4);
    if (c.P < 1) c.P = 1;
    // a table entry's P was measured on square tiles; a skinny problem's super-tile has far
    // fewer threads, so a CTA below 96 threads is raised to at least 96 (whole warps)
    if (c.P * tpp < 96) {
        while (c.P * tpp < 96 && (c.P + 1) * tpp <= 512) c.P++;
        while ((c.P * tpp) % 32 != 0 && (c.P + 1) * tpp <= 512) c.P++;
    }
    while (c.P > 1 && c.P * tpp > 512) c.P--;
    if (c.KC < 1 || c.KC > k) c.KC = k > 0 ? k : 1;
    if (c.variant == VAR_PACKED) {
        while (c.KC > 1 && gemm_smem_bytes(c) > kSmemBudget) c.KC = (c.KC + 1) / 2;
        while (c.P > 1 && gemm_smem_bytes(c) > kSmemBudget) c.P--;
    }
}

GemmConfig choose_gemm(bool ta, bool tb, int m, int n, int k, int lda, long long batch) {
    (void)batch;
    GemmConfig c;
    const int size = m > n ? m : n;
    // built-in default: whole small problems per CTA, 64 x 64 super-tiles for large ones
    if (m <= 64 && n <= 64) {
        c.TM = ceil4(m);
        c.TN = ceil4(n);
    } else {
        // split each dimension into the fewest super-tiles of at most 64, as even as possible
        c.TM = ceil4((m + (m + 63) / 64 - 1) / ((m + 63) / 64));
        c.TN = ceil4((n + (n + 63) / 64 - 1) / ((n + 63) / 64));
    }
    int tpp = (c.TM / 4) * (c.TN / 4);
    c.P = 256 / tpp > 0 ? 256 / tpp : 1;
    while ((c.P * tpp) % 32 != 0 && (c.P + 1) * tpp <= 512) c.P++;  // whole warps
    // measured on GB300: the direct form feeds the FP64 pipe as well as the packed one except
    // where op(B) is read across columns at large orders (nt/tt, n >= 64)
    c.variant = (tb && size >= 64) ? VAR_PACKED : VAR_DIRECT;
    c.KC = (m <= 64 && n <= 64) ? k : (k < 32 ? k : 32);
    TuneEntry e;
    if (lookup(BF_ROUTINE_DGEMM, (ta ? 2 : 0) + (tb ? 1 : 0), size, &e)) {
        // the tiny form pays off when a CTA's problems are one contiguous run (16-byte staging);
        // a padded A means padded problems, where the direct form reads them better
        if (e.variant == VAR_TINY && lda != (ta ? k : m)) e.variant = VAR_DIRECT;
        c.variant = e.variant;
        if (e.p0 > 0) c.TM = e.p0;
        if (e.p1 > 0) c.TN = e.p1;
        if (e.p2 > 0) c.KC = e.p2;
        if (e.p3 > 0) {
            c.P = e.p3;
        } else {
            tpp = (ceil4(c.TM < ceil4(m) ? c.TM : ceil4(m)) / 4) * (ceil4(c.TN < ceil4(n) ? c.TN : ceil4(n)) / 4);
            c.P = 256 / tpp > 0 ? 256 / tpp : 1;
            while ((c.P * tpp) % 32 != 0 && (c.P + 1) * tpp <= 512) c.P++;  // whole warps
        }
    }
    sanitize_gemm(c, m, n, k);
    return c;
}

static size_t trsm_smem(int P, int order) {
    return sizeof(double) * ((size_t)P * order * (order + 1) + (size_t)P * order);
}

static const int kGetrfCtaMaxN = 1024;  // the panel (16 n doubles) in shared memory

// largest batch for which one problem per CTA beats the lane LU, by order (n <= 64; measured
// crossovers: n = 16-24 between 2,432 and 9,728 problems, 32 ~5,000, 48 ~16,000, 64 ~32,000)
static long long getrf_cta_batch_limit(int n) {
    if (n < 32) return 2432;
    if (n < 48) return 4096;
    if (n < 64) return 16384;
    return 24576;
}

// blocked dtrsm below this many independent rows (batch x rows) from this order on
static const long long kTrsmBlockedRows = 262144;  // measured: n = 64 x 3,072 (197k rows) gains, n = 96 x 3,072 (295k) loses
static const int kTrsmBlockedMinOrder = 64;

TrsmConfig choose_trsm(int side, int uplo, int trans, int unit, int m, int n, long long batch) {
    TrsmConfig c;
    const int rows = side == 1 ? m : n;
    const int order = side == 1 ? n : m;
    const int code = side * 8 + uplo * 4 + trans * 2 + unit;
    c.variant = VAR_DIRECT;
    c.MR = rows >= 16 ? 8 : 4;
    c.P = 1;
    c.minb = 1;
    TuneEntry e;
    bool force = false;
    if (lookup(BF_ROUTINE_DTRSM, code, order, &e)) {
        force = e.force;
        c.variant = e.variant == VAR_PACKED ? VAR_PACKED
                  : e.variant == VAR_TINY  ? VAR_TINY
                  : e.variant == VAR_BLOCKED ? VAR_BLOCKED : VAR_DIRECT;
        if (e.p0 == 4 || e.p0 == 8) c.MR = e.p0;
        c.P = e.p1 > 0 ? e.p1 : 0;
        if (e.p2 == 1 || e.p2 == 2) c.minb = e.p2;
    }
    if (c.variant == VAR_TINY && (m > 8 || n > 8)) c.variant = VAR_DIRECT;  // tiny: both orders <= 8
    if (c.variant == VAR_PACKED) {
        const int tpp = (rows + c.MR - 1) / c.MR;
        if (tpp > 256) {
            c.variant = VAR_DIRECT;  // a problem's rows do not fit one CTA
        } else {
            if (c.P <= 0) c.P = 128 / tpp > 0 ? 128 / tpp : 1;
            while (c.P > 1 && c.P * tpp > 256) c.P--;
            while (c.P > 1 && trsm_smem(c.P, order) > kSmemBudget) c.P--;
            if (trsm_smem(c.P, order) > kSmemBudget) c.variant = VAR_DIRECT;
        }
    }
    // the table is measured on 2 GiB batches: with far fewer independent rows than that, the
    // row kernels leave the GPU idle, and larger orders go to the blocked form (row-parallel
    // block solves + dgemm updates with 2-D parallelism)
    if (!force && order >= kTrsmBlockedMinOrder && batch * (long long)rows < kTrsmBlockedRows) c.variant = VAR_BLOCKED;
    if (c.variant == VAR_BLOCKED && order <= 32) c.variant = VAR_DIRECT;  // one block: nothing to hoist
    if (c.variant == VAR_DIRECT || c.variant == VAR_BLOCKED) c.P = 1;
    return c;
}

// Largest batch for which one problem per CTA beats the other forms, by order (measured
// crossovers against the team and lane forms: n = 16-27: ~900; 28-31: ~1,500; 32-39: ~1,800;
// 40-47: ~2,200; 48-63: ~3,000; 64-95: ~4,500; 96-191: ~5,000-6,000; 192: above the sweep's
// 7,281 (995 against 970 GFLOP/s); 256: above 9,728).  0: never (n < 16, where a CTA per
// problem idles most of its threads).
static long long cta_batch_limit(int n) {
    if (n < 16 || n > 256) return 0;
    if (n < 28) return 896;
    if (n < 32) return 1536;
    if (n < 40) return 1792;
    if (n < 48) return 2048;
    if (n < 64) return 3072;
    if (n < 96) return 4096;
    if (n < 192) return 6144;
    return 9728;
}

// Team size of the team form (lanes per problem) for batches between the CTA form's and the
// lane form's ranges, 0 for none.  A lane kernel on B problems runs B / 32 warps, each as
// long as one problem's whole instruction stream; while that leaves FP64 pipes idle, a team
// of t lanes per problem shortens the stream (the diagonal block's k loop is split t ways and
// the row blocks dealt out) at the price of more issue slots per problem.  Measured on GB300
// (GFLOP/s, lane -> team): n = 24 x 4,096: 153 -> 251 (t = 4); n = 32 x 6,144: 268 -> 440
// (t = 4); n = 32 x 14,592: 623 -> 746 (t = 2); n = 48 x 9,728: 457 -> 730 (t = 4).  An odd
// leading dimension slows the lane form more than the team form (single-word strips), so
// teams of 2 go on to batches half as large again (n = 32 x 19,456, lda 35: 601 -> 772).
static int team_size(int n, int lda, long long batch) {
    if (n < 12 || n > 64) return 0;
    long long u4, u2;  // largest batches for teams of 4 and of 2
    if (n < 16) {
        u4 = 0; u2 = 4096;
    } else if (n < 20) {
        u4 = 4096; u2 = 4096;
    } else if (n < 40) {
        u4 = 6144; u2 = 14592;
    } else if (n < 64) {
        u4 = 9728; u2 = 19456;
    } else {
        u4 = 9728; u2 = 14592;
    }
    if (n >= 20 && (lda & 1)) u2 = u2 * 3 / 2;
    if (batch <= u4) return 4;
    if (batch <= u2) return 2;
    return 0;
}

// The group form (a group of problems per CTA in shared memory, bf_potrf_group.cu, with the
// group size from its launch model) beats every other form on batches up to these sizes,
// measured on GB300 against the best of the lane, team, one-problem-per-CTA and blocked forms
// (GFLOP/s ratio at the bound / one step above it): n = 8: 12,288 (1.06 / 0.98); n = 16:
// 24,576 (1.02 / 0.88); n = 24: 65,536 and beyond (1.05); n = 32: 24,576 (1.00 / 0.98);
// n = 40: 16,384 (1.02 / 0.97); n = 48: 12,288 (1.05 / 0.99); n = 56: 12,288 (1.03 / 0.94);
// n = 64: 8,192 (1.15 / 0.97); n = 72: 12,288 (1.08); n = 80: 8,192 (1.04 / 0.93); n = 96:
// 1,216 (4,096: 0.98 against one problem per CTA); n = 112..143: 456 (n = 128: 1.25 / 0.94 at
// 532 problems); n = 144..192: 304 (at 384 problems 0.86-0.87).
static long long group_batch_limit(int n) {
    if (n < 4 || n > 192) return 0;
    if (n < 8) return 16384;
    if (n < 12) return 12288;
    if (n < 16) return 16384;
    if (n < 24) return 24576;
    if (n < 32) return 49152;
    if (n < 40) return 24576;
    if (n < 48) return 16384;
    if (n < 64) return 12288;
    if (n < 72) return 8192;
    if (n < 80) return 12288;
    if (n < 96) return 8192;
    if (n < 112) return 1216;
    if (n < 144) return 456;
    return 304;
}

PotrfConfig choose_potrf(int n, int lda, long long batch, bool allow_group) {
    // Table code 0 holds even leading dimensions, code 1 odd ones (an odd lda leaves
    // every other column's strips off the 16-byte boundary, which changes the best
    // lane kernel).
    const int code = lda & 1;
    PotrfConfig c;
    c.NB = 32;
    c.T = 64;
    // one problem per thread needs tens of thousands of problems to fill the GPU;
    // below that, larger orders go to the blocked sequence
    if (n <= 64 || batch >= 20000) {
        c.variant = VAR_DIRECT;
    } else {
        c.variant = VAR_BLOCKED;
    }
    // lane kernels: 8-row blocks (fewer requests per multiply-add, more registers)
    // once the k loops are long enough; sooner when strips are misaligned
    c.rows = (code ? n >= 16 : n >= 24) ? 8 : 4;
    c.unroll = 2;
    TuneEntry e;
    bool force = false;
    if (lookup(BF_ROUTINE_DPOTRF, code, n, &e)) {
        force = e.force;
        c.variant = e.variant;
        if (e.p0 > 0) c.T = e.p0;
        if (e.p1 > 0) c.NB = e.p1;
        if (e.p2 > 0) c.rows = e.p2;
        if (e.p3 > 0) c.unroll = e.p3;
    }
    // the table is measured on 2 GiB batches; a lane kernel on far fewer problems than
    // that leaves most of the GPU idle (one warp issues an FP64 instruction every 64 cycles):
    // small batches go to one problem per CTA, up to the crossover measured on GB300
    // (e.g. n = 128: 818 against 196 GFLOP/s at 608 problems), and the rest of the small
    // batches of larger orders to the blocked sequence
    long long cta_max = cta_batch_limit(n);
    int team = team_size(n, lda, batch);
    BatchRule r;
    if (lookup_rule(code, n, &r)) {  // measured bounds replace the built-in ones
        if (r.cta_max >= 0) cta_max = r.cta_max;
        if (r.team4_max >= 0 || r.team2_max >= 0) {  // the team bounds as a pair (< 0: none)
            team = (r.team4_max >= 0 && batch <= r.team4_max)   ? 4
                 : (r.team2_max >= 0 && batch <= r.team2_max) ? 2
                                                                : 0;
        }
    }
    // the group form first, up to its own measured bound; a batch rule (from the autotuner, which
    // times the one-problem-per-CTA, team and lane forms) decides among the forms above it
    if (allow_group && !force && batch <= group_batch_limit(n) && potrf_group_smem(n, 1) <= kGroupSmemMax) {
        c.variant = VAR_GROUP;
        c.T = 384;
        c.NB = 0;  // problems per group from the launch's time model
        c.rows = 4;
        c.unroll = 2;
        return c;
    }
    if (!force && batch <= cta_max) c.variant = VAR_CTA;
    if (!force && c.variant != VAR_CTA && team) {
        c.variant = VAR_TEAM;
        c.rows = team;  // the team size travels in the rows field (p2) below
        c.T = 64;
    }
    if (!force && c.variant != VAR_BLOCKED && c.variant != VAR_CTA && n > 64 && batch < 20000)
        c.variant = VAR_BLOCKED;
    // the table's threads per CTA are measured on 2 GiB batches: a lane kernel on a smaller
    // batch keeps at least two CTAs per SM (n = 48 x 9,728: 284 GFLOP/s with the table's 256
    // threads, 457 with 64)
    if (!force && c.variant == VAR_DIRECT) {
        const long long cap = batch / (2 * kSMs) / 32 * 32;
        if (c.T > cap) c.T = (int)(cap < 32 ? 32 : cap);
    }
    if (c.variant == VAR_GROUP) {  // p0: threads per CTA (256, 384 or 512), p1: groups per SM (1..4;
                                   // otherwise the group size from the launch's time model)
        c.T = (c.T == 384 || c.T == 512) ? c.T : 256;
        c.NB = (c.NB >= 1 && c.NB <= 4) ? c.NB : 0;
        c.rows = 4;
        c.unroll = 2;
        return c;
    }
    if (c.T < 32) c.T = 32;
    if (c.T > 256) c.T = 256;
    c.T = c.T / 32 * 32;
    if (c.NB < 4) c.NB = 4;
    if (c.variant == VAR_TEAM) c.tpp = c.rows == 2 ? 2 : 4;  // p2: lanes per problem
    c.rows = c.rows == 8 ? 8 : 4;
    c.unroll = c.unroll == 1 ? 1 : 2;
    if (c.variant == VAR_PACKED) {
        while (c.T > 32 && (size_t)(c.T + 1) * n * n * sizeof(double) > kSmemBudget) c.T -= 32;
        if ((size_t)(c.T + 1) * n * n * sizeof(double) > kSmemBudget) c.variant = VAR_DIRECT;
    }
    return c;
}

// dgetrf: the lane LU (VAR_DIRECT) or one problem per CTA (VAR_CTA, n <= 1024).  One problem
// per thread needs tens of thousands of problems; below the crossover measured per order, and
// for every order above 64 (where the lane LU's per-problem state outgrows its registers and
// L1), the CTA form is used.  A table entry (code 0) overrides, always with BF_TUNE_FORCE.
int choose_getrf(int n, long long batch) {
    TuneEntry e;
    if (lookup(BF_ROUTINE_DGETRF, 0, n, &e)) {
        const int v = e.variant == VAR_CTA ? VAR_CTA : e.variant == VAR_TEAM ? VAR_TEAM : VAR_DIRECT;
        if (e.force) {
            if (v == VAR_CTA && n > kGetrfCtaMaxN) return VAR_DIRECT;
            if (v == VAR_TEAM && n > kGetrfTeamMaxN) return VAR_DIRECT;
            return v;
        }
    }
    // four lanes per problem in shared memory from order 4 to 16, at every batch size, measured
    // on GB300 against the lane LU (GFLOP/s, 2 GiB batches): n = 4: 158 / 139, 8: 408 / 260,
    // 12: 567 / 325, 16: 627 / 448; at 4,096 problems 14 / 12, 76 / 39, 142 / 57, 207 / 79 (one
    // problem per CTA: 34 at n = 16).  Orders 2 and 3 keep the lane LU (a team of four lanes has
    // one or two rows to update).
    if (n >= 4 && n <= kGetrfTeamMaxN) return VAR_TEAM;
    if (n > kGetrfCtaMaxN || n < 16) return VAR_DIRECT;
    if (n > 64) return VAR_CTA;
    return batch <= getrf_cta_batch_limit(n) ? VAR_CTA : VAR_DIRECT;
}

}  // namespace bf

extern "C" int bf_tune_set(int routine, int code, int n_lo, int n_hi, int variant, int p0, int p1,
                           int p2, int p3) {
    if (routine < BF_ROUTINE_DGEMM || routine > BF_ROUTINE_DGETRF) return -1;
    if (n_lo > n_hi) return -3;
    const bool force = (variant & BF_TUNE_FORCE) != 0;
    variant &= ~BF_TUNE_FORCE;
    if (variant < 0 || variant > 6) return -5;
    std::lock_guard<std::mutex> lk(bf::g_mu);
    bf::g_table.push_back(bf::TuneEntry{routine, code, n_lo, n_hi, variant, p0, p1, p2, p3, force});
    return 0;
}

extern "C" void bf_tune_clear(void) {
    std::lock_guard<std::mutex> lk(bf::g_mu);
    bf::g_table.clear();
    bf::g_rules.clear();
}

extern "C" int bf_tune_set_batch_rule(int routine, int code, int n_lo, int n_hi, long long cta_max,
                                      long long team4_max, long long team2_max) {
    if (routine != BF_ROUTINE_DPOTRF) return -1;
    if (code < -1 || code > 1) return -2;
    if (n_lo > n_hi) return -3;
    std::lock_guard<std::mutex> lk(bf::g_mu);
    bf::g_rules.push_back(bf::BatchRule{code, n_lo, n_hi, cta_max, team4_max, team2_max});
    return 0;
}

extern "C" int bf_tune_query(int routine, int code, int m, int n, int k, long long batch, int* out) {
    if (!out) return -7;
    if (routine == BF_ROUTINE_DGEMM) {
        bf::GemmConfig c = bf::choose_gemm(code & 2, code & 1, m, n, k, m, batch);
        out[0] = c.variant; out[1] = c.TM; out[2] = c.TN; out[3] = c.KC; out[4] = c.P;
        return 0;
    }
    if (routine == BF_ROUTINE_DTRSM) {
        bf::TrsmConfig c = bf::choose_trsm((code >> 3) & 1, (code >> 2) & 1, (code >> 1) & 1, code & 1,
                                           m, n, batch);
        out[0] = c.variant; out[1] = c.MR; out[2] = c.P; out[3] = c.minb; out[4] = 0;
        return 0;
    }
    if (routine == BF_ROUTINE_DPOTRF) {
        bf::PotrfConfig c = bf::choose_potrf(n, code == 1 ? n + 1 : n, batch);
        out[0] = c.variant; out[1] = c.T; out[2] = c.NB;
        out[3] = c.variant == bf::VAR_TEAM ? c.tpp : c.rows; out[4] = c.unroll;
        return 0;
    }
    if (routine == BF_ROUTINE_DGETRF) {
        out[0] = bf::choose_getrf(n, batch); out[1] = out[2] = out[3] = out[4] = 0;
        return 0;
    }
    return -1;
}
