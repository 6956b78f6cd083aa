// Residual-periodogram kernels (the hot loop).  Included by the per-P
// instantiation units and by the batched persistent kernels.
//
// Paper: Section 5 (GPU parallelization) spends >90% of the time in the
// trigonometric averages of Eq. avrg1; the observation series is preloaded in
// fast shared memory and every thread evaluates the same averages for its own
// frequency.  Per trial frequency f (omega = 2 pi f, c = cos omega t',
// s = sin omega t', t' = t - t_c) the kernel accumulates the 2P+4 weighted sums
//     V_c[k] = <psi_k c>, V_s[k] = <psi_k s>   (k < P, psi = orthonormal base)
//     R_c = <r c>, R_s = <r s>                  (r = base residual)
//     CC = <c^2>, CS = <c s>                    (<s^2> = <1> - CC, Eq. idn)
// and solves the 2x2 Schur complement of the extended normal matrix (the
// incremental Cholesky extension of Section 3):
//     S = [[CC, CS], [CS, W - CC]] - V^T V,  z = 1/2 rho^T S^{-1} rho,
//     rho = (R_c, R_s).
//
// Decomposition: a CTA owns 32*F consecutive grid frequencies (lane l owns
// F consecutive ones) and its warps split the observations; records are
// staged tile by tile in shared memory with TMA bulk copies (double buffer,
// mbarrier completion, bounded waits).  Along the grid, cos/sin are advanced
// by the rotation e^{i 2 pi df t'} (a complex multiply), re-seeded for every
// point at each thread's first frequency from the exact fixed-point phase.
#pragma once

#include <algorithm>
#include <atomic>

#include "device_util.cuh"
#include "fredec_internal.cuh"

namespace fredec {

// Mixed path: FP32 block sums are flushed into FP32 running sums in shared
// memory (two-level summation; per warp for <r c>, <r s>, one array per CTA
// for the others: pgram_block_cs; on long series a third, compensated level
// for <r c>, <r s>: COMP below).  The random-phase residual sums <r c>, <r s> are
// flushed every 32 points: their FP32 rounding is amplified at low-z bins
// (dz/z = 2 drho/rho) and sets the z error.  The other 2P+2 sums are flushed
// every FLUSH_BLOCKS_ALL x 32 = 256 points.  Measured (largest z error against
// the FP64 kernel, floor 1e-3 of the highest peak; short series N < 700 against
// the oracle; kernel time on the N = 2000, 1e6-frequency residual periodogram):
//   all sums every 32 points: 1.8e-6, 5.5e-6; 1.99 ms
//   all sums every 64 points: 2.8e-6, 8e-6; 1.90 ms
//   <r c>, <r s> every 32, the rest every 128: 1.8e-6, 5.8e-6; 1.873 ms
//   <r c>, <r s> every 32, the rest every 256: 1.8e-6, 5.8e-6; 1.855 ms (N = 7e4: 5.4e-6, N = 1e5: 3.3e-6)
//   <r c>, <r s> every 32, the rest every 512: 2.9e-6, 5.8e-6; 1.847 ms
//   with COMP (below) at N = 1e5, p = 11 and N = 7e4, p = 7: 99th percentile
//   of the error over 290 bins 6.1e-6 -> 1.4e-6 and 4.8e-6 -> 1.1e-6, median
//   5.3e-7 -> 1.7e-7 and 4.8e-7 -> 1.8e-7 (the largest errors, 6.0e-6 and
//   5.5e-6, are at nearly degenerate bins that the float-float re-evaluation
//   serves, within their bound); short series unchanged (the FP32 cos/sin of
//   the first level sets their error)
constexpr int FLUSH_POINTS = 32;
constexpr int FLUSH_BLOCKS_ALL = 8;

// Long series: a warp's FP32 running residual sums take one flush per tile,
// and their rounding grows as sqrt(flushes).  The COMP kernels move them,
// every FLUSH_BLOCKS_ALL tiles, into CTA-level totals with Kahan compensation
// (kahan_add2), so that no FP32 running sum takes more than FLUSH_BLOCKS_ALL
// plain additions.  They serve series with more than COMP_MIN_FLUSHES tiles
// (N > 8192 with four warps).  On shorter series the running sums take few
// flushes and the plain kernels run: the compensated variant measured 1.7%
// slower on the N = 2000, p = 7, F = 10 kernel (a different schedule of the
// point loop, not the additions themselves: a plain-add variant of the same
// structure measured the same); on N = 1e5 it runs as fast as the plain one.
constexpr int COMP_MIN_FLUSHES = 64;

// A block of the tail of a launch is shared by at most TAIL_MAX_PARTS CTAs
// (the launcher gives every tail CTA at least tiles / (TAIL_MAX_PARTS - 1) of
// them).
constexpr int TAIL_MAX_PARTS = 9;
inline bool pgram_comp(int64_t N, int warps) { return (N + 32LL * warps - 1) / (32LL * warps) > COMP_MIN_FLUSHES; }

// Frequencies per thread of the two-set kernels (z and dz/df): mixed, two
// frequency pairs for bases of up to 7 columns (2 (2P+4) float2 sums a pair in
// registers: 218 registers at P = 7; 0.643 of the FP32 peak against 0.562
// with one pair) and one pair for wider bases (the second pair, reached by
// the two-step rotation, carries rounding that the t'-weighted dz/df sums
// amplify: 1.2e-4 at P = 11 on a 300-point series, above the 1e-4 bar);
// FP64, one frequency.
__host__ __device__ constexpr int grad_fpt_mixed(int p) { return p <= 7 ? 4 : 2; }
constexpr int GRAD_FPT_FP64 = 1;

struct PgramParams {
    const SeriesDesc *desc;
    const SeriesState *state;
    const unsigned char *rec;   // record buffer base (series offsets in desc)
    double *z;                  // output base (series offsets in desc)
    double *z_mirror;           // optional second destination of z (same offsets)
    double *coef;               // optional (a_j, b_j) output, same offsets * 2
    double flag_tau;            // mixed: re-evaluation threshold (< 0: never)
    int64_t *flag_list;         // mixed: global z indices of bins to re-evaluate (float-float)
    int32_t *flag_count;
    int64_t flag_cap;           // entries of flag_list (a full list records FREDEC_EINVAL in err)
    int32_t *err;               // FREDEC_ETIMEOUT on a bounded-wait timeout
    double *dzdf;               // two-set kernels: dz/df per bin (same offsets as z)
    const double *wt_sum;       // two-set kernels: <t'> = sum of the records' w t' (one series)
    int seed_mode;              // mixed: 0 = table-driven FP32 sin/cos seed, 1 = MUFU __sincosf
    int comp;                   // mixed: compensated residual totals (pgram_comp)
};

// Mixed, one series: the last part-filled wave of blocks split over a wave of
// CTAs (pgram_tail_kernel).  A separate kernel argument: a larger PgramParams
// changed the main kernel's register allocation and slowed it by 1.5%.
struct TailParams {
    float2 *part;     // partial sums, 2 slots per tail CTA
    int32_t *cnt;     // tiles done per tail block (zero at launch)
    int gcap;         // tail CTAs the two arrays hold
    int n_points;     // the series' N (host copy)
    int64_t b0;       // first block of the tail (set by the launcher)
};

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Shared memory of a CTA: [mbarriers | seed table | 2 record tiles | warp
// partial sums].  The seed table sits at a fixed offset (independent of P and
// F) so that persistent kernels switching between (P, F) fill it once.
constexpr size_t OFF_TABLE = 128;
constexpr size_t OFF_TILES_BASE = OFF_TABLE + sizeof(SeedTable);
static_assert(sizeof(SeedTableF) <= sizeof(SeedTable), "both seed tables fit the table region");

// Shared memory of the FP64 kernels (pgram_block).  NSET = 2: every record
// carries a second set of weighted values, the t'-weighted ones, and the
// kernel accumulates 2 (2P+4) sums per frequency.
template <int PREC, int P, int F, int NSET = 1>
struct PgramLayout {
    static_assert(PREC == FREDEC_FP64, "the mixed kernels use PgramCsLayout");
    static constexpr int Q = NSET * (2 * P + 4);
    static constexpr int RB = rec_bytes(P, PREC, NSET);
    // records per tile: TILE_POINTS, or fewer for records above 64 bytes so
    // that the two tiles stay within 16 KB
    static constexpr int TP = RB <= 64 ? TILE_POINTS : (8192 / RB) / 8 * 8;
    static constexpr size_t TILE_BYTES = (size_t)TP * RB;
    static constexpr size_t OFF_TILES = OFF_TILES_BASE;
    static constexpr size_t OFF_RED = OFF_TILES + 2 * TILE_BYTES;
    // warp running sums: Q x F doubles per lane
    static constexpr int RED_PER_WARP = Q * F * 32;
    static __host__ __device__ size_t red_bytes(int nw) { return (size_t)nw * RED_PER_WARP * sizeof(double); }
    static __host__ __device__ size_t smem_bytes(int nw) { return OFF_RED + red_bytes(nw); }
};

// Per-frequency 2x2 solve in FP64.  Returns z; writes the joint-fit
// coefficients of cos/sin (a, b) and the smaller pivot ratio (1 = orthogonal
// to the base, 0 = dependent).
__device__ __forceinline__ double solve2(double CC, double CS, double SS, double vcc, double vcs,
                                         double vss, double Rc, double Rs, double *pa, double *pb,
                                         double *pr) {
    const double S11 = CC - vcc, S12 = CS - vcs, S22 = SS - vss;
    const bool kc = S11 > DROP2 * CC && CC > 0.0;
    double a = 0.0, b = 0.0, z = 0.0, r1 = kc ? S11 / CC : 0.0, r2;
    if (kc) {
        const double l21 = S12 / S11;
        const double S22p = S22 - S12 * l21;
        r2 = SS > 0.0 ? S22p / SS : 0.0;
        if (S22p > DROP2 * SS && SS > 0.0) {
            const double y1 = Rc * rsqrt(S11);
            const double y2 = (Rs - l21 * Rc) * rsqrt(S22p);
            z = 0.5 * (y1 * y1 + y2 * y2);
            b = (Rs - l21 * Rc) / S22p;
            a = (Rc - S12 * b) / S11;
        } else {
            z = 0.5 * Rc * Rc / S11;
            a = Rc / S11;
        }
    } else {
        r2 = SS > 0.0 ? S22 / SS : 0.0;
        if (S22 > DROP2 * SS && SS > 0.0) {
            z = 0.5 * Rs * Rs / S22;
            b = Rs / S22;
        }
    }
    *pa = a;
    *pb = b;
    *pr = fmin(fmin(r1, r2), fmin(CC, SS) / (CC + SS));
    return z;
}

// The same 2x2 solve with one reciprocal, for well-conditioned bins:
// theta = S^{-1} rho by the adjugate, z = 1/2 rho^T theta.  Returns false
// (and leaves the outputs alone) when a pivot ratio is below tau, i.e. when
// the bin must be re-evaluated with FP64-grade sums; no divisions are spent on the test.
__device__ __forceinline__ bool solve2_fast(double CC, double CS, double SS, double vcc, double vcs, double vss,
                                            double Rc, double Rs, double tau, double *pz, double *pa, double *pb) {
    const double S11 = CC - vcc, S12 = CS - vcs, S22 = SS - vss;
    const double det = fma(S11, S22, -S12 * S12);
    // pivot ratios S11/CC and (det/S11)/SS, and the column-norm balance
    const bool ok = S11 >= tau * CC && det >= tau * S11 * SS && CC >= tau * (CC + SS) && SS >= tau * (CC + SS) &&
                    det > 0.0;
    if (!ok) return false;
    const double inv = 1.0 / det;
    const double a = (S22 * Rc - S12 * Rs) * inv;
    const double b = (S11 * Rs - S12 * Rc) * inv;
    *pa = a;
    *pb = b;
    *pz = 0.5 * fma(a, Rc, b * Rs);
    return true;
}

// dz/df of the residual periodogram at one trial frequency from its two sets
// of sums and its joint-fit coefficients (a, b) of c and s.  By the envelope
// theorem (the linear parameters are optimal) dz/df = <r_f dmu/df> with
// dmu/df = 2 pi t' (b c - a s) and r_f the residual of the joint fit,
// r_f = r - a c~ - b s~, c~ = c - sum_k <psi_k c> psi_k (the trial columns
// projected off the orthonormal base; Section 3, the derivatives of Eq. Hn
// through the t-weighted averages of Eq. avrg1).  S0: <psi_k c>, <psi_k s>,
// <r c>, <r s>, <c^2>, <c s>; S1: the same sums weighted by t';
// wt = <t'>, so that <t' s^2> = <t'> - <t' c^2>.
template <int P>
__device__ __forceinline__ double dz_df(const double *S0, const double *S1, double wt, double a, double b) {
    double cc = 0.0, sc = 0.0, cs = 0.0, ss = 0.0;   // sum_k <psi_k x> <psi_k t' y>
#pragma unroll
    for (int q = 0; q < P; ++q) {
        cc = fma(S0[q], S1[q], cc);
        sc = fma(S0[P + q], S1[q], sc);
        cs = fma(S0[q], S1[P + q], cs);
        ss = fma(S0[P + q], S1[P + q], ss);
    }
    const double tcc = S1[2 * P + 2], tcs = S1[2 * P + 3], tss = wt - tcc;
    const double rtc = S1[2 * P] - a * (tcc - cc) - b * (tcs - sc);   // <r_f t' c>
    const double rts = S1[2 * P + 1] - a * (tcs - cs) - b * (tss - ss);   // <r_f t' s>
    return TWO_PI_D * (b * rtc - a * rts);
}

// ---------------------------------------------------------------------------
// Inner loops: one observation record against this thread's F frequencies.

// One observation record, ready for the F-step loop: the seed cos/sin at the
// thread's first frequency, scaled by s = sqrt(w), the one- and two-step
// rotations, and the values that multiply the scaled cos/sin: s r, s psi_k
// (w[0] = s itself).  With NSET = 2 the second set holds t' (w[1], the
// factor of the t'-weighted (s c)^2 and (s c)(s s) sums), s r t', s psi_k t'.
template <int P, int NSET = 1>
struct MixedPoint {
    float c, s, cr, sr, c2, s2;
    float w[NSET], wr[NSET];
    float u[NSET][4 * ((P + 2 + 3) / 4) - 2];
};

// The record's rotations and the values that multiply the scaled cos/sin
// (everything but the seed).
template <int P, int NSET = 1>
__device__ __forceinline__ void mixed_load_values(const uint4 *__restrict__ r4, MixedPoint<P, NSET> &pt) {
    constexpr int C4 = (P + 2 + 3) / 4;   // float4s of one set [s, s r, s psi_k]
    const float4 m = *reinterpret_cast<const float4 *>(r4 + 1);
#pragma unroll
    for (int g = 0; g < NSET; ++g) {
        float v[4 * C4];
#pragma unroll
        for (int q4 = 0; q4 < C4; ++q4) {
            const float4 x = reinterpret_cast<const float4 *>(r4 + 2 + g * C4)[q4];
            v[4 * q4] = x.x;
            v[4 * q4 + 1] = x.y;
            v[4 * q4 + 2] = x.z;
            v[4 * q4 + 3] = x.w;
        }
        pt.w[g] = v[0];
        pt.wr[g] = v[1];
#pragma unroll
        for (int q = 0; q < 4 * C4 - 2; ++q) pt.u[g][q] = v[2 + q];
    }
    pt.cr = m.x;
    pt.sr = m.y;
    pt.c2 = m.z;
    pt.s2 = m.w;
}

template <int P, int SEED, int NSET = 1>
__device__ __forceinline__ void mixed_load(const uint4 *__restrict__ r4, const SeedTableF &tab, uint32_t j0,
                                           MixedPoint<P, NSET> &pt) {
    mixed_load_values<P, NSET>(r4, pt);
    const uint4 h = r4[0];
    const uint64_t A = ((uint64_t)h.y << 32) | h.x;
    const uint64_t B = ((uint64_t)h.w << 32) | h.z;
    const uint64_t ph = A + (uint64_t)j0 * B;          // exact phase (turns * 2^64) at f_{j0}
    if constexpr (SEED == 0) {
        seed_from_table_f(tab, (uint32_t)(ph >> 32), &pt.s, &pt.c);
    } else {
        const float ang = (float)(int32_t)(ph >> 32) * TWO_PI_OVER_2_32;
        __sincosf(ang, &pt.s, &pt.c);
    }
    pt.c *= pt.w[0];   // the point's cos/sin scaled by s = sqrt(w)
    pt.s *= pt.w[0];
}

// Mixed accumulators: the F frequencies of a thread in pairs (k, k+1), every
// sum of a pair in one float2 register pair, so that one packed FP32
// instruction (FFMA2: two FMAs of one warp instruction) updates the sums of
// both frequencies.  With F odd the last pair's second half is not used.
template <int P, int F, int NSET = 1>
struct MixedAcc {
    static constexpr int Q = NSET * (2 * P + 4);
    static constexpr int NPC = (F + 1) / 2;
    float2 a[NPC][Q];
};

// Compensated (Kahan) addition of v to the running sum m with compensation
// c, two lanes at a time: c holds the low-order part lost by the earlier
// additions, so that m - c carries the total to within a few roundings
// whatever the number of additions.  a - b is formed as fma(b, -1, a), one
// rounding.
__device__ __forceinline__ void kahan_add2(float2 &m, float2 &c, float2 v) {
    const float2 neg1 = make_float2(-1.0f, -1.0f);
    const float2 y = __ffma2_rn(c, neg1, v);
    const float2 t = __fadd2_rn(m, y);
    c = __ffma2_rn(y, neg1, __ffma2_rn(m, neg1, t));
    m = t;
}

// F consecutive frequencies of one point, two at a time.  The pair starts at
// (f_{j0}, f_{j0+1}) (the seed and one step of the rotation e^{i theta},
// theta = 2 pi df t') and advances by e^{2 i theta} (from the record, rounded
// once from FP64, so that the recurrence drifts by the rounding of one
// constant per step); with the cos/sin scaled by s = sqrt(w), per pair the
// 2P+4 sums
//     <psi_k c>, <psi_k s>, <r c>, <r s>, <c^2>, <c s>
// take one packed FMA each ((s psi_k)(s c), ..., (s c)(s c), (s c)(s s)):
// (2P + 8) packed instructions per two frequencies, the rotation included.
// The second set's <t' c^2>, <t' c s> take one packed multiply more (t' s c).
template <int P, int F, int NSET = 1>
__device__ __forceinline__ void mixed_accumulate(const MixedPoint<P, NSET> &pt, MixedAcc<P, F, NSET> &A) {
    constexpr int NPC = MixedAcc<P, F, NSET>::NPC, Q0 = 2 * P + 4;
    float2 c = make_float2(pt.c, fmaf(pt.c, pt.cr, -pt.s * pt.sr));
    float2 s = make_float2(pt.s, fmaf(pt.s, pt.cr, pt.c * pt.sr));
    const float2 cc = make_float2(pt.c2, pt.c2), ss = make_float2(pt.s2, pt.s2), nss = make_float2(-pt.s2, -pt.s2);
#pragma unroll
    for (int kk = 0; kk < NPC; ++kk) {
#pragma unroll
        for (int g = 0; g < NSET; ++g) {   // the set's sums; the same (c, s) for both sets
            float2 *a = A.a[kk] + g * Q0;
            if ((F & 1) && kk == NPC - 1) {   // the odd last frequency on its own
                const float wc = g == 0 ? c.x : pt.w[g] * c.x;
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    a[q].x = fmaf(pt.u[g][q], c.x, a[q].x);
                    a[P + q].x = fmaf(pt.u[g][q], s.x, a[P + q].x);
                }
                a[2 * P].x = fmaf(pt.wr[g], c.x, a[2 * P].x);
                a[2 * P + 1].x = fmaf(pt.wr[g], s.x, a[2 * P + 1].x);
                a[2 * P + 2].x = fmaf(wc, c.x, a[2 * P + 2].x);
                a[2 * P + 3].x = fmaf(wc, s.x, a[2 * P + 3].x);
            } else {
#pragma unroll
                for (int q = 0; q < P; ++q) {
                    const float2 uu = make_float2(pt.u[g][q], pt.u[g][q]);
                    a[q] = __ffma2_rn(uu, c, a[q]);
                    a[P + q] = __ffma2_rn(uu, s, a[P + q]);
                }
                const float2 wr2 = make_float2(pt.wr[g], pt.wr[g]), w2 = make_float2(pt.w[g], pt.w[g]);
                a[2 * P] = __ffma2_rn(wr2, c, a[2 * P]);
                a[2 * P + 1] = __ffma2_rn(wr2, s, a[2 * P + 1]);
                const float2 wc = g == 0 ? c : __fmul2_rn(w2, c);
                a[2 * P + 2] = __ffma2_rn(wc, c, a[2 * P + 2]);
                a[2 * P + 3] = __ffma2_rn(wc, s, a[2 * P + 3]);
            }
        }
        if (kk + 1 < NPC) {
            const float2 cn = __ffma2_rn(s, nss, __fmul2_rn(c, cc));
            s = __ffma2_rn(c, ss, __fmul2_rn(s, cc));
            c = cn;
        }
    }
}

// m >= 1 consecutive points of this warp (records p, p + stride, ...),
// software-pipelined: the next point's record and seed are fetched while the
// current point's F-step loop runs (two alternating point buffers).  The loop
// is over pairs with no per-point branch; an even run ends by re-fetching its
// last point, which is not accumulated.
template <int P, int F, int SEED, int NSET = 1>
__device__ __forceinline__ void mixed_run(const unsigned char *p, size_t stride, int m, const SeedTableF &tab,
                                          uint32_t j0, MixedAcc<P, F, NSET> &acc) {
    auto rec = [&](int i) { return reinterpret_cast<const uint4 *>(p + (size_t)i * stride); };
    if constexpr (NSET == 2 && P >= 23) {
        // two-set kernels of the widest bases: 2 (2P+4) float2 sums leave no
        // room for a second point in flight; one point at a time spills less
        // (P = 25: 1984 -> 1148 bytes) and runs faster (z and dz/df, N = 2000,
        // 1e6 frequencies: P = 25 27.7 -> 15.0 ms, P = 23 11.74 -> 11.36 ms;
        // narrower bases keep the two points: one at a time lost 1% at P = 21
        // and 3-11% at P = 9-19)
        for (int j = 0; j < m; ++j) {
            MixedPoint<P, NSET> pc;
            mixed_load<P, SEED, NSET>(rec(j), tab, j0, pc);
            mixed_accumulate<P, F, NSET>(pc, acc);
        }
        return;
    }
    MixedPoint<P, NSET> pa, pb;
    mixed_load<P, SEED, NSET>(rec(0), tab, j0, pa);
    int j = 0;
    for (; j + 2 <= m; j += 2) {
        mixed_load<P, SEED, NSET>(rec(j + 1), tab, j0, pb);
        mixed_accumulate<P, F, NSET>(pa, acc);
        mixed_load<P, SEED, NSET>(rec(min(j + 2, m - 1)), tab, j0, pa);
        mixed_accumulate<P, F, NSET>(pb, acc);
    }
    if (j < m) mixed_accumulate<P, F, NSET>(pa, acc);
}

template <int P, int F, int NSET = 1>
__device__ __forceinline__ void fp64_point(const double2 *__restrict__ r2, const SeedTable &tab, uint32_t j0,
                                           double (&acc)[F][NSET * (2 * P + 4)]) {
    constexpr int C2 = (P + 1) / 2, Q0 = 2 * P + 4;
    const ulonglong2 h = *reinterpret_cast<const ulonglong2 *>(r2);
    const double2 rot = r2[1];
    double w[NSET], wr[NSET], u[NSET][2 * C2];
    const double2 ww = r2[2];
    w[0] = ww.x;
    wr[0] = ww.y;
#pragma unroll
    for (int q2 = 0; q2 < C2; ++q2) {
        const double2 v = r2[3 + q2];
        u[0][2 * q2] = v.x;
        u[0][2 * q2 + 1] = v.y;
    }
    if constexpr (NSET == 2) {   // the t'-weighted set after the first
        const double2 w2 = r2[3 + C2];
        w[1] = w2.x;
        wr[1] = w2.y;
#pragma unroll
        for (int q2 = 0; q2 < C2; ++q2) {
            const double2 v = r2[4 + C2 + q2];
            u[1][2 * q2] = v.x;
            u[1][2 * q2 + 1] = v.y;
        }
    }
    const uint64_t ph = h.x + (uint64_t)j0 * h.y;
    double s, c;
    seed_from_table(tab, ph, &s, &c);
    const double cr = rot.x, sr = rot.y;
#pragma unroll
    for (int k = 0; k < F; ++k) {
#pragma unroll
        for (int g = 0; g < NSET; ++g) {
            double *a = acc[k] + g * Q0;
            const double wc = w[g] * c;
#pragma unroll
            for (int q = 0; q < P; ++q) {
                a[q] = fma(u[g][q], c, a[q]);
                a[P + q] = fma(u[g][q], s, a[P + q]);
            }
            a[2 * P] = fma(wr[g], c, a[2 * P]);
            a[2 * P + 1] = fma(wr[g], s, a[2 * P + 1]);
            a[2 * P + 2] = fma(wc, c, a[2 * P + 2]);
            a[2 * P + 3] = fma(wc, s, a[2 * P + 3]);
        }
        if (k + 1 < F) {
            const double cn = fma(c, cr, -s * sr);
            s = fma(s, cr, c * sr);
            c = cn;
        }
    }
}

// ---------------------------------------------------------------------------
// One CTA-block of 32*F frequencies of one series, FP64 (the FP64 grid,
// two-set and batched kernels): each lane's F x Q sums in FP64 registers over
// all points, then the warps' running sums in shared memory (red) combined
// per frequency.  use0/use1: per-buffer mbarrier phase counters, identical in
// all threads.
template <int PREC, int P, int F, int NSET = 1>
__device__ __forceinline__ void pgram_block(const PgramParams &prm, const SeriesDesc &d, const SeriesState &st,
                                            int64_t blk, unsigned char *smem, uint32_t &use0, uint32_t &use1) {
    static_assert(PREC == FREDEC_FP64, "the mixed kernels use pgram_block_cs");
    using L = PgramLayout<PREC, P, F, NSET>;
    constexpr int Q = L::Q;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    unsigned char *tiles = smem + L::OFF_TILES;
    double *red = reinterpret_cast<double *>(smem + L::OFF_RED);
    const SeedTable &tab = *reinterpret_cast<const SeedTable *>(smem + OFF_TABLE);

    const int N = d.N;
    const int64_t jblock = blk * 32 * F;
    const uint32_t j0 = (uint32_t)(jblock + lane * F);
    const unsigned char *src = prm.rec + d.rec_off;
    const int ntiles = (N + L::TP - 1) / L::TP;

    __syncthreads();   // previous block's epilogue is done with red / tiles
    if (tid == 0) {
        for (int k = 0; k < 2 && k < ntiles; ++k) {
            const unsigned n = (unsigned)min(L::TP, N - k * L::TP);
            mbar_arrive_expect_tx(&bars[k], n * L::RB);
            bulk_g2s(tiles + k * L::TILE_BYTES, src + (size_t)k * L::TILE_BYTES, n * L::RB, &bars[k]);
        }
    }

    double acc[F][Q];
#pragma unroll
    for (int k = 0; k < F; ++k)
#pragma unroll
        for (int q = 0; q < Q; ++q) acc[k][q] = 0.0;

    for (int tile = 0; tile < ntiles; ++tile) {
        const int b = tile & 1;
        const uint32_t par = b ? (use1++ & 1u) : (use0++ & 1u);
        if (!mbar_wait_bounded(&bars[b], par)) {
            if (lane == 0) atomicExch(prm.err, FREDEC_ETIMEOUT);
        }
        const int n = min(L::TP, N - tile * L::TP);
        const unsigned char *tb = tiles + b * L::TILE_BYTES;
        for (int i = warp; i < n; i += nw)
            fp64_point<P, F, NSET>(reinterpret_cast<const double2 *>(tb + (size_t)i * L::RB), tab, j0, acc);
        __syncthreads();   // all warps are done with buffer b
        if (tid == 0 && tile + 2 < ntiles) {
            const unsigned nn = (unsigned)min(L::TP, N - (tile + 2) * L::TP);
            mbar_arrive_expect_tx(&bars[b], nn * L::RB);
            bulk_g2s(tiles + b * L::TILE_BYTES, src + (size_t)(tile + 2) * L::TILE_BYTES, nn * L::RB, &bars[b]);
        }
    }
    double *mine = red + (size_t)warp * L::RED_PER_WARP;
#pragma unroll
    for (int k = 0; k < F; ++k)
#pragma unroll
        for (int q = 0; q < Q; ++q) mine[(q * F + k) * 32 + lane] = acc[k][q];
    __syncthreads();

    // Epilogue: combine the warps' sums and solve per frequency.
    const double W = st.W;
    const int64_t nf = d.nf;
    for (int fs = tid; fs < 32 * F; fs += blockDim.x) {
        const int k = fs >> 5, ln = fs & 31;
        const int64_t j = jblock + (int64_t)ln * F + k;
        if (j >= nf) continue;
        double S[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            double sq = 0.0;
            for (int w = 0; w < nw; ++w) sq += red[((size_t)w * Q + q) * F * 32 + k * 32 + ln];
            S[q] = sq;
        }
        double vcc = 0.0, vcs = 0.0, vss = 0.0;
#pragma unroll
        for (int q = 0; q < P; ++q) {
            vcc = fma(S[q], S[q], vcc);
            vcs = fma(S[q], S[P + q], vcs);
            vss = fma(S[P + q], S[P + q], vss);
        }
        const double CC = S[2 * P + 2], CS = S[2 * P + 3];
        double a, bb, ratio;
        const double zz = solve2(CC, CS, W - CC, vcc, vcs, vss, S[2 * P], S[2 * P + 1], &a, &bb, &ratio);
        if constexpr (NSET == 2) prm.dzdf[d.z_off + j] = dz_df<P>(S, S + 2 * P + 4, *prm.wt_sum, a, bb);
        prm.z[d.z_off + j] = zz;
        if (prm.coef) {
            prm.coef[2 * (d.z_off + j)] = a;
            prm.coef[2 * (d.z_off + j) + 1] = bb;
        }
    }
}

template <int PREC>
__device__ __forceinline__ void pgram_cta_init(unsigned char *smem) {
    if (threadIdx.x == 0) {
        uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    if constexpr (PREC == FREDEC_FP64)
        fill_seed_table(*reinterpret_cast<SeedTable *>(smem + OFF_TABLE));
    else
        fill_seed_table_f(*reinterpret_cast<SeedTableF *>(smem + OFF_TABLE));
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Mixed kernels (single-series, two-set and batched) with CTA-level
// second-level sums.  The 2P+2 slow sums (<psi_k c>, <psi_k s>, <c^2>,
// <c s>) of all warps go into ONE running array per CTA: every
// FLUSH_BLOCKS_ALL tiles (256 points per warp), at the tile barrier, the
// warps add their register sums in nw steps separated by CTA barriers, warp
// w adding in step s the slow sums b with b % nw == (w + s) % nw, so that no
// two warps touch the same entries in a step and the order of the additions
// is fixed (deterministic).  The residual sums <r c>, <r s> keep per-warp
// running sums, flushed every FLUSH_POINTS points.  This
// takes the warps' running sums from (2P+4) nw to 2P+2 + 2 nw rows of
// 32 F floats (92 -> 31 KB at P = 7, F = 10, four warps; with two warps a
// CTA four CTAs fit an SM, where per-warp sums allowed three).  A tile holds
// 32 points per warp: one run of the software-pipelined point loop per flush
// of the residual sums (measured at P = 7, F = 10, four warps: 64-point tiles
// 1.749 ms, 96 1.724 ms, 128 1.690 ms, against 1.704 ms with per-warp
// running sums).  With NSET = 2 (z and dz/df) both sets are split the same
// way: 2 (2P+2) slow sums, 4 residual sums.
template <int P, int F, int NSET = 1, bool COMP = false>
struct PgramCsLayout {
    static constexpr int Q0 = 2 * P + 4, Q = NSET * Q0, QS = NSET * (2 * P + 2), NPC = (F + 1) / 2;
    static constexpr int RB = rec_bytes(P, FREDEC_MIXED, NSET);
    static __host__ __device__ int tile_points(int nw) { return 32 * nw; }
    static __host__ __device__ size_t tile_bytes(int nw) { return (size_t)tile_points(nw) * RB; }
    static constexpr size_t OFF_TILES = OFF_TILES_BASE;
    // two record tiles; also z of the CTA's 32 F frequencies (mirror kernels)
    static __host__ __device__ size_t rr_off(int nw) {
        const size_t t = 2 * tile_bytes(nw), zs = 32 * F * sizeof(double);
        return align_up(OFF_TILES + (t > zs ? t : zs), 16);
    }
    static constexpr int QR = 2 * NSET;   // residual sums
    static constexpr size_t RR_PER_WARP = (size_t)QR * NPC * 32;   // float2 entries
    static __host__ __device__ size_t rs_off(int nw) { return rr_off(nw) + (size_t)nw * RR_PER_WARP * sizeof(float2); }
    // CTA array: QS slow-sum rows, then with COMP QR residual-total rows and
    // QR rows of their compensation terms; a row is NPC * 32 float2 entries
    static constexpr size_t RS_ENTRIES = (size_t)(QS + (COMP ? 2 * QR : 0)) * NPC * 32;
    static __host__ __device__ size_t smem_bytes(int nw) { return rs_off(nw) + RS_ENTRIES * sizeof(float2); }
    // the sum index q of slow sum b and of residual sum j
    static __host__ __device__ constexpr int slow_q(int b) {
        return (b / (2 * P + 2)) * Q0 + (b % (2 * P + 2) < 2 * P ? b % (2 * P + 2) : b % (2 * P + 2) + 2);
    }
    static __host__ __device__ constexpr int fast_q(int j) { return (j / 2) * Q0 + 2 * P + j % 2; }
};

// Tail of a single-series launch (pgram_tail_kernel): the blocks from
// TailParams::b0 on are cut into their tiles, U = blocks x tiles units in all,
// and tail CTA g of G takes the units [u0(g), u0(g + 1)), u0(g) = g U / G, in
// (block, tile) order: every CTA has the same work, so the last wave of a
// launch ends together instead of leaving SMs idle.  A block that CTAs share
// is completed by the CTA whose tiles complete its count; no CTA waits for
// another.
__host__ __device__ inline int64_t tail_u0(int64_t g, int64_t U, int64_t G) { return g * U / G; }

// After a part of block blk (ntl of its ntiles tiles) has been summed: write
// this CTA's partial sums, the slow-sum rows and the residual rows (the warps'
// running sums added in warp order; with COMP total minus compensation), to
// its slot (2 g for the first block of its range, 2 g + 1 for the last), and
// count the tiles.  The CTA that completes the count adds the parts in the
// order of the CTAs that hold them (deterministic) into its own shared-memory
// sums, laid out as the epilogue reads them, and returns true.
template <int P, int F, int NSET, bool COMP>
__device__ bool tail_exchange(const PgramParams &prm, const TailParams &tp, int64_t blk, int ntiles, int ntl, float2 *rr,
                              float2 *rs) {
    using L = PgramCsLayout<P, F, NSET, COMP>;
    constexpr int SE = L::QS * L::NPC * 32, RE = L::QR * L::NPC * 32, PE = SE + RE;
    __shared__ int s_last, s_nslot, s_slot[TAIL_MAX_PARTS];
    const int tid = threadIdx.x, nw = blockDim.x >> 5;
    const int64_t G = gridDim.x, g = blockIdx.x;
    const int64_t nblocks = (prm.desc[0].nf + 32 * F - 1) / (32 * F);
    const int64_t U = (nblocks - tp.b0) * ntiles, ub = (blk - tp.b0) * ntiles, ue = ub + ntiles;
    const int64_t mine = 2 * g + (tail_u0(g, U, G) < ub ? 1 : 0);
    float2 *dst = tp.part + (size_t)mine * PE;
    for (int e = tid; e < SE; e += blockDim.x) dst[e] = rs[e];
    for (int e = tid; e < RE; e += blockDim.x) {
        float2 v;
        if constexpr (COMP) {
            const float2 m = rs[SE + e], c = rs[SE + RE + e];
            v = make_float2(m.x - c.x, m.y - c.y);
        } else {
            v = make_float2(0.0f, 0.0f);
            for (int w = 0; w < nw; ++w) v = __fadd2_rn(v, rr[(size_t)w * L::RR_PER_WARP + e]);
        }
        dst[SE + e] = v;
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();   // the partial before the count
        const int old = atomicAdd(tp.cnt + (blk - tp.b0), ntl);
        s_last = old + ntl == ntiles;
        if (s_last) {
            __threadfence();   // the other parts after the count
            int64_t h = ub * G / U;   // the CTA holding the block's first unit
            while (h + 1 < G && tail_u0(h + 1, U, G) <= ub) ++h;
            while (h > 0 && tail_u0(h, U, G) > ub) --h;
            int n = 0;
            for (; h < G && tail_u0(h, U, G) < ue && n < TAIL_MAX_PARTS; ++h)
                s_slot[n++] = (int)(2 * h + (tail_u0(h, U, G) < ub ? 1 : 0));
            s_nslot = n;
        }
    }
    __syncthreads();
    if (!s_last) return false;
    const int n = s_nslot;
    for (int e = tid; e < PE; e += blockDim.x) {
        float2 v = make_float2(0.0f, 0.0f);
        for (int i = 0; i < n; ++i) v = __fadd2_rn(v, __ldcg(tp.part + (size_t)s_slot[i] * PE + e));
        if (e < SE) {
            rs[e] = v;
        } else if constexpr (COMP) {
            rs[e] = v;
            rs[RE + e] = make_float2(0.0f, 0.0f);
        } else {
            rr[e - SE] = v;   // warp 0's running sums; the other warps' are zero
            for (int w = 1; w < nw; ++w) rr[(size_t)w * L::RR_PER_WARP + e - SE] = make_float2(0.0f, 0.0f);
        }
    }
    __syncthreads();
    return true;
}

// MIRROR: z also goes to prm.z_mirror (page-locked host memory), staged in
// shared memory so that the host-memory stores are contiguous.  The mirror
// kernels are instantiated in translation units of their own
// (pgram_mirror_*.cu): with them in the same module the kernels without a
// mirror measured 1.5% slower, identical code notwithstanding.
template <int P, int F, bool MIRROR, int NSET = 1, bool COMP = false, bool TAIL = false>
__device__ __forceinline__ void pgram_block_cs(const PgramParams &prm, const SeriesDesc &d, const SeriesState &st,
                                               int64_t blk, unsigned char *smem, uint32_t &use0, uint32_t &use1,
                                               int t_begin = 0, int t_end = 0, const TailParams *tp = nullptr) {
    static_assert(NSET == 1 || !MIRROR, "the two-set kernels write z to device memory only");
    using L = PgramCsLayout<P, F, NSET, COMP>;
    constexpr int Q = L::Q, QS = L::QS, NPC = L::NPC;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    unsigned char *tiles = smem + L::OFF_TILES;
    float2 *rr = reinterpret_cast<float2 *>(smem + L::rr_off(nw));
    float2 *rs = reinterpret_cast<float2 *>(smem + L::rs_off(nw));
    const SeedTableF &tabf = *reinterpret_cast<const SeedTableF *>(smem + OFF_TABLE);

    const int N = d.N;
    const int64_t jblock = blk * 32 * F;
    const uint32_t j0 = (uint32_t)(jblock + lane * F);
    const unsigned char *src = prm.rec + d.rec_off;
    const int TP = L::tile_points(nw);
    const size_t TB = L::tile_bytes(nw);
    const int ntiles = (N + TP - 1) / TP;
    const int ks = FLUSH_BLOCKS_ALL;   // tiles between slow flushes: 32 FLUSH_BLOCKS_ALL points per warp
    // tiles [tb, te) of the block (TAIL: a part of it)
    const int tbeg = TAIL ? t_begin : 0, tend = TAIL ? t_end : ntiles;

    __syncthreads();   // previous block's epilogue is done with the sums and tiles
    // each thread clears the residual entries it flushes into; the slow sums
    // are first touched after a tile barrier
    for (int q = lane; q < (int)L::RR_PER_WARP; q += 32) rr[(size_t)warp * L::RR_PER_WARP + q] = make_float2(0.f, 0.f);
    for (int q = tid; q < (int)L::RS_ENTRIES; q += blockDim.x) rs[q] = make_float2(0.f, 0.f);
    auto issue = [&](int k, uint64_t *bar) {
        const unsigned n = (unsigned)min(TP, N - k * TP);
        mbar_arrive_expect_tx(bar, n * L::RB);
        bulk_g2s(tiles + ((k - tbeg) & 1) * TB, src + (size_t)k * TB, n * L::RB, bar);
    };
    if (tid == 0)
        for (int k = tbeg; k < tbeg + 2 && k < tend; ++k) issue(k, &bars[(k - tbeg) & 1]);

    MixedAcc<P, F, NSET> acc;
#pragma unroll
    for (int k = 0; k < NPC; ++k)
#pragma unroll
        for (int q = 0; q < Q; ++q) acc.a[k][q] = make_float2(0.0f, 0.0f);
    float2 *mine = rr + (size_t)warp * L::RR_PER_WARP;
    auto flush_r = [&]() {
#pragma unroll
        for (int k = 0; k < NPC; ++k)
#pragma unroll
            for (int j = 0; j < 2 * NSET; ++j) {
                float2 &m = mine[(j * NPC + k) * 32 + lane];
                m = __fadd2_rn(m, acc.a[k][L::fast_q(j)]);
                acc.a[k][L::fast_q(j)] = make_float2(0.0f, 0.0f);
            }
    };
    auto flush_slow = [&]() {   // all threads; nw steps, a CTA barrier after each
        for (int s = 0; s < nw; ++s) {
            const int slice = (warp + s) % nw;
#pragma unroll
            for (int b = 0; b < QS; ++b)
                if (b % nw == slice)
#pragma unroll
                    for (int k = 0; k < NPC; ++k) {
                        float2 &m = rs[(b * NPC + k) * 32 + lane];
                        m = __fadd2_rn(m, acc.a[k][L::slow_q(b)]);
                        acc.a[k][L::slow_q(b)] = make_float2(0.0f, 0.0f);
                    }
            if constexpr (COMP) {   // the warp's residual running sums (at most
                                    // FLUSH_BLOCKS_ALL flushes) into the CTA's compensated totals
#pragma unroll 1
                for (int j = 0; j < L::QR; ++j)
                    if ((QS + j) % nw == slice)
#pragma unroll 1
                        for (int k = 0; k < NPC; ++k) {
                            float2 &v = mine[(j * NPC + k) * 32 + lane];
                            kahan_add2(rs[((QS + j) * NPC + k) * 32 + lane], rs[((QS + L::QR + j) * NPC + k) * 32 + lane], v);
                            v = make_float2(0.0f, 0.0f);
                        }
            }
            __syncthreads();
        }
    };
    int since = 0;   // points of this warp since the last flush of the residual sums

    for (int tile = tbeg; tile < tend; ++tile) {
        const int b = (tile - tbeg) & 1;
        const uint32_t par = b ? (use1++ & 1u) : (use0++ & 1u);
        if (!mbar_wait_bounded(&bars[b], par)) {
            if (lane == 0) atomicExch(prm.err, FREDEC_ETIMEOUT);
        }
        const int n = min(TP, N - tile * TP);
        const unsigned char *tb = tiles + b * TB;
        const int cnt = n > warp ? (n - warp + nw - 1) / nw : 0;
        const unsigned char *pw = tb + (size_t)warp * L::RB;
        const size_t stride = (size_t)nw * L::RB;
        for (int k = 0; k < cnt;) {
            const int take = min(cnt - k, FLUSH_POINTS - since);
            if (prm.seed_mode == 0)
                mixed_run<P, F, 0, NSET>(pw + (size_t)k * stride, stride, take, tabf, j0, acc);
            else
                mixed_run<P, F, 1, NSET>(pw + (size_t)k * stride, stride, take, tabf, j0, acc);
            k += take;
            since += take;
            if (since == FLUSH_POINTS) {
                flush_r();
                since = 0;
            }
        }
        __syncthreads();   // all warps are done with buffer b
        if (tid == 0 && tile + 2 < tend) issue(tile + 2, &bars[b]);
        if ((tile + 1 - tbeg) % ks == 0 && tile + 1 < tend) flush_slow();
    }
    flush_r();
    flush_slow();
    if constexpr (TAIL)
        if ((tbeg != 0 || tend != ntiles) && !tail_exchange<P, F, NSET, COMP>(prm, *tp, blk, ntiles, tend - tbeg, rr, rs))
            return;   // another CTA completes the block

    // Epilogue: the slow sums (and with COMP the residual totals) from the
    // CTA array, else the residual sums from the warps'; FP64 solve per
    // frequency.
    double *zbuf = reinterpret_cast<double *>(tiles);
    const double W = st.Wf;
    const int64_t nf = d.nf;
    const bool mixed_flags = prm.flag_tau >= 0.0;
    auto rd = [&](const float2 *a, int k, int ln) {
        const float2 v = a[(k >> 1) * 32 + ln];
        return (k & 1) ? v.y : v.x;
    };
    for (int fs = tid; fs < 32 * F; fs += blockDim.x) {
        const int k = fs >> 5, ln = fs & 31;
        const int64_t j = jblock + (int64_t)ln * F + k;
        if (j >= nf) continue;
        double S[Q];
#pragma unroll
        for (int bq = 0; bq < QS; ++bq) S[L::slow_q(bq)] = (double)rd(rs + (size_t)bq * NPC * 32, k, ln);
#pragma unroll
        for (int jr = 0; jr < L::QR; ++jr) {
            if constexpr (COMP) {   // total minus its compensation, rounded once to FP32
                S[L::fast_q(jr)] = (double)(rd(rs + (size_t)(QS + jr) * NPC * 32, k, ln) -
                                            rd(rs + (size_t)(QS + L::QR + jr) * NPC * 32, k, ln));
            } else {   // the warps' running sums, added in FP32
                float v = 0.0f;
                for (int w = 0; w < nw; ++w) v += rd(rr + (size_t)w * L::RR_PER_WARP + (size_t)jr * NPC * 32, k, ln);
                S[L::fast_q(jr)] = (double)v;
            }
        }
        double vcc = 0.0, vcs = 0.0, vss = 0.0;
#pragma unroll
        for (int q = 0; q < P; ++q) {
            vcc = fma(S[q], S[q], vcc);
            vcs = fma(S[q], S[P + q], vcs);
            vss = fma(S[P + q], S[P + q], vss);
        }
        const double CC = S[2 * P + 2], CS = S[2 * P + 3];
        double a, bb, zz;
        bool done = false;
        if (mixed_flags) {
            done = solve2_fast(CC, CS, W - CC, vcc, vcs, vss, S[2 * P], S[2 * P + 1], prm.flag_tau, &zz, &a, &bb);
            if (!done) {   // ill-conditioned: provisional value now, FP64-grade re-evaluation later
                const int32_t at = atomicAdd(prm.flag_count, 1);
                if (at < prm.flag_cap) prm.flag_list[at] = d.z_off + j;
                else atomicExch(prm.err, FREDEC_EINVAL);
            }
        }
        if (!done) {
            double ratio;
            zz = solve2(CC, CS, W - CC, vcc, vcs, vss, S[2 * P], S[2 * P + 1], &a, &bb, &ratio);
        }
        if constexpr (NSET == 2) prm.dzdf[d.z_off + j] = dz_df<P>(S, S + L::Q0, *prm.wt_sum, a, bb);
        if constexpr (MIRROR) zbuf[ln * F + k] = zz;
        else prm.z[d.z_off + j] = zz;
        if (prm.coef) {
            prm.coef[2 * (d.z_off + j)] = a;
            prm.coef[2 * (d.z_off + j) + 1] = bb;
        }
    }
    if constexpr (MIRROR) {
        fence_proxy_async_smem();
        __syncthreads();
        for (int i = tid; i < 32 * F; i += blockDim.x) {
            const int64_t j = jblock + i;
            if (j < nf) {
                prm.z[d.z_off + j] = zbuf[i];
                prm.z_mirror[d.z_off + j] = zbuf[i];
            }
        }
    }
}

// Register cap of the grid kernel (which may be launched with up to 256
// threads): mixed kernels whose F x (2P+4) accumulators fit take 128
// registers (16 warps per SM) up to 80 accumulators and 168 (three CTAs of
// four warps) up to 120 (two-set kernels: 168 up to 120 accumulators, their
// second set of per-point values needs the registers); the others, and the
// FP64 kernels, are not capped.
template <int PREC, int P, int F, int NSET = 1>
constexpr int pgram_maxreg() {
    return PREC != FREDEC_MIXED                      ? 255
           : NSET == 1 && F * (2 * P + 4) <= 80       ? 128
           : NSET * F * (2 * P + 4) <= 120            ? 168
                                                      : 255;
}

// Grid kernel: one CTA per block of 32*F frequencies of the series desc[0].
// The single-series mixed kernels keep CTA-level slow sums (pgram_block_cs).
template <int PREC, int NSET>
constexpr bool pgram_cs() { return PREC == FREDEC_MIXED; }

template <int PREC, int P, int F, bool MIRROR, int NSET = 1, bool COMP = false>
__global__ void __launch_bounds__(256, 1) __maxnreg__((pgram_maxreg<PREC, P, F, NSET>())) pgram_kernel(PgramParams prm) {
    extern __shared__ __align__(128) unsigned char smem[];
    pgram_cta_init<PREC>(smem);
    grid_dependency_wait();   // prep's records and state
    allow_dependents();       // the tail kernel's CTAs may start as this grid's drain
    const SeriesDesc d = prm.desc[0];
    const SeriesState &st = prm.state[0];
    if (st.status != FREDEC_OK) return;
    uint32_t use0 = 0u, use1 = 0u;
    if constexpr (pgram_cs<PREC, NSET>())
        pgram_block_cs<P, F, MIRROR, NSET, COMP>(prm, d, st, blockIdx.x, smem, use0, use1);
    else
        pgram_block<PREC, P, F, NSET>(prm, d, st, blockIdx.x, smem, use0, use1);
}

// The tail of a mixed single-series launch: tail CTA g sums the tiles
// [u0(g), u0(g + 1)) of the blocks from tp.b0 on (tail_exchange).
template <int PREC, int P, int F, bool MIRROR, int NSET, bool COMP>
__global__ void __launch_bounds__(256, 1) __maxnreg__((pgram_maxreg<PREC, P, F, NSET>())) pgram_tail_kernel(PgramParams prm,
                                                                                                TailParams tp) {
    extern __shared__ __align__(128) unsigned char smem[];
    pgram_cta_init<PREC>(smem);
    // No wait here: this grid starts once every CTA of the main launch has
    // passed its own wait for prep (allow_dependents), so the records are in
    // place; its CTAs fill the SMs that the main launch's last wave frees.
    const SeriesDesc d = prm.desc[0];
    const SeriesState &st = prm.state[0];
    if (st.status != FREDEC_OK) {
        grid_dependency_wait();
        return;
    }
    const int TP = 32 * (int)(blockDim.x >> 5), ntiles = (d.N + TP - 1) / TP;
    const int64_t nblocks = (d.nf + 32 * F - 1) / (32 * F);
    const int64_t U = (nblocks - tp.b0) * ntiles, G = gridDim.x;
    const int64_t u1 = tail_u0((int64_t)blockIdx.x + 1, U, G);
    uint32_t use0 = 0u, use1 = 0u;
    for (int64_t u = tail_u0(blockIdx.x, U, G); u < u1;) {
        const int64_t blk = tp.b0 + u / ntiles;
        const int t0 = (int)(u % ntiles), t1 = t0 + (u1 - u) < ntiles ? (int)(t0 + (u1 - u)) : ntiles;
        pgram_block_cs<P, F, MIRROR, NSET, COMP, true>(prm, d, st, blk, smem, use0, use1, t0, t1, &tp);
        u += t1 - t0;
    }
    // this grid ends after the main launch, so that a kernel that waits for
    // it (the re-evaluation of flagged bins) sees both launches' z
    grid_dependency_wait();
}

constexpr size_t SMEM_LIMIT = 227 * 1024;

template <int PREC, int P, int F, int NSET = 1, bool COMP = false>
size_t pgram_smem_t(int warps) {
    if constexpr (pgram_cs<PREC, NSET>()) return PgramCsLayout<P, F, NSET, COMP>::smem_bytes(warps);
    else return PgramLayout<PREC, P, F, NSET>::smem_bytes(warps);
}

template <int PREC, int P, int F, bool MIRROR, int NSET, bool COMP>
int launch_pgram_k(const PgramParams &prm, int64_t nblocks, int warps, cudaStream_t st) {
    const size_t smem = pgram_smem_t<PREC, P, F, NSET, COMP>(warps);
    if (smem > SMEM_LIMIT) return fail(FREDEC_EINVAL, "launch shape needs more than 227 KB of shared memory");
    if ((prm.z_mirror != nullptr) != MIRROR) return fail(FREDEC_EINVAL, "z mirror and kernel variant differ");
    auto kern = pgram_kernel<PREC, P, F, MIRROR, NSET, COMP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail(FREDEC_ECUDA, std::string("smem attribute: ") + cudaGetErrorString(e));
    if (nblocks <= 0) return FREDEC_OK;
    e = launch_pdl(kern, dim3((unsigned)nblocks), dim3(warps * 32), smem, st, prm);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(FREDEC_ECUDA, std::string("pgram launch: ") + cudaGetErrorString(e));
    return FREDEC_OK;
}

// Mixed single-series launch with a tail split: the main kernel takes the
// whole waves of blocks (resident CTAs per SM x SMs), pgram_tail_kernel the
// rest, spread evenly over up to a wave of CTAs.  Measured on the N = 2000,
// p = 7 series with F = 10 and four warps (two CTAs per SM): 947,200
// frequencies (10 whole waves) 1.514 ms, 1e6 (10.56 waves) 1.657 ms, 1,041,920
// (11 waves) 1.663 ms: a part-filled last wave that puts two CTAs on some SMs
// costs a whole one (split: 1.620 ms).  The split pays when the rest puts more
// than one CTA on some SM, or leaves fewer than 3 warps per SM on average (1e6
// frequencies with two warps: 1.678 -> 1.647 ms; z and dz/df at F = 4, 117
// blocks left, two warps: 3.321 -> 3.271 ms); with one 4-warp CTA on each of
// 117 SMs the lone CTAs already run faster than shared ones, and the split
// cost 1.1% (3.273 -> 3.310 ms).  Not when the rest fills 90% of a wave.
template <int P, int F, bool MIRROR, int NSET, bool COMP>
int launch_pgram_split(const PgramParams &prm, const TailParams &tail, int64_t nblocks, int warps, cudaStream_t st) {
    constexpr int PREC = FREDEC_MIXED;
    static std::atomic<int> occ_cache[9];
    const size_t smem = pgram_smem_t<PREC, P, F, NSET, COMP>(warps);
    int occ = warps >= 1 && warps <= 8 ? occ_cache[warps].load() : 0;
    if (occ == 0 && smem <= SMEM_LIMIT) {
        auto kern = pgram_kernel<PREC, P, F, MIRROR, NSET, COMP>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, warps * 32, smem) == cudaSuccess && occ > 0)
            occ_cache[warps].store(occ);
        else
            occ = 0, (void)cudaGetLastError();
    }
    const int64_t slots = (int64_t)occ * sm_count();
    const int64_t full = slots > 0 ? nblocks / slots * slots : 0, rem = nblocks - full;
    const int64_t ntiles = ((int64_t)tail.n_points + 32 * warps - 1) / (32 * warps);
    const int64_t U = rem * ntiles, min_units = (ntiles + TAIL_MAX_PARTS - 2) / (TAIL_MAX_PARTS - 1);
    const int64_t G = std::min<int64_t>(std::min<int64_t>(slots, tail.gcap), U / std::max<int64_t>(min_units, 1));
    const int64_t sms = sm_count();
    const bool pays = rem > sms || rem * warps < 3 * sms;   // see above
    if (full == 0 || rem == 0 || rem > tail.gcap || rem * 10 > slots * 9 || G < 1 || !pays)
        return launch_pgram_k<PREC, P, F, MIRROR, NSET, COMP>(prm, nblocks, warps, st);
    if (int rc = launch_pgram_k<PREC, P, F, MIRROR, NSET, COMP>(prm, full, warps, st)) return rc;
    TailParams tp = tail;
    tp.b0 = full;
    auto kern = pgram_tail_kernel<PREC, P, F, MIRROR, NSET, COMP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = launch_pdl(kern, dim3((unsigned)G), dim3(warps * 32), smem, st, prm, tp);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(FREDEC_ECUDA, std::string("pgram tail launch: ") + cudaGetErrorString(e));
    return FREDEC_OK;
}

// The mixed kernels with compensated residual totals serve series whose warps
// would otherwise add more than COMP_MIN_FLUSHES flushes into their FP32
// running sums (prm.comp, set by the launcher).
template <int PREC, int P, int F, bool MIRROR = false, int NSET = 1>
int launch_pgram_t(const PgramParams &prm, int64_t nblocks, int warps, cudaStream_t st,
                   const TailParams *tail = nullptr) {
    if constexpr (PREC == FREDEC_MIXED)
        if (tail && tail->part)
            return prm.comp ? launch_pgram_split<P, F, MIRROR, NSET, true>(prm, *tail, nblocks, warps, st)
                            : launch_pgram_split<P, F, MIRROR, NSET, false>(prm, *tail, nblocks, warps, st);
    if constexpr (PREC == FREDEC_MIXED)
        if (prm.comp) return launch_pgram_k<PREC, P, F, MIRROR, NSET, true>(prm, nblocks, warps, st);
    return launch_pgram_k<PREC, P, F, MIRROR, NSET, false>(prm, nblocks, warps, st);
}

}  // namespace fredec
