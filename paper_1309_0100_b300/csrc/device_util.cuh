// Device helpers: fixed-point phases, sin/cos seeds, TMA bulk copies with
// bounded mbarrier waits, deterministic reductions, small Cholesky factors.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fredec {

constexpr double TWO_PI_D = 6.283185307179586476925286766559;
constexpr float TWO_PI_OVER_2_32 = 1.46291807926715968e-9f;   // 2 pi / 2^32
constexpr double TWO_POW_64 = 18446744073709551616.0;
constexpr double TWO_POW_M64 = 5.421010862427522170037e-20;
constexpr unsigned WAIT_LIMIT = 1u << 24;                       // bounded mbarrier polls

// Programmatic dependent launch.  A kernel launched with the programmatic
// stream serialization attribute (launch_pdl) may start while its predecessor
// in the stream is still running; grid_dependency_wait() returns once every
// prerequisite grid has completed and its memory writes are visible (at once
// when there is none), so it comes before the first read of their results.
// allow_dependents() lets the next such kernel start launching before this
// grid ends (otherwise it does when this grid's CTAs exit).
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// frac(f * t) as unsigned 64-bit fixed-point turns.  The product is split into
// its rounded value x and its exact rounding error e (fma).  r = x - rint(x)
// is exact (Sterbenz: x and rint(x) are within a factor 2 unless rint(x) = 0,
// where r = x), so r and e are converted to 2^-64 units separately and added
// modulo 2^64; the result is within one unit (5.4e-20 turns) of frac(f t) for
// |f t| < 2^20.
__device__ __forceinline__ uint64_t frac_turns_u64(double f, double t) {
    const double x = f * t;
    const double e = fma(f, t, -x);
    double r = x - rint(x);                         // exact, in [-0.5, 0.5]
    if (r >= 0.5) r -= 1.0;                         // same phase, keeps r * 2^64 inside int64
    const int64_t ir = __double2ll_rn(r * TWO_POW_64);
    const int64_t ie = __double2ll_rn(e * TWO_POW_64);
    return (uint64_t)ir + (uint64_t)ie;
}

// Signed turns in [-0.5, 0.5) of a fixed-point phase, as double (53 bits).
__device__ __forceinline__ double turns_of(uint64_t ph) {
    return (double)(int64_t)ph * TWO_POW_M64;
}

// cos and sin of 2 pi k / 256, k = 0..255, evaluated at compile time: the
// quadrant and the complement symmetry reduce the angle to x = r pi/128 in
// [0, pi/4], whose Taylor series (to x^24 / x^25, truncation below 1e-22) is
// summed in nested form in double.  Within 1.3e-16 of the exact values (about
// 1 ulp); the seed tables of every precision are filled from it, so no CTA
// spends FP64 sin/cos work (FP64 runs at 1/64 of the FP32 rate on this GPU).
struct SinCos256 { double c[256]; double s[256]; };
constexpr SinCos256 make_sincos256() {
    SinCos256 t{};
    constexpr double PI_128 = 0.024543692606170259675489401431871;   // pi / 128
    for (int k = 0; k < 256; ++k) {
        const int q = k / 64, r = k % 64;
        const bool comp = r > 32;                       // x = pi/2 - (64 - r) pi/128
        const double x = (comp ? 64 - r : r) * PI_128, x2 = x * x;
        double c = 1.0, s = 1.0;
        for (int n = 12; n >= 1; --n) {
            c = 1.0 - x2 / ((2.0 * n - 1.0) * (2.0 * n)) * c;
            s = 1.0 - x2 / ((2.0 * n) * (2.0 * n + 1.0)) * s;
        }
        s *= x;
        const double cr = comp ? s : c, sr = comp ? c : s;   // angle r pi/128
        t.c[k] = q == 0 ? cr : q == 1 ? -sr : q == 2 ? -cr : sr;
        t.s[k] = q == 0 ? sr : q == 1 ? cr : q == 2 ? -sr : -cr;
    }
    return t;
}
static __device__ const SinCos256 g_sincos256 = make_sincos256();

// FP64 sin/cos of a fixed-point phase by table lookup and a short Taylor
// polynomial (Tang's table-driven method): the top 8 bits select
// e^{2 pi i k/256} from the table above, the remaining fraction (< 1/256 turn,
// |theta| < 0.0246 rad) is evaluated by Taylor series to degree 7 (sin) and
// 8 (cos), then the two rotations are multiplied.  Truncation error < 1e-20,
// about 2e-16 in all.  Kernels copy the table into shared memory.
using SeedTable = SinCos256;

__device__ __forceinline__ void seed_from_table(const SeedTable &tab, uint64_t ph, double *s, double *c) {
    const unsigned k = (unsigned)(ph >> 56);
    const uint64_t rem = ph & 0x00FFFFFFFFFFFFFFull;
    const double th = (double)(int64_t)rem * (TWO_PI_D * TWO_POW_M64);
    const double t2 = th * th;
    const double ps = th * fma(t2, fma(t2, fma(t2, -1.0 / 5040.0, 1.0 / 120.0), -1.0 / 6.0), 1.0);
    const double pc = fma(t2, fma(t2, fma(t2, fma(t2, 1.0 / 40320.0, -1.0 / 720.0), 1.0 / 24.0), -0.5), 1.0);
    const double tc = tab.c[k], ts = tab.s[k];
    *c = fma(tc, pc, -ts * ps);
    *s = fma(ts, pc, tc * ps);
}

// The same from the table in global memory (L1/L2-resident), for code that
// evaluates a few sin/cos per thread and keeps no table of its own.
__device__ __forceinline__ void sincos_turns_d(uint64_t ph, double *s, double *c) {
    seed_from_table(g_sincos256, ph, s, c);
}

// FP32 variant for the mixed kernel: table of e^{2 pi i k/256} rounded to FP32
// and a Taylor polynomial of degree 3 (sin) / 4 (cos) on the remaining
// < 1/256 turn (truncation < 1e-10); the low 32 bits of the phase are dropped
// (< 1.5e-9 rad).
struct SeedTableF { float2 cs[256]; };

__device__ __forceinline__ void seed_from_table_f(const SeedTableF &tab, uint32_t ph_hi, float *s, float *c) {
    const float2 t = tab.cs[ph_hi >> 24];
    const float th = (float)(int32_t)(ph_hi & 0x00FFFFFFu) * TWO_PI_OVER_2_32;
    const float t2 = th * th;
    const float ps = th * fmaf(t2, -1.0f / 6.0f, 1.0f);
    const float pc = fmaf(t2, fmaf(t2, 1.0f / 24.0f, -0.5f), 1.0f);
    *c = fmaf(t.x, pc, -t.y * ps);
    *s = fmaf(t.y, pc, t.x * ps);
}

__device__ __forceinline__ void fill_seed_table_f(SeedTableF &tab) {
    for (int k = threadIdx.x; k < 256; k += blockDim.x)
        tab.cs[k] = make_float2(__double2float_rn(g_sincos256.c[k]), __double2float_rn(g_sincos256.s[k]));
}

__device__ __forceinline__ void fill_seed_table(SeedTable &tab) {
    for (int k = threadIdx.x; k < 256; k += blockDim.x) {
        tab.c[k] = g_sincos256.c[k];
        tab.s[k] = g_sincos256.s[k];
    }
}

// ---------------------------------------------------------------------------
// Float-float ("FF") arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2,
// about 48 significant bits, from the error-free transformations TwoSum
// (Knuth), FastTwoSum (Dekker) and the FMA product error.  Every step is an
// explicitly rounded intrinsic, so the compiler neither contracts nor
// reassociates them.  On this GPU a float-float operation costs a few FP32
// instructions, against one FP64 instruction at 1/64 of the FP32 rate.

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ ff ff_from_double(double d) {
    const float hi = __double2float_rn(d);
    return {hi, __double2float_rn(d - (double)hi)};
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
// a + b with both parts' errors carried (no loss when a ~ -b)
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = ff_two_sum(a.hi, b.hi);
    const ff t = ff_two_sum(a.lo, b.lo);
    s = ff_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return ff_fast_two_sum(p, e);
}

// Running float-float sum H + L: each addend's hi part enters by TwoSum, the
// error and the lo parts go into L, and (H, L) is renormalised (FastTwoSum) --
// the double-float sum, about 1e-16 of the summed magnitudes (a compensated
// sum with a single-float compensation would keep an error of order 1e-7 of
// them per term).
struct ff_acc {
    float H = 0.0f, L = 0.0f;
    __device__ __forceinline__ void add(ff p) {
        const ff s = ff_two_sum(H, p.hi);
        const ff r = ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(L, p.lo)));
        H = r.hi;
        L = r.lo;
    }
    __device__ __forceinline__ void add_prod(ff a, ff b) {   // add a * b (exact hi product, cross terms)
        const float p = __fmul_rn(a.hi, b.hi);
        float e = __fmaf_rn(a.hi, b.hi, -p);
        e = __fmaf_rn(a.hi, b.lo, e);
        e = __fmaf_rn(a.lo, b.hi, e);
        add({p, e});
    }
    __device__ __forceinline__ double value() const { return (double)H + (double)L; }
};

// FF sin/cos of a 64-bit fixed-point phase (Tang's table method in float-float
// arithmetic): the top 8 bits select e^{2 pi i k/256} from a table of FF pairs
// (the compile-time table g_sincos256, split), the remaining < 1/256 turn x = 2 pi rem 2^-64
// (|x| < 0.0246) is evaluated by its Taylor series -- the x^2 terms in FF, the
// terms below 2e-8 in FP32 -- and the two rotations are multiplied in FF.
// Error about 1e-15 absolute.
struct SeedTableFF { float4 cs[256]; };   // (cos hi, cos lo, sin hi, sin lo)

__device__ __forceinline__ void fill_seed_table_ff(SeedTableFF &tab) {
    for (int k = threadIdx.x; k < 256; k += blockDim.x) {
        const ff fc = ff_from_double(g_sincos256.c[k]), fs = ff_from_double(g_sincos256.s[k]);
        tab.cs[k] = make_float4(fc.hi, fc.lo, fs.hi, fs.lo);
    }
}

// sin/cos of 2 pi k/256 + x, |x| < 0.0246 (the shared part of the two entry
// points below).
__device__ __forceinline__ void ff_sincos_reduced(const SeedTableFF &tab, int k, ff x, ff *s, ff *c) {
    const ff x2 = ff_mul(x, x);
    const float t4 = __fmul_rn(x2.hi, x2.hi);
    // cos x = 1 - (x^2/2 - x^4/24 + x^6/720);  sin x = x - x (x^2/6 - x^4/120 + x^6/5040)
    const float hc = __fmul_rn(t4, __fmaf_rn(-x2.hi, 1.0f / 720.0f, 1.0f / 24.0f));
    const ff h = ff_add({__fmul_rn(x2.hi, 0.5f), __fmul_rn(x2.lo, 0.5f)}, {-hc, 0.0f});
    const ff cx = ff_sub({1.0f, 0.0f}, h);
    constexpr ff SIXTH = {0.1666666716337204f, -4.967053879312289e-09f};   // 1/6 = hi + lo
    const float hs = __fmul_rn(t4, __fmaf_rn(-x2.hi, 1.0f / 5040.0f, 1.0f / 120.0f));
    const ff g = ff_add(ff_mul(x2, SIXTH), {-hs, 0.0f});
    const ff sx = ff_sub(x, ff_mul(x, g));
    const float4 T = tab.cs[k & 255];
    const ff tc = {T.x, T.y}, ts = {T.z, T.w};
    *c = ff_sub(ff_mul(tc, cx), ff_mul(ts, sx));
    *s = ff_add(ff_mul(ts, cx), ff_mul(tc, sx));
}

__device__ __forceinline__ void ff_sincos_turns(const SeedTableFF &tab, uint64_t ph, ff *s, ff *c) {
    const uint64_t rem = ph & 0x00FFFFFFFFFFFFFFull;
    // x = rem * (2 pi 2^-64): rem = rh + rl with rh exact in FP32, rl rounded
    // (error < 2^-56 turn); 2 pi 2^-64 as an FF constant
    const float rh = __fmul_rn((float)(uint32_t)(rem >> 32), 4294967296.0f);
    const float rl = (float)(uint32_t)(rem & 0xFFFFFFFFull);
    constexpr float CH = 3.4061216748705226e-19f, CL = -9.478396428567739e-27f;   // 2 pi 2^-64 = CH + CL
    const float p = __fmul_rn(rh, CH);
    float e = __fmaf_rn(rh, CH, -p);
    e = __fmaf_rn(rh, CL, e);
    e = __fmaf_rn(rl, CH, e);
    ff_sincos_reduced(tab, (int)(ph >> 56), ff_fast_two_sum(p, e), s, c);
}

// FF sin/cos of 2 pi r for a float-float number of turns r (any size; only its
// fractional part matters): r is reduced to k/256 + rem with |rem| <= 1/512
// turn, exactly, and rem is turned into radians in FF.
__device__ __forceinline__ void ff_sincos_ff_turns(const SeedTableFF &tab, ff r, ff *s, ff *c) {
    const float whole = rintf(r.hi);
    r = ff_fast_two_sum(__fsub_rn(r.hi, whole), r.lo);          // exact: |r.hi - whole| <= 1/2
    const float kf = rintf(__fmul_rn(r.hi, 256.0f));
    const ff rem = ff_fast_two_sum(__fsub_rn(r.hi, __fmul_rn(kf, 1.0f / 256.0f)), r.lo);   // exact subtraction
    constexpr ff TWO_PI = {6.2831854820251465f, -1.7484555314695172e-07f};   // 2 pi = hi + lo
    ff_sincos_reduced(tab, (int)kf, ff_mul(rem, TWO_PI), s, c);
}

// ---------------------------------------------------------------------------
// Shared-memory addresses, mbarriers and TMA bulk copies (inline PTX).

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Orders this thread's earlier generic-proxy accesses to shared memory before
// later async-proxy (TMA) accesses to it.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// One-dimensional TMA bulk copy global -> shared, completing on an mbarrier.
// dst and src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; returns false (and the caller records FREDEC_ETIMEOUT) when the
// phase did not complete within WAIT_LIMIT polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity) {
    for (unsigned it = 0; it < WAIT_LIMIT; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ---------------------------------------------------------------------------
// Fifth-generation tensor cores (tcgen05, inline PTX; one CTA, cta_group::1):
// tensor-memory allocation, bf16 MMAs accumulating in FP32 in tensor memory,
// loads from tensor memory.

// Shared-memory matrix descriptor of a K-major bf16 operand in the 128-byte
// swizzled layout: rows of 64 elements (128 bytes), 8-row groups 1024 bytes
// apart, the 16-byte chunk j of row r stored at chunk j ^ (r % 8); the
// operand starts in a 1024-byte aligned group, and a K step of 16 elements
// advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Byte offset of element (row r, k) of such an operand (k < 64).
__device__ __forceinline__ int umma_sw128_offset(int r, int k) {
    return r * 128 + ((((k >> 3) ^ (r & 7)) & 7) << 4) + ((k & 7) << 1);
}
// Instruction descriptor of kind::f16: bf16 x bf16 -> FP32, A and B K-major,
// D of M x N.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Whole warp: allocate ncols columns (a power of two, 32..512) of tensor
// memory; the address goes to *slot (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {   // whole warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// One thread: D (tensor memory) = A B^T (+ D when acc), operands by descriptor.
__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, bool acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"((uint32_t)acc)
        : "memory");
}
// One thread: the mbarrier receives one arrival when this thread's earlier
// MMAs have completed.
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// Whole warp: 16 consecutive 32-bit columns of each lane's tensor-memory row
// (taddr: lane offset in the upper 16 bits, the warp's quarter of the lanes).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *out) {
    uint32_t v[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) out[j] = __uint_as_float(v[j]);
}

// ---------------------------------------------------------------------------
// Deterministic block reductions (fixed shuffle tree, fixed warp order).

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums v over the block; every thread gets the result.  scratch: >= 32 doubles.
__device__ __forceinline__ double block_sum_d(double v, double *scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum_d(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    double r = 0.0;
    for (int i = 0; i < nw; ++i) r += scratch[i];
    return r;
}

// ---------------------------------------------------------------------------
// Small dense linear algebra in FP64 (packed lower triangle, row-major:
// L[i*(i+1)/2 + j] for j <= i).

__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// In-place Cholesky of a packed symmetric matrix.  Returns false when a pivot is
// not positive or falls below rel * (its original diagonal).
// rinv[j] receives 1 / L_jj: one FP64 reciprocal square root per column
// (L_jj = d / sqrt(d)), the rest are multiplications (an FP64 square root or
// division is a long dependent sequence on this GPU).
__device__ inline bool chol_packed(double *A, int n, double rel, double *rinv) {
    for (int j = 0; j < n; ++j) {
        const double d0 = A[tri(j, j)];
        double d = d0;
        for (int k = 0; k < j; ++k) d -= A[tri(j, k)] * A[tri(j, k)];
        if (!(d > rel * d0) || !(d0 > 0.0)) return false;
        const double il = rsqrt(d);
        A[tri(j, j)] = d * il;
        rinv[j] = il;
        for (int i = j + 1; i < n; ++i) {
            double s = A[tri(i, j)];
            for (int k = 0; k < j; ++k) s -= A[tri(i, k)] * A[tri(j, k)];
            A[tri(i, j)] = s * il;
        }
    }
    return true;
}

// The same factorisation by the 32 lanes of one warp (n <= 32), right-looking:
// for each column j one FP64 reciprocal square root gives 1 / L_jj (and
// L_jj = d / sqrt(d)), the lanes scale column j, then update the trailing
// lower triangle one entry per lane.  Every entry is updated by one lane in a
// fixed order, so the result is deterministic.  The pivot test is the serial
// version's: the updated diagonal against rel times the original one.  All
// lanes return the same value.
__device__ inline bool chol_packed_warp(double *A, int n, double rel, double *rinv) {
    const int lane = threadIdx.x & 31;
    const double d0_own = lane < n ? A[tri(lane, lane)] : 0.0;
    __syncwarp();
    for (int j = 0; j < n; ++j) {
        const double d = A[tri(j, j)];
        const double d0 = __shfl_sync(0xffffffffu, d0_own, j);
        if (!(d > rel * d0) || !(d0 > 0.0)) return false;   // the same in every lane
        const double il = rsqrt(d);
        __syncwarp();
        if (lane == 0) {
            A[tri(j, j)] = d * il;
            rinv[j] = il;
        }
        for (int i = j + 1 + lane; i < n; i += 32) A[tri(i, j)] *= il;
        __syncwarp();
        const int m = n - j - 1, cnt = m * (m + 1) / 2;
        for (int e = lane; e < cnt; e += 32) {
            // e = r (r + 1) / 2 + c, c <= r: entry (j+1+r, j+1+c) of the trailing triangle
            int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
            if ((r + 1) * (r + 2) / 2 <= e) ++r;
            if (r * (r + 1) / 2 > e) --r;
            const int c = e - r * (r + 1) / 2;
            const int i = j + 1 + r, k = j + 1 + c;
            A[tri(i, k)] -= A[tri(i, j)] * A[tri(k, j)];
        }
        __syncwarp();
    }
    return true;
}

// x <- L^{-1} x (forward substitution), packed L, rinv[i] = 1 / L_ii.
__device__ __forceinline__ void forward_packed(const double *L, const double *rinv, double *x, int n) {
    for (int i = 0; i < n; ++i) {
        double s = x[i];
        for (int k = 0; k < i; ++k) s -= L[tri(i, k)] * x[k];
        x[i] = s * rinv[i];
    }
}

}  // namespace fredec
