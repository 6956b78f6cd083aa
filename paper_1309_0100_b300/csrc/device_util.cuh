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

// FP64 sin/cos of a fixed-point phase with the CUDA sincospi (exact reduction
// is already done by the fixed-point representation).
__device__ __forceinline__ void sincos_turns_d(uint64_t ph, double *s, double *c) {
    sincospi(2.0 * turns_of(ph), s, c);
}

// FP64 sin/cos of a fixed-point phase by table lookup and a short Taylor
// polynomial (Tang's table-driven method): the top 8 bits select
// e^{2 pi i k/256} from a table built with sincospi, the remaining fraction
// (< 1/256 turn, |theta| < 0.0246 rad) is evaluated by Taylor series to
// degree 7 (sin) and 8 (cos), then the two rotations are multiplied.
// Truncation error < 1e-20.
struct SeedTable { double c[256]; double s[256]; };

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
    for (int k = threadIdx.x; k < 256; k += blockDim.x) {
        double s, c;
        sincospi((double)k / 128.0, &s, &c);
        tab.cs[k] = make_float2((float)c, (float)s);
    }
}

__device__ __forceinline__ void fill_seed_table(SeedTable &tab) {
    for (int k = threadIdx.x; k < 256; k += blockDim.x) {
        double s, c;
        sincospi((double)k / 128.0, &s, &c);
        tab.c[k] = c;
        tab.s[k] = s;
    }
}

// ---------------------------------------------------------------------------
// Shared-memory addresses, mbarriers and TMA bulk copies (inline PTX).

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
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
__device__ inline bool chol_packed(double *A, int n, double rel) {
    for (int j = 0; j < n; ++j) {
        const double d0 = A[tri(j, j)];
        double d = d0;
        for (int k = 0; k < j; ++k) d -= A[tri(j, k)] * A[tri(j, k)];
        if (!(d > rel * d0) || !(d0 > 0.0)) return false;
        const double l = sqrt(d);
        A[tri(j, j)] = l;
        for (int i = j + 1; i < n; ++i) {
            double s = A[tri(i, j)];
            for (int k = 0; k < j; ++k) s -= A[tri(i, k)] * A[tri(j, k)];
            A[tri(i, j)] = s / l;
        }
    }
    return true;
}

// x <- L^{-1} x (forward substitution), packed L.
__device__ __forceinline__ void forward_packed(const double *L, double *x, int n) {
    for (int i = 0; i < n; ++i) {
        double s = x[i];
        for (int k = 0; k < i; ++k) s -= L[tri(i, k)] * x[k];
        x[i] = s / L[tri(i, i)];
    }
}

}  // namespace fredec
