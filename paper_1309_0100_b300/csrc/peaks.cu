// Pipe-throughput microbenchmarks: FP32 FMA, FP64 FMA and MUFU sin/cos
// instruction rates of the whole GPU, for the roofline denominators of the
// ALU-bound kernels.  Each thread runs 8 independent dependency chains so the
// pipes, not latency, limit the rate.
#include <algorithm>

#include "device_util.cuh"
#include "fredec_internal.cuh"

namespace {

constexpr int ITERS = 4096;

__global__ void __launch_bounds__(256) ffma_loop(float *out, float a, float b) {
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3f + k;
    for (int i = 0; i < ITERS; ++i)
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 12345.678f) out[0] = s;
}

__global__ void __launch_bounds__(256) dfma_loop(double *out, double a, double b) {
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3 + k;
    for (int i = 0; i < ITERS / 16; ++i)
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 12345.678) out[0] = s;
}

__global__ void __launch_bounds__(256) mufu_loop(float *out) {
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3f + k * 0.1f;
    for (int i = 0; i < ITERS / 8; ++i)
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = __sinf(x[k]);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 12345.678f) out[0] = s;
}

}  // namespace

using namespace fredec;

// out[0] = FP32 FMA/s, out[1] = FP64 FMA/s, out[2] = MUFU sin/s (lane operations).
extern "C" int fredec_pipe_peaks(double *out) {
    if (!out) return fail(FREDEC_EINVAL, "null out");
    const int blocks = sm_count() * 8;
    const double threads = (double)blocks * 256;
    float *dummy;
    FREDEC_CUDA_TRY(cudaMalloc(&dummy, 64));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms;
    double best[3] = {0, 0, 0};
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0);
        ffma_loop<<<blocks, 256>>>(dummy, 0.999f, 1e-3f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        best[0] = std::max(best[0], threads * 8.0 * ITERS / (ms * 1e-3));
        cudaEventRecord(e0);
        dfma_loop<<<blocks, 256>>>((double *)dummy, 0.999, 1e-3);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        best[1] = std::max(best[1], threads * 8.0 * (ITERS / 16) / (ms * 1e-3));
        cudaEventRecord(e0);
        mufu_loop<<<blocks, 256>>>(dummy);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        best[2] = std::max(best[2], threads * 8.0 * (ITERS / 8) / (ms * 1e-3));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(dummy);
    FREDEC_CUDA_TRY(cudaGetLastError());
    for (int k = 0; k < 3; ++k) out[k] = best[k];
    return FREDEC_OK;
}

namespace {
// A bounded wait that nothing completes: one mbarrier expecting one arrival,
// polled a fixed number of times; reports FREDEC_ETIMEOUT, faults nothing.
__global__ void wait_timeout_probe(int32_t *status, unsigned polls) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
    }
    __syncthreads();
    unsigned ok = 0;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
    for (unsigned it = 0; it < polls && !ok; ++it)
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(a)
                     : "memory");
    if (threadIdx.x == 0) *status = ok ? FREDEC_OK : FREDEC_ETIMEOUT;
}
// Largest |FF sin/cos - FP64 sin/cos| over the phases (FP64: the table seed
// of the FP64 path, error < 1e-16).  Deterministic block maximum.
__global__ void ff_sincos_check(const uint64_t *ph, int64_t n, double *out) {
    __shared__ SeedTable tab;
    __shared__ SeedTableFF tabff;
    __shared__ double red[32];
    fill_seed_table(tab);
    fill_seed_table_ff(tabff);
    __syncthreads();
    double m = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double s, c;
        seed_from_table(tab, ph[i], &s, &c);
        ff fs, fc;
        ff_sincos_turns(tabff, ph[i], &fs, &fc);
        m = fmax(m, fmax(fabs(ff_to_double(fs) - s), fabs(ff_to_double(fc) - c)));
        // the same angle given as a float-float number of turns in [-1/2, 1/2)
        ff_sincos_ff_turns(tabff, ff_from_double(turns_of(ph[i])), &fs, &fc);
        m = fmax(m, fmax(fabs(ff_to_double(fs) - s), fabs(ff_to_double(fc) - c)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
        *out = r;
    }
}
}  // namespace

extern "C" int fredec_selftest_ff_sincos(const uint64_t *phases, int64_t n, double *max_err_out) {
    if (!phases || n < 1 || !max_err_out) return fail(FREDEC_EINVAL, "bad self-test arguments");
    void *d = nullptr;
    FREDEC_CUDA_TRY(cudaMalloc(&d, (size_t)n * 8 + 8));
    cudaError_t e = cudaMemcpy(d, phases, (size_t)n * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        ff_sincos_check<<<1, 256>>>((const uint64_t *)d, n, (double *)d + n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(max_err_out, (double *)d + n, 8, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(FREDEC_ECUDA, cudaGetErrorString(e));
    return FREDEC_OK;
}

extern "C" int fredec_selftest_wait_timeout(int32_t *status_out) {
    if (!status_out) return fail(FREDEC_EINVAL, "null status");
    int32_t *d = nullptr;
    FREDEC_CUDA_TRY(cudaMalloc(&d, 4));
    wait_timeout_probe<<<1, 32>>>(d, 1000u);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(status_out, d, 4, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return fail(FREDEC_ECUDA, cudaGetErrorString(e));
    return FREDEC_OK;
}

extern "C" int fredec_profile_events(void *ev_start, void *ev_stop) {
    set_profile_events((cudaEvent_t)ev_start, (cudaEvent_t)ev_stop);
    return FREDEC_OK;
}
