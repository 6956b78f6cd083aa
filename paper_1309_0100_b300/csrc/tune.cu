// Launch-shape autotuner: times every compiled (frequencies per thread, warps
// per CTA) shape of the periodogram kernel on synthetic device data and keeps
// the fastest per (precision, p, log2 N, log2 nf).  Optional text cache file
// named by FREDEC_TUNE_CACHE: one line "prec p nbucket nfbucket fpt warps".
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "fredec_internal.cuh"

namespace fredec {

int compiled_fpts(int precision, int p, int *out);

namespace {

using Key = std::tuple<int, int, int, int>;
std::mutex g_mu;
std::map<Key, PgramShape> g_table;
bool g_loaded = false;

int bucket(int64_t n) { return n <= 1 ? 0 : (int)std::floor(std::log2((double)n)); }

void load_locked() {
    if (g_loaded) return;
    g_loaded = true;
    const char *path = std::getenv("FREDEC_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    int pr, p, nb, fb, fpt, w;
    while (std::fscanf(f, "%d %d %d %d %d %d", &pr, &p, &nb, &fb, &fpt, &w) == 6)
        if (shape_supported(pr, p, fpt) && w >= 1 && w <= 8) g_table[Key(pr, p, nb, fb)] = PgramShape{fpt, w};
    std::fclose(f);
}

void save_locked() {
    const char *path = std::getenv("FREDEC_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "w");
    if (!f) return;
    for (const auto &kv : g_table)
        std::fprintf(f, "%d %d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                     std::get<3>(kv.first), kv.second.fpt, kv.second.warps);
    std::fclose(f);
}

// Counter-based synthetic inputs (splitmix64 of the index).
__device__ __forceinline__ double u01(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

__global__ void synth_kernel(double *t, double *y, double *s, double *base, int64_t N, int nb) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        t[i] = 3000.0 * (double)i / (double)N + u01(4 * i);
        y[i] = 4.0 * u01(4 * i + 1) - 2.0;
        s[i] = 0.5 + u01(4 * i + 2);
    }
    if (blockIdx.x == 0 && threadIdx.x < nb) base[threadIdx.x] = 0.01 + 0.37 * (threadIdx.x + 1);
}

}  // namespace

bool tuned_shape(int precision, int p, int64_t N, int64_t nf, PgramShape *out) {
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    auto it = g_table.find(Key(precision, p, bucket(N), bucket(nf)));
    if (it == g_table.end()) return false;
    *out = it->second;
    return true;
}

}  // namespace fredec

using namespace fredec;

extern "C" int fredec_tune(int32_t precision, int32_t n_base, int64_t N, int64_t nf, int32_t *best_fpt,
                           int32_t *best_warps) {
    if (precision != FREDEC_FP64 && precision != FREDEC_MIXED) return fail(FREDEC_EINVAL, "bad precision");
    if (n_base < 0 || n_base > FREDEC_MAX_NBASE || N < 2LL * n_base + 3 || nf <= 0 || nf > (1LL << 31) - 1)
        return fail(FREDEC_EINVAL, "bad tuning sizes");
    const int p = 2 * n_base + 1;
    cudaStream_t st;
    FREDEC_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    int rc = FREDEC_OK;
    PgramShape best{0, 0};
    {
        DevBuf in, out;
        if ((rc = in.alloc((3 * N + n_base + 1) * 8, st)) || (rc = out.alloc(nf * 8, st))) {
            cudaStreamDestroy(st);
            return rc;
        }
        double *t = in.as<double>(), *y = t + N, *s = y + N, *base = s + N;
        synth_kernel<<<256, 256, 0, st>>>(t, y, s, base, N, n_base);
        int fpts[4];
        const int nfpt = compiled_fpts(precision, p, fpts);
        const int warps_opts[4] = {1, 2, 4, 8};
        float best_ms = 1e30f;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int a = 0; a < nfpt && !rc; ++a)
            for (int b = 0; b < 4 && !rc; ++b) {
                fredec_opts o;
                fredec_opts_init(&o);
                o.precision = precision;
                o.fpt = fpts[a];
                o.warps = warps_opts[b];
                o.flag_tau = -1.0;
                float ms_min = 1e30f;
                bool skip = false;
                for (int rep = 0; rep < 3 && !rc && !skip; ++rep) {
                    cudaEventRecord(e0, st);
                    rc = fredec_periodogram_dev(t, y, s, N, base, n_base, 1e-4, 2e-6, nf, &o, out.as<double>(),
                                                nullptr, nullptr, nullptr, st);
                    if (rc == FREDEC_EINVAL) {   // shape does not fit (shared memory): not a candidate
                        rc = FREDEC_OK;
                        skip = true;
                        break;
                    }
                    cudaEventRecord(e1, st);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) ms_min = std::fmin(ms_min, ms);
                }
                if (!rc && !skip && ms_min < best_ms) {
                    best_ms = ms_min;
                    best = PgramShape{fpts[a], warps_opts[b]};
                }
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        load_locked();
        g_table[Key(precision, p, bucket(N), bucket(nf))] = best;
        save_locked();
    }
    if (best_fpt) *best_fpt = best.fpt;
    if (best_warps) *best_warps = best.warps;
    return FREDEC_OK;
}
