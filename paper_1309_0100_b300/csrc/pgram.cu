// Dispatch of the periodogram kernels over (precision, base size P,
// frequencies per thread F).  The kernels themselves are in pgram_impl.cuh and
// are instantiated per P in pgram_p*.cu.
#include <algorithm>
#include <cstdlib>

#include "fpt_options.h"
#include "pgram_impl.cuh"

namespace fredec {

static thread_local cudaEvent_t g_ev0 = nullptr, g_ev1 = nullptr;

// Mixed-kernel sin/cos seed of each point, from the exact fixed-point phase:
// 0 = 256-entry table + Taylor polynomial (default; error about 1e-7, about 15
// instructions), 1 = the MUFU sin/cos of the phase reduced to [-pi, pi)
// (absolute error about 4e-7, 6 instructions).  Measured: the MUFU seed is 5%
// faster on the N = 2000, 1e6-frequency residual periodogram (largest z error
// against the FP64 kernel 3.0e-6 against 1.8e-6), but on short series with a
// strong signal its error reaches 1.4e-5 at low-z bins, above the 1e-5 bar.
// FREDEC_SEED_MODE=1 in the environment selects it (comparison runs).
int seed_mode() {
    static const int m = [] {
        const char *e = std::getenv("FREDEC_SEED_MODE");
        return (e && e[0] == '1') ? 1 : 0;
    }();
    return m;
}
void set_profile_events(cudaEvent_t a, cudaEvent_t b) { g_ev0 = a; g_ev1 = b; }
void profile_events(cudaEvent_t *a, cudaEvent_t *b) { *a = g_ev0; *b = g_ev1; }

#define FREDEC_DECL_P(P)                                                                              \
    int launch_pgram_p##P(int, int, const PgramParams &, int64_t, int, cudaStream_t, const TailParams *); \
    size_t smem_pgram_p##P(int, int, int);
FREDEC_DECL_P(1) FREDEC_DECL_P(3) FREDEC_DECL_P(5) FREDEC_DECL_P(7) FREDEC_DECL_P(9) FREDEC_DECL_P(11)
FREDEC_DECL_P(13) FREDEC_DECL_P(15) FREDEC_DECL_P(17) FREDEC_DECL_P(19) FREDEC_DECL_P(21)
FREDEC_DECL_P(23) FREDEC_DECL_P(25)
#undef FREDEC_DECL_P

int launch_pgram_mirror_a(int, int, const PgramParams &, int64_t, int, cudaStream_t, const TailParams *);
int launch_pgram_mirror_b(int, int, const PgramParams &, int64_t, int, cudaStream_t, const TailParams *);
int launch_pgram_mirror_c(int, int, const PgramParams &, int64_t, int, cudaStream_t, const TailParams *);

static int dispatch(int p, int prec, int F, const PgramParams &prm, int64_t nblocks, int warps, cudaStream_t st,
                    const TailParams *tail) {
    if (prm.z_mirror) {   // mixed precision only (pgram_mirror_*.cu)
        if (prec != FREDEC_MIXED) return -1;
        int rc = launch_pgram_mirror_a(p, F, prm, nblocks, warps, st, tail);
        if (rc == -2) rc = launch_pgram_mirror_b(p, F, prm, nblocks, warps, st, tail);
        if (rc == -2) rc = launch_pgram_mirror_c(p, F, prm, nblocks, warps, st, tail);
        return rc == -2 ? -1 : rc;
    }
    switch (p) {
#define C(P) case P: return launch_pgram_p##P(prec, F, prm, nblocks, warps, st, tail);
        C(1) C(3) C(5) C(7) C(9) C(11) C(13) C(15) C(17) C(19) C(21) C(23) C(25)
#undef C
    }
    return -1;
}

size_t pgram_smem(int p, int prec, int F, int warps) {
    switch (p) {
#define C(P) case P: return smem_pgram_p##P(prec, F, warps);
        C(1) C(3) C(5) C(7) C(9) C(11) C(13) C(15) C(17) C(19) C(21) C(23) C(25)
#undef C
    }
    return 0;
}

static const FptOptions *options_for(int p) {
    for (const auto &o : kFptOptions)
        if (o.p == p) return &o;
    return nullptr;
}

bool shape_supported(int precision, int p, int fpt) {
    const FptOptions *o = options_for(p);
    if (!o) return false;
    const int *v = precision == FREDEC_MIXED ? o->mixed : o->fp64;
    const int n = precision == FREDEC_MIXED ? o->nmixed : o->nfp64;
    for (int i = 0; i < n; ++i)
        if (v[i] == fpt) return true;
    return false;
}

int compiled_fpts(int precision, int p, int *out) {
    const FptOptions *o = options_for(p);
    if (!o) return 0;
    const int *v = precision == FREDEC_MIXED ? o->mixed : o->fp64;
    const int n = precision == FREDEC_MIXED ? o->nmixed : o->nfp64;
    for (int i = 0; i < n; ++i) out[i] = v[i];
    return n;
}

// Widest mixed shape worth taking for series of at most SHORT_N points, by p
// = 1, 3, ..., 13 (the autotuner's choices at N = 300, nf = 1e6: the
// per-CTA epilogue weighs more against a short point loop, and the widest
// shapes run fewer CTAs per SM); longer series take the widest compiled shape
// (the autotuner's choice for every p <= 13 at N = 2000).  From p = 15 on,
// mixed series of any length take F = 2: F = 3 holds 3 of its 4 frequency
// slots and ran slower at both lengths (kernel ms, nf = 1e6, 4 warps: p = 15
// 3.50 against 3.68 at N = 2000, 0.61 against 0.68 at N = 300; p = 17 3.83
// against 4.20, 0.67 against 0.79).
constexpr int64_t SHORT_N = 1024;
constexpr int SHORT_MIXED_FPT[7] = {12, 8, 8, 6, 8, 4, 4};
constexpr int WIDE_MIXED_FPT = 2;

// Built-in default (without a tuned entry): the largest compiled F (fewest
// re-seeds; for short mixed series at most SHORT_MIXED_FPT) and 4 warps,
// reduced when the grid would not fill the GPU once.
PgramShape default_shape(int precision, int p, int64_t N, int64_t nf) {
    PgramShape s{1, 4};
    const FptOptions *o = options_for(p);
    if (!o) return s;
    const int *v = precision == FREDEC_MIXED ? o->mixed : o->fp64;
    int n = precision == FREDEC_MIXED ? o->nmixed : o->nfp64;
    if (precision == FREDEC_MIXED && N <= SHORT_N && p <= 13)
        while (n > 1 && v[n - 1] > SHORT_MIXED_FPT[(p - 1) / 2]) --n;
    if (precision == FREDEC_MIXED && p >= 15)
        while (n > 1 && v[n - 1] > WIDE_MIXED_FPT) --n;
    s.fpt = v[n - 1];
    const int64_t want = 2LL * sm_count();
    for (int i = n - 1; i > 0; --i) {
        if ((nf + 32LL * v[i] - 1) / (32LL * v[i]) >= want) break;
        s.fpt = v[i - 1];
    }
    if (N < 256) s.warps = 2;
    return s;
}

// Two slots of nset (2p+4) ceil(F/2) 32 float2 partial sums per tail CTA, up to
// two tail CTAs per SM.
size_t pgram_tail_bytes(int precision, int p, int fpt, int *gcap, int nset) {
    *gcap = 0;
    if (precision != FREDEC_MIXED || fpt < 1) return 0;
    *gcap = 2 * sm_count();
    return (size_t)2 * *gcap * nset * (2 * p + 4) * ((fpt + 1) / 2) * 32 * sizeof(float2);
}

int launch_pgram(int precision, const SeriesDesc *desc_dev, const SeriesState *state_dev, const void *rec, int p,
                 int N, int64_t nf, PgramShape shape, double flag_tau, double *z, double *coef, int64_t *flag_list,
                 int32_t *flag_count, int32_t *err, cudaStream_t st, double *z_mirror, float2 *tail_part,
                 int32_t *tail_cnt, int tail_gcap) {
    if (!shape_supported(precision, p, shape.fpt))
        return fail(FREDEC_EINVAL, "no compiled kernel for this (precision, p, frequencies per thread)");
    if (shape.warps < 1 || shape.warps > 8) return fail(FREDEC_EINVAL, "warps per CTA must be in 1..8");
    PgramParams prm{};
    prm.desc = desc_dev;
    prm.state = state_dev;
    prm.rec = (const unsigned char *)rec;
    prm.z = z;
    prm.z_mirror = z_mirror;
    prm.coef = coef;
    prm.flag_tau = (precision == FREDEC_MIXED && flag_list) ? flag_tau : -1.0;
    prm.flag_list = flag_list;
    prm.flag_cap = flag_list ? nf : 0;
    prm.flag_count = flag_count;
    prm.err = err;
    prm.seed_mode = seed_mode();
    prm.comp = pgram_comp(N, shape.warps);
    TailParams tail{};
    if (precision == FREDEC_MIXED && tail_part && tail_cnt && tail_gcap > 0) {
        tail.part = tail_part;
        tail.cnt = tail_cnt;
        tail.gcap = tail_gcap;
        tail.n_points = N;
    }
    const int64_t nblocks = (nf + 32LL * shape.fpt - 1) / (32LL * shape.fpt);
    cudaEvent_t e0, e1;
    profile_events(&e0, &e1);
    if (e0) cudaEventRecord(e0, st);
    const int rc = dispatch(p, precision, shape.fpt, prm, nblocks, shape.warps, st, tail.part ? &tail : nullptr);
    if (e1) cudaEventRecord(e1, st);
    return rc < 0 ? fail(FREDEC_EINVAL, "kernel dispatch failed") : rc;
}

}  // namespace fredec
