// ctx.cu -- host side of libmt.so: the context, argument checks, device
// buffers, the Metropolis super-step as a CUDA graph, and the C ABI of
// include/mt.h.  No step of the path runs on the host; each is one of the
// kernels in data.cu, march_*.cu, mcmc.cu, adjoint.cu, copula.cu, linear.cu
// and diag.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

namespace mt {
template <int MODE>
cudaError_t launch_march_mode(const Prob &, HRef, int, int, size_t, void *, double *, double *,
                              cudaStream_t);
cudaError_t launch_accept_fused(const Prob &pb, int mode, int n_chains, const void *partial,
                                const double *lp_prop, const double *extra, double *ll,
                                double *lp, double *ll_prop_out, uint8_t *cur, uint8_t *prop_sel,
                                int64_t *accepts, int32_t *acc_last, double *logu_out,
                                uint64_t seed, const int64_t *step_base, int step_off,
                                cudaStream_t st, double *alpha_out = nullptr);
size_t nodes_bytes_f64(int L, int N);

int march_rays_per_block(const Prob &pb)
{
    // up to MT_RAYS_PER_CTA rays per CTA (8 per thread of the FP32 modes'
    // 768-thread CTAs); small problems use fewer.
    const int per = MT_RAYS_PER_CTA;
    const int need = ((pb.n_rays + 255) / 256) * 256;
    return need < per ? need : per;
}

size_t march_smem_bytes(const Prob &pb, int mode)
{
    // FP32 modes: one plane of (h, dx) float pairs per surface
    if (is_dx_mode(mode)) return (size_t)8 * pb.L * pb.N;
    const int es = mode == MODE_F64 ? 8 : 2;
    const int raw = pb.L * es;
    const int bytes = raw <= 4 ? 4 : raw <= 8 ? 8 : ((raw + 15) / 16) * 16;
    return (size_t)bytes * pb.N;
}

bool march_fits_smem(const Prob &pb, int mode)
{
    return march_smem_bytes(pb, mode) + MT_SMEM_STATIC <= MT_MAX_SMEM;
}

size_t march_phased_smem_bytes(const Prob &pb)
{
    // one surface's (h, dx) plane and a float-float sum per ray slot
    return (size_t)8 * pb.N + (size_t)8 * march_rays_per_block(pb);
}

bool march_fits_phased(const Prob &pb, int mode)
{
    return is_dx_mode(mode) && march_phased_smem_bytes(pb) + MT_SMEM_STATIC <= MT_MAX_SMEM;
}

cudaError_t launch_march(const Prob &pb, int mode, HRef h, int n_chains, void *partial,
                         double *ray_O, double *ray_term, cudaStream_t st)
{
    const int rpb = march_rays_per_block(pb);
    const size_t smem = march_smem_bytes(pb, mode);
    switch (mode) {
        case MODE_F64:
            return launch_march_mode<MODE_F64>(pb, h, n_chains, rpb, smem, partial, ray_O, ray_term, st);
        case MODE_F32:
            return launch_march_mode<MODE_F32>(pb, h, n_chains, rpb, smem, partial, ray_O, ray_term, st);
        case MODE_F32C:
            return launch_march_mode<MODE_F32C>(pb, h, n_chains, rpb, smem, partial, ray_O, ray_term, st);
        case MODE_BF16:
            return launch_march_mode<MODE_BF16>(pb, h, n_chains, rpb, smem, partial, ray_O, ray_term, st);
        case MODE_F32A:
            return launch_march_mode<MODE_F32A>(pb, h, n_chains, rpb, smem, partial, ray_O, ray_term, st);
    }
    return cudaErrorInvalidValue;
}
}  // namespace mt

using namespace mt;

struct EvPair {
    cudaEvent_t a, b;
};

struct mt_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaMemPool_t pool = nullptr;    // a server's stream-ordered pool (nullptr: cudaMalloc)
    bool own_stream = false;
    mt_config cfg{};
    int mode = MODE_F32;
    std::string err;

    int L = 0, R = 0, Q = 0, S = 0, P = 0;
    double box[3] = {0, 0, 0};
    std::vector<double> rho, mu;
    bool have_grid = false, have_sensors = false, have_pixels = false, have_counts = false;
    Prob pb{};

    double *d_mu = nullptr, *d_sensors = nullptr, *d_dirs = nullptr;
    float2 *d_muff = nullptr;        // float-float prior mean (FP32-mode prior)
    float4 *d_o4 = nullptr, *d_s4 = nullptr;
    float *d_kz0 = nullptr;
    float4 *d_xa4 = nullptr, *d_xb4 = nullptr;  // ray table of the FP32 march
    int2 *d_xc2 = nullptr;
    float *d_kz1 = nullptr;
    float *d_kzm = nullptr;   // z in metres of the FP32 march
    float2 *d_szm = nullptr;
    float psi_kc = 0.f;              // calibrated logistic correction (kappa * 2^-28)
    double *d_od = nullptr, *d_sd = nullptr, *d_dt = nullptr, *d_a = nullptr, *d_sumK = nullptr;
    float2 *d_dtff = nullptr, *d_aff = nullptr;
    int32_t *d_cnt = nullptr;
    int *d_flag = nullptr;
    int *d_perm = nullptr;           // march order of the rays

    int C = 0;
    uint64_t seed = 0;
    void *d_H = nullptr;  // [2][C][n]
    uint8_t *d_cur = nullptr, *d_psel = nullptr;
    double *d_ll = nullptr, *d_lp = nullptr, *d_llp = nullptr, *d_lpp = nullptr, *d_logu = nullptr;
    int64_t *d_acc = nullptr, *d_step = nullptr;
    int32_t *d_accl = nullptr;
    double *d_G = nullptr;           // [2][C][n] log-posterior gradients (MALA)
    bool g_valid = false;            // d_G[cur] holds the current states' gradients
    double *d_extra = nullptr;       // [C] Hastings terms
    void *d_gacc = nullptr;          // adjoint fixed-point accumulators
    size_t gacc_cap = 0;
    void *d_dO = nullptr;            // per-ray d ll / d O_p of gradient evaluations
    size_t dO_cap = 0;
    void *d_tmp = nullptr;           // small per-chain scratch
    size_t tmp_cap = 0;
    void *d_diag = nullptr;          // diagnostics scratch
    size_t diag_cap = 0;
    bool linear = false;             // linearised forward model instead of the march
    int lin_nz = 0;
    std::vector<double> lin_href;    // reference heights of the linearisation
    int *d_lrow = nullptr, *d_lcol = nullptr;  // voxel path lengths (CSR by ray)
    int *d_lcptr = nullptr, *d_lcrow = nullptr;  // the same by voxel (CSC), for gradients
    void *d_lcval = nullptr, *d_fO = nullptr, *d_gcell = nullptr;
    size_t fO_cap = 0, gcell_cap = 0;
    void *d_lval = nullptr, *d_R0 = nullptr, *d_dR = nullptr;  // d_R0: reference voxel densities
    double *d_fine = nullptr;        // linearised model: fine-block partial sums
    size_t fine_cap = 0;
    size_t dR_cap = 0;
    double *d_lam0 = nullptr, *d_amc = nullptr;
    int hmc_leap = 8;                // leapfrog steps per HMC proposal
    int nuts_depth = 8;              // capped NUTS: 2^depth - 1 leapfrog steps
    NutsBufs nuts{};
    // step-size adaptation of MALA / HMC (mt_set_adapt): target acceptance,
    // number of adapted steps (0 = off), state not yet initialised
    double adapt_target = 0.8;
    int adapt_n = 0;
    bool adapt_pending = false;
    double *d_eps = nullptr, *d_da = nullptr, *d_alpha = nullptr;
    // diagonal inverse metric of HMC adapted in the same warm-up
    // (mt_set_metric_adapt): Welford mean / M2 and the metric, [C][n] each
    bool metric_on = false;
    double metric_shrink = 1e-3;
    double *d_minv = nullptr, *d_wmean = nullptr, *d_wm2 = nullptr;
    double *d_P = nullptr;           // HMC momentum [C][n]
    double *d_Q64 = nullptr;         // HMC trajectory position in FP64 [C][n]
    double *d_k0 = nullptr;          // HMC initial kinetic energy [C]
    bool copula = false;             // copula prior: chain states are latents (z, r)
    void *d_terr = nullptr;          // copula prior: terrain (top surface), mode dtype
    void *d_Hd = nullptr;            // copula prior: heights derived from latents
    size_t hd_cap = 0;

    void *d_part = nullptr;
    size_t part_cap = 0;
    void *d_nodes = nullptr;         // HBM node records for large grids
    size_t nodes_cap = 0;
    void *d_in = nullptr;
    size_t in_cap = 0;
    void *d_out = nullptr;
    size_t out_cap = 0;
    void *d_out2 = nullptr;
    size_t out2_cap = 0;

    cudaGraphExec_t gexec = nullptr;
    int g_kernel = -1, g_nw = 0, g_C = 0;
    double g_step = 0.0;

    bool timing = false;
    unsigned long long *d_work = nullptr;  // evaluated surface-samples (timing mode)
    double work_total = 0.0;               // surface-samples of the method in timed launches
    std::vector<EvPair> ev_open[2];
    std::vector<cudaEvent_t> ev_pool;
    double t_ms[2] = {0, 0};
    int64_t t_n[2] = {0, 0};
};

static thread_local std::string g_create_err;

static mt_status fail(mt_ctx *ctx, mt_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    else g_create_err = buf;
    return st;
}

#define CK(ctx, x)                                                                           \
    do {                                                                                     \
        cudaError_t e_ = (x);                                                                \
        if (e_ != cudaSuccess) {                                                             \
            cudaGetLastError();                                                              \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? MT_ENOMEM : MT_ECUDA, "%s: %s", \
                        #x, cudaGetErrorString(e_));                                         \
        }                                                                                    \
    } while (0)

#define TRY(x)                          \
    do {                                \
        mt_status s_ = (x);             \
        if (s_ != MT_OK) return s_;     \
    } while (0)

static bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device memory of a context: from the server's stream-ordered pool when the
// context belongs to a server (allocation and release are ordered on the
// context's stream, and neither goes to the driver nor synchronises the
// device), otherwise cudaMalloc / cudaFree.
static cudaError_t dev_alloc(mt_ctx *ctx, void **p, size_t bytes)
{
    if (ctx->pool) return cudaMallocFromPoolAsync(p, bytes, ctx->pool, ctx->stream);
    return cudaMalloc(p, bytes);
}

static void dev_free(mt_ctx *ctx, void *p)
{
    if (!p) return;
    if (ctx->pool) cudaFreeAsync(p, ctx->stream);
    else cudaFree(p);
}

template <typename T> static void dfree(mt_ctx *ctx, T *&p)
{
    dev_free(ctx, (void *)p);
    p = nullptr;
}

static mt_status grow(mt_ctx *ctx, void **p, size_t *cap, size_t bytes)
{
    if (bytes <= *cap && *p) return MT_OK;
    if (*p) dev_free(ctx, *p);
    *p = nullptr;
    *cap = 0;
    size_t want = bytes < 256 ? 256 : bytes;
    CK(ctx, dev_alloc(ctx, (void **)p, want));
    *cap = want;
    return MT_OK;
}

template <typename T> static mt_status dalloc(mt_ctx *ctx, T **p, size_t n)
{
    dfree(ctx, *p);
    CK(ctx, dev_alloc(ctx, (void **)p, n * sizeof(T) + 16));
    return MT_OK;
}

static size_t elem_size(const mt_ctx *ctx) { return ctx->mode == MODE_F64 ? 8 : 4; }
static size_t n_per_chain(const mt_ctx *ctx) { return (size_t)ctx->L * ctx->R * ctx->Q; }

static void drop_graph(mt_ctx *ctx)
{
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
    ctx->g_kernel = -1;
}

static void drop_chains(mt_ctx *ctx)
{
    drop_graph(ctx);
    dfree(ctx, ctx->d_H);
    dfree(ctx, ctx->d_cur);
    dfree(ctx, ctx->d_psel);
    dfree(ctx, ctx->d_ll);
    dfree(ctx, ctx->d_lp);
    dfree(ctx, ctx->d_llp);
    dfree(ctx, ctx->d_lpp);
    dfree(ctx, ctx->d_logu);
    dfree(ctx, ctx->d_acc);
    dfree(ctx, ctx->d_accl);
    dfree(ctx, ctx->d_G);
    dfree(ctx, ctx->d_extra);
    dfree(ctx, ctx->d_P);
    dfree(ctx, ctx->d_Q64);
    dfree(ctx, ctx->d_k0);
    dfree(ctx, ctx->d_eps);
    dfree(ctx, ctx->d_da);
    dfree(ctx, ctx->d_alpha);
    dfree(ctx, ctx->d_minv);
    dfree(ctx, ctx->d_wmean);
    dfree(ctx, ctx->d_wm2);
    for (double **p : {&ctx->nuts.qL, &ctx->nuts.pL, &ctx->nuts.gL, &ctx->nuts.qR, &ctx->nuts.pR,
                       &ctx->nuts.gR, &ctx->nuts.ph, &ctx->nuts.gsel, &ctx->nuts.gsub, &ctx->nuts.sc})
        dfree(ctx, *p);
    dfree(ctx, ctx->nuts.hsel);
    dfree(ctx, ctx->nuts.hsub);
    ctx->adapt_pending = ctx->adapt_n > 0;  // new chains adapt from the start
    ctx->g_valid = false;
    ctx->C = 0;
}

static void refresh_prob(mt_ctx *ctx)
{
    Prob &pb = ctx->pb;
    pb.L = ctx->L;
    pb.R = ctx->R;
    pb.Q = ctx->Q;
    pb.S = ctx->S;
    pb.P = ctx->P;
    pb.G = ctx->cfg.n_grid;
    pb.n_rays = ctx->S * ctx->P;
    pb.N = ctx->R * ctx->Q;
    for (int a = 0; a < 3; ++a) pb.box[a] = ctx->box[a];
    pb.gamma = ctx->cfg.gamma;
    pb.I0 = ctx->cfg.I0;
    pb.Lambda = ctx->cfg.atten;
    pb.inv_Lambda = 1.0 / ctx->cfg.atten;
    pb.tau = ctx->cfg.tau;
    pb.car_r = ctx->cfg.car_r;
    pb.delta = ctx->cfg.min_thick;
    pb.kg64 = ctx->cfg.gamma > 0.0 ? 1.4426950408889634074 / ctx->cfg.gamma : 1.0;
    pb.kg = (float)pb.kg64;
    pb.kgl = (float)(pb.kg64 - (double)pb.kg);
    // largest float below n - 3/2 by 8 ulps: keeps the cell index <= n - 2
    auto hi = [](int n) {
        float v = (float)n - 1.5f;
        for (int i = 0; i < 8; ++i) v = nextafterf(v, -INFINITY);
        return v;
    };
    pb.gm_hi_x = hi(ctx->Q);
    pb.gm_hi_y = hi(ctx->R);
    if (!ctx->rho.empty()) {
        pb.rho_top = ctx->rho[ctx->L];
        for (int l = 0; l < MT_MAX_L; ++l) {
            pb.drho[l] = l < ctx->L ? ctx->rho[l] - ctx->rho[l + 1] : 0.0;
            pb.drho_f[l] = (float)pb.drho[l];
            pb.drho_ff[l] = make_float2(pb.drho_f[l], (float)(pb.drho[l] - (double)pb.drho_f[l]));
        }
    }
    // Reference height per surface for the FP32 paths: the mean prior height
    // (or evenly spaced levels when the prior mean is all zero), as a float.
    const size_t N = (size_t)ctx->R * ctx->Q;
    for (int l = 0; l < MT_MAX_L; ++l) {
        double m = 0.0;
        if (l < ctx->L && ctx->mu.size() >= (l + 1) * N) {
            for (size_t i = 0; i < N; ++i) m += ctx->mu[l * N + i];
            m /= (double)N;
            if (m == 0.0) m = ctx->box[2] * (l + 1) / (ctx->L + 1);
        }
        pb.ref[l] = (float)m;
    }
    pb.kz0 = ctx->d_kz0;
    // Grid of the march's z high parts (log2 units): 2^(e - 24) with 2^e above
    // twice the largest kg64 * |z - ref_l| a sample can have, so that
    // hi + k * step_hi (each off the exact value by at most half a grid step
    // per term, k < G) stays below 2^e and is exact in FP32.
    {
        double rmax = 0.0;
        for (int l = 0; l < ctx->L && l < MT_MAX_L; ++l) rmax = fmax(rmax, fabs((double)pb.ref[l]));
        const double bound = 2.0 * (pb.kg64 * (ctx->box[2] + rmax) + 1.0);
        pb.zgrid = ldexp(1.0, ilogb(bound) + 1 - 24);
        const double bound_m = 2.0 * (ctx->box[2] + rmax + 1.0);
        pb.zgrid_m = ldexp(1.0, ilogb(bound_m) + 1 - 24);
    }
    pb.xa4 = ctx->d_xa4;
    pb.xb4 = ctx->d_xb4;
    pb.xc2 = ctx->d_xc2;
    pb.kz1 = ctx->d_kz1;
    pb.kzm = ctx->d_kzm;
    pb.szm = ctx->d_szm;
    pb.psi_kc = ctx->psi_kc;
    pb.mu_ff = ctx->d_muff;
    pb.lz_f = (float)ctx->box[2];
    if ((double)pb.lz_f > ctx->box[2]) pb.lz_f = nextafterf(pb.lz_f, -INFINITY);
    pb.delta_ff = make_float2((float)ctx->cfg.min_thick,
                              (float)(ctx->cfg.min_thick - (double)(float)ctx->cfg.min_thick));
    pb.perm = ctx->d_perm;
    pb.gnodes = nullptr;  // set per launch by ensure_nodes when the grid needs it
    pb.dO = nullptr;      // set in the copies that gradient launches use
    pb.flag = ctx->d_flag;
    pb.work = ctx->timing ? ctx->d_work : nullptr;
    pb.o4 = ctx->d_o4;
    pb.s4 = ctx->d_s4;
    pb.o_d = ctx->d_od;
    pb.s_d = ctx->d_sd;
    pb.dt = ctx->d_dt;
    pb.a = ctx->d_a;
    pb.a_ff = ctx->d_aff;
    pb.dt_ff = ctx->d_dtff;
    pb.cnt = ctx->d_cnt;
    const double grho = (double)pb.G * pb.rho_top;
    pb.grho_ff = make_float2((float)grho, (float)(grho - (double)(float)grho));
    const double il = pb.inv_Lambda;
    pb.invL_ff = make_float2((float)il, (float)(il - (double)(float)il));
}

static mt_status need(mt_ctx *ctx, bool counts)
{
    if (!ctx) return fail(nullptr, MT_EINVAL, "null context");
    if (!ctx->have_grid) return fail(ctx, MT_ESTATE, "mt_set_grid has not been called");
    if (!ctx->have_sensors) return fail(ctx, MT_ESTATE, "mt_set_sensors has not been called");
    if (!ctx->have_pixels) return fail(ctx, MT_ESTATE, "mt_set_pixels has not been called");
    if (counts && !ctx->have_counts)
        return fail(ctx, MT_ESTATE, "no observed counts: call mt_set_counts or mt_generate_data");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return fail(ctx, MT_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return MT_OK;
}

static mt_status build_raytab(mt_ctx *ctx)
{
    if (!(ctx->have_grid && ctx->have_sensors && ctx->have_pixels)) return MT_OK;
    const size_t n = (size_t)ctx->S * ctx->P;
    TRY(dalloc(ctx, &ctx->d_o4, n));
    TRY(dalloc(ctx, &ctx->d_s4, n));
    TRY(dalloc(ctx, &ctx->d_kz0, 2 * (size_t)ctx->L * n));
    TRY(dalloc(ctx, &ctx->d_xa4, n));
    TRY(dalloc(ctx, &ctx->d_xb4, n));
    TRY(dalloc(ctx, &ctx->d_xc2, n));
    TRY(dalloc(ctx, &ctx->d_kz1, 2 * (size_t)ctx->L * n));
    TRY(dalloc(ctx, &ctx->d_kzm, 2 * (size_t)ctx->L * n));
    TRY(dalloc(ctx, &ctx->d_szm, n));
    TRY(dalloc(ctx, &ctx->d_od, 3 * n));
    TRY(dalloc(ctx, &ctx->d_sd, 3 * n));
    TRY(dalloc(ctx, &ctx->d_dt, n));
    TRY(dalloc(ctx, &ctx->d_dtff, n));
    TRY(dalloc(ctx, &ctx->d_perm, n));
    refresh_prob(ctx);
    CK(ctx, launch_raytab(ctx->pb, ctx->d_sensors, ctx->d_dirs, ctx->d_o4, ctx->d_s4, ctx->d_kz0,
                          ctx->d_od, ctx->d_sd, ctx->d_dt, ctx->d_dtff, ctx->d_flag, ctx->stream));
    CK(ctx, launch_raytab_march(ctx->pb, ctx->d_sensors, ctx->d_dirs, ctx->d_xa4, ctx->d_xb4, ctx->d_xc2,
                                ctx->d_kz1, ctx->d_kzm, ctx->d_szm, ctx->d_flag, ctx->stream));
    if (ctx->mode == MODE_F32A) {
        // the approximate logistic's mean error, calibrated once per context on its device
        double *d_k = nullptr, kappa = 0.0;
        TRY(dalloc(ctx, &d_k, 1));
        CK(ctx, launch_psi_calib(d_k, ctx->stream));
        CK(ctx, cudaMemcpyAsync(&kappa, d_k, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        dfree(ctx, d_k);
        if (!(fabs(kappa) < 1e-5)) return fail(ctx, MT_ECUDA, "logistic calibration out of range: %g", kappa);
        ctx->psi_kc = (float)(kappa * 0x1p-28);
        ctx->pb.psi_kc = ctx->psi_kc;
    }
    // March order: rays sorted by their vertical step per sample, then by the
    // height of their first sample (ties by ray index).  A surface's sample
    // window depends on those two numbers only, so a warp's 32 rays then run
    // loops of near-equal length.
    std::vector<float4> s4(n);
    std::vector<float> z0(n);
    CK(ctx, cudaMemcpyAsync(s4.data(), ctx->d_s4, n * sizeof(float4), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaMemcpyAsync(z0.data(), ctx->d_kz0, n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    std::vector<int> perm(n);
    for (size_t i = 0; i < n; ++i) perm[i] = (int)i;
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) {
        if (s4[a].z != s4[b].z) return s4[a].z < s4[b].z;
        return z0[a] < z0[b];
    });
    CK(ctx, cudaMemcpyAsync(ctx->d_perm, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MT_OK;
}

static mt_status eval_logpost(mt_ctx *ctx, HRef h, int n, double *d_ll, double *d_lp);

static mt_status counts_ready(mt_ctx *ctx)
{
    const size_t n = (size_t)ctx->S * ctx->P;
    TRY(dalloc(ctx, &ctx->d_a, n));
    TRY(dalloc(ctx, &ctx->d_aff, n));
    if (!ctx->d_sumK) TRY(dalloc(ctx, &ctx->d_sumK, 1));
    refresh_prob(ctx);
    CK(ctx, launch_counts_prep(ctx->pb, ctx->d_a, ctx->d_aff, ctx->d_sumK, ctx->stream));
    double sk = 0.0;
    CK(ctx, cudaMemcpyAsync(&sk, ctx->d_sumK, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->have_counts = true;
    refresh_prob(ctx);
    ctx->pb.sumK = sk;
    if (ctx->linear)
        CK(ctx, launch_lin_amc(ctx->pb.n_rays, ctx->d_lam0, ctx->d_cnt, ctx->d_amc, ctx->stream));
    drop_graph(ctx);
    ctx->g_valid = false;
    if (ctx->C > 0) {  // live chains: their log-likelihoods refer to the old counts
        const size_t np = n_per_chain(ctx);
        HRef h{ctx->d_H, (long long)np, ctx->d_cur, (long long)(ctx->C * np), 0};
        TRY(eval_logpost(ctx, h, ctx->C, ctx->d_ll, ctx->d_lp));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return MT_OK;
}

// Device view of a caller array of `bytes`: the pointer itself when it is
// device memory, else a copy in the staging buffer `slot`.
static mt_status dev_in(mt_ctx *ctx, const void *p, size_t bytes, const void **out)
{
    if (is_device_ptr(p)) {
        *out = p;
        return MT_OK;
    }
    TRY(grow(ctx, &ctx->d_in, &ctx->in_cap, bytes));
    CK(ctx, cudaMemcpyAsync(ctx->d_in, p, bytes, cudaMemcpyHostToDevice, ctx->stream));
    *out = ctx->d_in;
    return MT_OK;
}

// Output target: device pointer as is, host pointer via a staging buffer.
struct OutBuf {
    void *user = nullptr;
    void *dev = nullptr;
    size_t bytes = 0;
    bool host = false;
};

static mt_status dev_out(mt_ctx *ctx, void *p, size_t bytes, void **slot, size_t *cap, OutBuf *o)
{
    o->user = p;
    o->bytes = bytes;
    if (!p) {
        o->dev = nullptr;
        return MT_OK;
    }
    if (is_device_ptr(p)) {
        o->dev = p;
        o->host = false;
        return MT_OK;
    }
    TRY(grow(ctx, slot, cap, bytes));
    o->dev = *slot;
    o->host = true;
    return MT_OK;
}

static mt_status finish_out(mt_ctx *ctx, OutBuf *o)
{
    if (o->user && o->host)
        CK(ctx, cudaMemcpyAsync(o->user, o->dev, o->bytes, cudaMemcpyDeviceToHost, ctx->stream));
    return MT_OK;
}

static mt_status ensure_nodes(mt_ctx *ctx, int n);

static mt_status ensure_partials(mt_ctx *ctx, int n_chains)
{
    const int rpb = march_rays_per_block(ctx->pb);
    const size_t n_blk = (ctx->pb.n_rays + rpb - 1) / rpb;
    void *old = ctx->d_part;
    TRY(grow(ctx, &ctx->d_part, &ctx->part_cap, n_blk * (size_t)n_chains * 8));
    if (ctx->d_part != old) drop_graph(ctx);  // a captured graph holds the old pointer
    return ensure_nodes(ctx, n_chains);
}

// Grids whose planes exceed shared memory run the FP32 modes one surface's
// plane at a time (k_march_phased) or, when not even one plane and the
// rays' sums fit, from records in HBM (see k_stage_dx_global); the other
// modes need their records to fit.
static bool use_global_nodes(const mt_ctx *ctx)
{
    return !march_fits_smem(ctx->pb, ctx->mode) && !march_fits_phased(ctx->pb, ctx->mode) &&
           is_dx_mode(ctx->mode);
}

static mt_status check_smem(mt_ctx *ctx)
{
    const size_t smem = march_smem_bytes(ctx->pb, ctx->mode);
    if (!march_fits_smem(ctx->pb, ctx->mode) && !march_fits_phased(ctx->pb, ctx->mode) && !use_global_nodes(ctx))
        return fail(ctx, MT_EINVAL,
                    "surfaces need %zu bytes of shared memory per block (limit %d): use "
                    "MT_PREC_F32 (records in HBM) or a smaller grid",
                    smem, MT_MAX_SMEM - MT_SMEM_STATIC);
    return MT_OK;
}

// HBM node records for n chains when the grid is too large for shared memory.
static mt_status ensure_nodes(mt_ctx *ctx, int n)
{
    if (!use_global_nodes(ctx)) {
        ctx->pb.gnodes = nullptr;
        return MT_OK;
    }
    void *old = ctx->d_nodes;
    TRY(grow(ctx, &ctx->d_nodes, &ctx->nodes_cap, march_smem_bytes(ctx->pb, ctx->mode) * (size_t)n));
    if (ctx->d_nodes != old) drop_graph(ctx);
    ctx->pb.gnodes = (float *)ctx->d_nodes;
    return MT_OK;
}

static cudaEvent_t ev_get(mt_ctx *ctx)
{
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launch-time bookkeeping of the method's work for mt_get_work.
static void count_work(mt_ctx *ctx, int n_chains)
{
    ctx->work_total += (double)n_chains * ctx->pb.n_rays * ctx->pb.G * ctx->pb.L;
}

static void ev_begin(mt_ctx *ctx, int id, EvPair *p)
{
    p->a = ev_get(ctx);
    p->b = ev_get(ctx);
    cudaEventRecord(p->a, ctx->stream);
}
static void ev_end(mt_ctx *ctx, int id, EvPair *p)
{
    cudaEventRecord(p->b, ctx->stream);
    ctx->ev_open[id].push_back(*p);
}

// log-likelihood + log-prior of n chains given by h, into device arrays.
// Heights buffer for n chains' derived heights (copula prior).
static mt_status ensure_derived(mt_ctx *ctx, int n)
{
    void *old = ctx->d_Hd;
    TRY(grow(ctx, &ctx->d_Hd, &ctx->hd_cap, (size_t)n * n_per_chain(ctx) * elem_size(ctx)));
    if (ctx->d_Hd != old) drop_graph(ctx);  // a captured graph holds the old pointer
    return MT_OK;
}

// Log-prior of n chain states h into d_lp (nullable), and the heights the ray
// kernel marches: the states themselves (CAR prior), or the heights derived
// from latent states (copula prior).
static mt_status prior_and_heights(mt_ctx *ctx, HRef h, int n, double *d_lp, HRef *hm)
{
    if (!ctx->copula) {
        if (d_lp) CK(ctx, launch_prior(ctx->pb, ctx->mode, h, ctx->d_mu, n, d_lp, ctx->stream));
        *hm = h;
        return MT_OK;
    }
    if (d_lp) CK(ctx, launch_prior_latent(ctx->pb, ctx->mode, h, n, d_lp, ctx->stream));
    TRY(ensure_derived(ctx, n));
    CK(ctx, launch_copula(ctx->pb, ctx->mode, h, ctx->d_terr, ctx->d_Hd, n, ctx->stream));
    *hm = HRef{ctx->d_Hd, (long long)n_per_chain(ctx), nullptr, 0, 0};
    return MT_OK;
}

// Storage format of the per-CTA log-likelihood partials in d_part: the ray
// kernel's (the linearised model writes FP64 partials in every mode).
static int part_mode(const mt_ctx *ctx) { return ctx->linear ? MODE_F32 : ctx->mode; }

// Scratch of the linearised model for n chains (dR, [voxels][n padded to 32]).
static mt_status ensure_lin(mt_ctx *ctx, int n)
{
    if (!ctx->linear) return MT_OK;
    const size_t nvox = (size_t)ctx->lin_nz * (ctx->R - 1) * (ctx->Q - 1);
    const size_t Cp = ((size_t)n + 31) / 32 * 32;
    void *old = ctx->d_dR, *old_f = ctx->d_fine;
    TRY(grow(ctx, &ctx->d_dR, &ctx->dR_cap, nvox * Cp * elem_size(ctx)));
    TRY(grow(ctx, (void **)&ctx->d_fine, &ctx->fine_cap, lin_fine_partials(ctx->pb, n) * 8));
    if (ctx->d_dR != old || (void *)ctx->d_fine != old_f) drop_graph(ctx);
    return MT_OK;
}

// The per-(chain, CTA) log-likelihood partials of n chains' heights h:
// the march, or the linearised model.
static mt_status ray_kernel(mt_ctx *ctx, HRef h, int n)
{
    if (ctx->linear) {
        TRY(ensure_lin(ctx, n));
        CK(ctx, launch_lin(ctx->pb, ctx->mode, h, n, ctx->lin_nz, ctx->d_lrow, ctx->d_lcol, ctx->d_lval,
                           ctx->d_R0, ctx->d_dR, ctx->d_lam0, ctx->d_amc, ctx->d_fine,
                           (double *)ctx->d_part, ctx->stream));
        return MT_OK;
    }
    CK(ctx, launch_march(ctx->pb, ctx->mode, h, n, ctx->d_part, nullptr, nullptr, ctx->stream));
    return MT_OK;
}

static mt_status eval_logpost(mt_ctx *ctx, HRef h, int n, double *d_ll, double *d_lp)
{
    TRY(ensure_partials(ctx, n));
    TRY(prior_and_heights(ctx, h, n, d_lp, &h));
    if (d_ll) {
        EvPair ep;
        if (ctx->timing) {
            ev_begin(ctx, 0, &ep);
            count_work(ctx, n);
        }
        TRY(ray_kernel(ctx, h, n));
        if (ctx->timing) ev_end(ctx, 0, &ep);
        CK(ctx, launch_reduce_ll(ctx->pb, ctx->linear ? MODE_F32 : ctx->mode, n, ctx->d_part, d_ll,
                                 ctx->stream));
    }
    return MT_OK;
}

namespace mt {
mt_status ctx_view(mt_ctx *ctx, CtxView *v)
{
    TRY(need(ctx, true));
    if (ctx->copula)
        return fail(ctx, MT_EINVAL, "the copula prior derives heights into a library buffer; use mt_logpost");
    if (ctx->linear)
        return fail(ctx, MT_EINVAL, "the linearised model needs a library buffer; use mt_logpost");
    v->pb = ctx->pb;
    v->mode = ctx->mode;
    v->device = ctx->device;
    v->mu = ctx->d_mu;
    v->stream = ctx->stream;
    return MT_OK;
}

mt_status ctx_fail(mt_ctx *ctx, mt_status st, const char *msg) { return fail(ctx, st, "%s", msg); }
}  // namespace mt

// Buffers of a gradient evaluation of n chains: fixed-point accumulators and
// the per-ray d ll / d O_p.
static mt_status ensure_grad_bufs(mt_ctx *ctx, int n)
{
    const size_t np = n_per_chain(ctx);
    void *old_g = ctx->d_gacc, *old_d = ctx->d_dO;
    TRY(grow(ctx, &ctx->d_gacc, &ctx->gacc_cap, (size_t)n * np * 8));
    TRY(grow(ctx, &ctx->d_dO, &ctx->dO_cap, (size_t)n * (ctx->pb.n_rays + 1) * 4));  // + the adjoint's units
    if (ctx->d_gacc != old_g || ctx->d_dO != old_d) drop_graph(ctx);
    if (ctx->linear) {  // d ll / d O per ray and the per-cell gradients, chains padded to 32
        const size_t Cp = ((size_t)n + 31) / 32 * 32, es = elem_size(ctx);
        const size_t ncell = (size_t)(ctx->R - 1) * (ctx->Q - 1);
        void *of = ctx->d_fO, *oc = ctx->d_gcell;
        TRY(grow(ctx, &ctx->d_fO, &ctx->fO_cap, (size_t)ctx->pb.n_rays * Cp * es));
        TRY(grow(ctx, &ctx->d_gcell, &ctx->gcell_cap, (size_t)ctx->L * ncell * Cp * es));
        if (ctx->d_fO != of || ctx->d_gcell != oc) drop_graph(ctx);
    }
    return MT_OK;
}

// Forward march (log-likelihood partials and each ray's d ll / d O_p) and the
// adjoint's scatter into the zeroed accumulators, for n chains given by h.
static mt_status enqueue_forward_adjoint(mt_ctx *ctx, HRef h, int n)
{
    if (ctx->linear) {  // the linearised model and its gradient
        TRY(ensure_lin(ctx, n));
        CK(ctx, launch_lin(ctx->pb, ctx->mode, h, n, ctx->lin_nz, ctx->d_lrow, ctx->d_lcol, ctx->d_lval,
                           ctx->d_R0, ctx->d_dR, ctx->d_lam0, ctx->d_amc, ctx->d_fine, (double *)ctx->d_part,
                           ctx->stream, ctx->d_fO));
        CK(ctx, launch_lin_grad(ctx->pb, ctx->mode, h, n, ctx->lin_nz, ctx->d_lcptr, ctx->d_lcrow, ctx->d_lcval,
                                ctx->d_fO, ctx->d_dR, ctx->d_gcell, (unsigned long long *)ctx->d_gacc,
                                ctx->stream));
        return MT_OK;
    }
    Prob pg = ctx->pb;
    pg.dO = (float *)ctx->d_dO;
    pg.work = nullptr;
    CK(ctx, cudaMemsetAsync(ctx->d_gacc, 0, (size_t)n * n_per_chain(ctx) * 8, ctx->stream));
    CK(ctx, launch_march(pg, ctx->mode, h, n, ctx->d_part, nullptr, nullptr, ctx->stream));
    CK(ctx, launch_adjoint(pg, h, n, (unsigned long long *)ctx->d_gacc, ctx->stream));
    return MT_OK;
}

// Gradient of the log-posterior (and its value) of n chains given by h, into
// device arrays grad [n][L][R][Q] and (nullable) ll / lp.  FP32 arithmetic.
static mt_status eval_grad(mt_ctx *ctx, HRef h, int n, double *d_grad, double *d_ll, double *d_lp)
{
    TRY(ensure_grad_bufs(ctx, n));
    TRY(ensure_partials(ctx, n));
    if (ctx->copula) {  // latents: heights from the transform, the gradient back through it
        HRef hh;
        TRY(prior_and_heights(ctx, h, n, d_lp, &hh));
        TRY(enqueue_forward_adjoint(ctx, hh, n));
        if (d_ll) CK(ctx, launch_reduce_ll(ctx->pb, part_mode(ctx), n, ctx->d_part, d_ll, ctx->stream));
        CK(ctx, launch_copula_vjp(ctx->pb, h, hh, ctx->d_terr, (const unsigned long long *)ctx->d_gacc, d_grad,
                                  nullptr, n, ctx->stream));
        return MT_OK;
    }
    TRY(enqueue_forward_adjoint(ctx, h, n));
    if (d_ll) CK(ctx, launch_reduce_ll(ctx->pb, part_mode(ctx), n, ctx->d_part, d_ll, ctx->stream));
    if (d_lp) CK(ctx, launch_prior(ctx->pb, ctx->mode, h, ctx->d_mu, n, d_lp, ctx->stream));
    CK(ctx, launch_grad_finish(ctx->pb, ctx->mode, h, ctx->d_mu, n,
                               (const unsigned long long *)ctx->d_gacc, d_grad, ctx->stream));
    return MT_OK;
}

static mt_status grad_ok(mt_ctx *ctx)
{
    if (ctx->copula && copula_vjp_smem_bytes(ctx->pb) + MT_SMEM_STATIC > MT_MAX_SMEM)
        return fail(ctx, MT_EINVAL, "grid too large for the copula transform's reverse pass");
    if (ctx->mode == MODE_F64)
        return fail(ctx, MT_EINVAL, "the adjoint computes in FP32: use an FP32 precision mode");
    if (adjoint_smem_bytes(ctx->pb, false) + MT_SMEM_STATIC > MT_MAX_SMEM)
        return fail(ctx, MT_EINVAL, "grid too large for the adjoint's shared-memory surfaces");
    if (!(ctx->cfg.gamma > 0.0))
        return fail(ctx, MT_EINVAL, "the gradient needs gamma > 0 (the hard indicator is flat)");
    return MT_OK;
}

namespace mt {
mt_status ctx_view(mt_ctx *ctx, CtxView *v);
}

// ------------------------------------------------------------------ C ABI
extern "C" {

mt_status mt_create(mt_ctx **out, int device, const mt_config *cfg, void *cuda_stream)
{
    return mt::ctx_create_pooled(out, device, cfg, cuda_stream, nullptr);
}

}  // extern "C"

// A context whose device memory comes from `pool` (stream-ordered on its
// stream; the server's contexts) or from cudaMalloc (pool == nullptr).
mt_status mt::ctx_create_pooled(mt_ctx **out, int device, const mt_config *cfg, void *cuda_stream,
                                cudaMemPool_t pool)
{
    if (!out || !cfg) return fail(nullptr, MT_EINVAL, "mt_create: null argument");
    *out = nullptr;
    if (cfg->precision < MT_PREC_F64 || cfg->precision > MT_PREC_F32A)
        return fail(nullptr, MT_EINVAL, "mt_create: precision %d out of range", cfg->precision);
    if (cfg->n_grid < 1 || cfg->n_grid > (1 << 20))
        return fail(nullptr, MT_EINVAL, "mt_create: n_grid %d out of range", cfg->n_grid);
    if (!(cfg->gamma >= 0.0) || !(cfg->I0 > 0.0) || !(cfg->atten > 0.0) || !(cfg->tau >= 0.0) ||
        !(cfg->car_r >= 0.0 && cfg->car_r < 1.0) || !(cfg->min_thick > 0.0))
        return fail(nullptr, MT_EINVAL,
                    "mt_create: need gamma >= 0, I0 > 0, atten > 0, tau >= 0, 0 <= car_r < 1, "
                    "min_thick > 0");
    int n_dev = 0;
    cudaError_t e = cudaGetDeviceCount(&n_dev);
    if (e != cudaSuccess || device < 0 || device >= n_dev) {
        cudaGetLastError();
        return fail(nullptr, MT_ECUDA, "mt_create: no CUDA device %d (%s)", device,
                    cudaGetErrorString(e));
    }
    mt_ctx *ctx = new (std::nothrow) mt_ctx();
    if (!ctx) return fail(nullptr, MT_ENOMEM, "mt_create: out of host memory");
    ctx->device = device;
    ctx->pool = pool;
    ctx->cfg = *cfg;
    ctx->mode = cfg->precision;
    const char *fw = getenv("MT_FULL_WINDOWS");
    ctx->pb.full_windows = (fw && fw[0] && fw[0] != '0') ? 1 : 0;
    e = cudaSetDevice(device);
    if (e == cudaSuccess) {
        if (cuda_stream) {
            ctx->stream = (cudaStream_t)cuda_stream;
        } else {
            e = cudaStreamCreate(&ctx->stream);
            ctx->own_stream = e == cudaSuccess;
        }
    }
    if (e == cudaSuccess) e = dev_alloc(ctx, (void **)&ctx->d_flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = dev_alloc(ctx, (void **)&ctx->d_step, sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_step, 0, sizeof(int64_t), ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        mt_destroy(ctx);
        return fail(nullptr, MT_ECUDA, "mt_create: %s", cudaGetErrorString(e));
    }
    refresh_prob(ctx);
    *out = ctx;
    return MT_OK;
}

extern "C" {

mt_status mt_destroy(mt_ctx *ctx)
{
    if (!ctx) return MT_OK;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    drop_chains(ctx);
    dfree(ctx, ctx->d_mu);
    dfree(ctx, ctx->d_muff);
    dfree(ctx, ctx->d_sensors);
    dfree(ctx, ctx->d_dirs);
    dfree(ctx, ctx->d_o4);
    dfree(ctx, ctx->d_s4);
    dfree(ctx, ctx->d_kz0);
    dfree(ctx, ctx->d_xa4);
    dfree(ctx, ctx->d_xb4);
    dfree(ctx, ctx->d_xc2);
    dfree(ctx, ctx->d_kz1);
    dfree(ctx, ctx->d_kzm);
    dfree(ctx, ctx->d_szm);
    dfree(ctx, ctx->d_od);
    dfree(ctx, ctx->d_sd);
    dfree(ctx, ctx->d_dt);
    dfree(ctx, ctx->d_dtff);
    dfree(ctx, ctx->d_a);
    dfree(ctx, ctx->d_aff);
    dfree(ctx, ctx->d_sumK);
    dfree(ctx, ctx->d_cnt);
    dfree(ctx, ctx->d_flag);
    dfree(ctx, ctx->d_perm);
    dfree(ctx, ctx->d_step);
    dfree(ctx, ctx->d_work);
    if (ctx->d_part) dev_free(ctx, ctx->d_part);
    if (ctx->d_in) dev_free(ctx, ctx->d_in);
    if (ctx->d_out) dev_free(ctx, ctx->d_out);
    if (ctx->d_out2) dev_free(ctx, ctx->d_out2);
    if (ctx->d_gacc) dev_free(ctx, ctx->d_gacc);
    if (ctx->d_dO) dev_free(ctx, ctx->d_dO);
    if (ctx->d_diag) dev_free(ctx, ctx->d_diag);
    if (ctx->d_terr) dev_free(ctx, ctx->d_terr);
    if (ctx->d_lrow) dev_free(ctx, ctx->d_lrow);
    for (void *p : {(void *)ctx->d_lcptr, (void *)ctx->d_lcrow, ctx->d_lcval, ctx->d_fO, ctx->d_gcell})
        if (p) dev_free(ctx, p);
    if (ctx->d_lcol) dev_free(ctx, ctx->d_lcol);
    if (ctx->d_lval) dev_free(ctx, ctx->d_lval);
    if (ctx->d_R0) dev_free(ctx, ctx->d_R0);
    if (ctx->d_dR) dev_free(ctx, ctx->d_dR);
    if (ctx->d_lam0) dev_free(ctx, ctx->d_lam0);
    if (ctx->d_amc) dev_free(ctx, ctx->d_amc);
    if (ctx->d_fine) dev_free(ctx, ctx->d_fine);
    if (ctx->d_Hd) dev_free(ctx, ctx->d_Hd);
    if (ctx->d_nodes) dev_free(ctx, ctx->d_nodes);
    if (ctx->d_tmp) dev_free(ctx, ctx->d_tmp);
    for (int i = 0; i < 2; ++i)
        for (auto &p : ctx->ev_open[i]) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return MT_OK;
}

const char *mt_last_error(const mt_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

mt_status mt_set_grid(mt_ctx *ctx, int n_layers, int n_rows, int n_cols, const double box[3],
                      const double *unit_density, const double *prior_mean)
{
    if (!ctx) return fail(nullptr, MT_EINVAL, "null context");
    if (n_layers < 1 || n_layers > MT_MAX_L)
        return fail(ctx, MT_EINVAL, "n_layers %d not in [1, %d]", n_layers, MT_MAX_L);
    if (n_rows < 2 || n_cols < 2 || (long long)n_rows * n_cols > (1 << 22))
        return fail(ctx, MT_EINVAL, "grid %d x %d: each side must be >= 2", n_rows, n_cols);
    if (!box || !unit_density) return fail(ctx, MT_EINVAL, "null box or unit_density");
    for (int a = 0; a < 3; ++a)
        if (!(box[a] > 0.0)) return fail(ctx, MT_EINVAL, "box side %d must be > 0", a);
    for (int u = 0; u <= n_layers; ++u)
        if (!(unit_density[u] >= 0.0)) return fail(ctx, MT_EINVAL, "unit_density[%d] < 0", u);
    CK(ctx, cudaSetDevice(ctx->device));
    drop_chains(ctx);
    ctx->copula = false;
    ctx->linear = false;
    ctx->L = n_layers;
    ctx->R = n_rows;
    ctx->Q = n_cols;
    for (int a = 0; a < 3; ++a) ctx->box[a] = box[a];
    ctx->rho.assign(unit_density, unit_density + n_layers + 1);
    const size_t n = (size_t)n_layers * n_rows * n_cols;
    ctx->mu.assign(n, 0.0);
    if (prior_mean) ctx->mu.assign(prior_mean, prior_mean + n);
    TRY(dalloc(ctx, &ctx->d_mu, n));
    CK(ctx, cudaMemcpyAsync(ctx->d_mu, ctx->mu.data(), n * 8, cudaMemcpyHostToDevice, ctx->stream));
    std::vector<float2> muff(n);
    for (size_t i = 0; i < n; ++i) {
        const float hi = (float)ctx->mu[i];
        muff[i] = make_float2(hi, (float)(ctx->mu[i] - (double)hi));
    }
    TRY(dalloc(ctx, &ctx->d_muff, n));
    CK(ctx, cudaMemcpyAsync(ctx->d_muff, muff.data(), n * sizeof(float2), cudaMemcpyHostToDevice,
                            ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));  // muff is a local host buffer
    ctx->have_grid = true;
    ctx->have_counts = false;
    refresh_prob(ctx);
    TRY(check_smem(ctx));
    TRY(build_raytab(ctx));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MT_OK;
}

mt_status mt_set_sensors(mt_ctx *ctx, int n_sensors, const double *pos)
{
    if (!ctx) return fail(nullptr, MT_EINVAL, "null context");
    if (!ctx->have_grid) return fail(ctx, MT_ESTATE, "mt_set_grid first");
    if (n_sensors < 1 || !pos) return fail(ctx, MT_EINVAL, "need n_sensors >= 1 and positions");
    for (int s = 0; s < n_sensors; ++s)
        for (int a = 0; a < 3; ++a)
            if (!(pos[3 * s + a] > 0.0 && pos[3 * s + a] < ctx->box[a]))
                return fail(ctx, MT_EINVAL, "sensor %d is not strictly inside the box", s);
    CK(ctx, cudaSetDevice(ctx->device));
    drop_chains(ctx);
    ctx->linear = false;
    ctx->S = n_sensors;
    TRY(dalloc(ctx, &ctx->d_sensors, 3 * (size_t)n_sensors));
    CK(ctx, cudaMemcpyAsync(ctx->d_sensors, pos, 24 * (size_t)n_sensors, cudaMemcpyHostToDevice,
                            ctx->stream));
    ctx->have_sensors = true;
    ctx->have_counts = false;
    TRY(build_raytab(ctx));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MT_OK;
}

mt_status mt_set_pixels(mt_ctx *ctx, int n_pixels, const double *dirs)
{
    if (!ctx) return fail(nullptr, MT_EINVAL, "null context");
    if (!ctx->have_grid) return fail(ctx, MT_ESTATE, "mt_set_grid first");
    if (n_pixels < 1 || !dirs) return fail(ctx, MT_EINVAL, "need n_pixels >= 1 and directions");
    for (int p = 0; p < n_pixels; ++p) {
        const double *d = dirs + 3 * p;
        const double nn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (!(fabs(nn - 1.0) <= 1e-6))
            return fail(ctx, MT_EINVAL, "pixel %d direction is not a unit vector", p);
    }
    if ((long long)ctx->S * n_pixels > (1LL << 30))
        return fail(ctx, MT_EINVAL, "too many rays");
    CK(ctx, cudaSetDevice(ctx->device));
    drop_chains(ctx);
    ctx->linear = false;
    ctx->P = n_pixels;
    TRY(dalloc(ctx, &ctx->d_dirs, 3 * (size_t)n_pixels));
    CK(ctx, cudaMemcpyAsync(ctx->d_dirs, dirs, 24 * (size_t)n_pixels, cudaMemcpyHostToDevice,
                            ctx->stream));
    ctx->have_pixels = true;
    ctx->have_counts = false;
    TRY(build_raytab(ctx));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MT_OK;
}

mt_status mt_set_counts(mt_ctx *ctx, const int32_t *counts)
{
    TRY(need(ctx, false));
    if (!counts) return fail(ctx, MT_EINVAL, "null counts");
    const size_t n = (size_t)ctx->S * ctx->P;
    if (!is_device_ptr(counts)) {
        for (size_t i = 0; i < n; ++i)
            if (counts[i] < 0) return fail(ctx, MT_EINVAL, "count %zu is negative", i);
    }
    TRY(dalloc(ctx, &ctx->d_cnt, n));
    CK(ctx, cudaMemcpyAsync(ctx->d_cnt, counts, n * 4, cudaMemcpyDefault, ctx->stream));
    return counts_ready(ctx);
}

mt_status mt_generate_data(mt_ctx *ctx, const double *h_true, uint64_t seed, int count_mode,
                           int32_t *counts_out, double *lambda_out)
{
    TRY(need(ctx, false));
    if (!h_true) return fail(ctx, MT_EINVAL, "null h_true");
    if (count_mode != MT_COUNTS_POISSON && count_mode != MT_COUNTS_ROUND)
        return fail(ctx, MT_EINVAL, "count_mode %d", count_mode);
    const size_t n = (size_t)ctx->S * ctx->P;
    const size_t nh = n_per_chain(ctx);
    TRY(dalloc(ctx, &ctx->d_cnt, n));
    refresh_prob(ctx);
    const size_t scratch = (nh + 1) * 8 + nodes_bytes_f64(ctx->L, ctx->pb.N) + 64;
    TRY(grow(ctx, &ctx->d_in, &ctx->in_cap, scratch));
    CK(ctx, cudaMemcpyAsync(ctx->d_in, h_true, nh * 8, cudaMemcpyDefault, ctx->stream));
    OutBuf lam;
    TRY(dev_out(ctx, lambda_out, n * 8, &ctx->d_out, &ctx->out_cap, &lam));
    double *d_lam = (double *)lam.dev;
    if (!d_lam) {
        TRY(grow(ctx, &ctx->d_out, &ctx->out_cap, n * 8));
        d_lam = (double *)ctx->d_out;
    }
    CK(ctx, launch_gen_counts(ctx->pb, (const double *)ctx->d_in, seed, count_mode, ctx->d_cnt,
                              d_lam, ctx->d_flag, ctx->stream));
    TRY(finish_out(ctx, &lam));
    if (counts_out)
        CK(ctx, cudaMemcpyAsync(counts_out, ctx->d_cnt, n * 4, cudaMemcpyDefault, ctx->stream));
    return counts_ready(ctx);
}

mt_status mt_logpost(mt_ctx *ctx, int n_chains, const void *heights, double *loglik_out,
                     double *logprior_out)
{
    TRY(need(ctx, true));
    if (n_chains < 1 || n_chains > 65535 || !heights)
        return fail(ctx, MT_EINVAL, "need 1 <= n_chains <= 65535 and heights");
    const size_t np = n_per_chain(ctx);
    const void *dh;
    TRY(dev_in(ctx, heights, (size_t)n_chains * np * elem_size(ctx), &dh));
    OutBuf ll, lp;
    TRY(dev_out(ctx, loglik_out, (size_t)n_chains * 8, &ctx->d_out, &ctx->out_cap, &ll));
    TRY(dev_out(ctx, logprior_out, (size_t)n_chains * 8, &ctx->d_out2, &ctx->out2_cap, &lp));
    HRef h{dh, (long long)np, nullptr, 0, 0};
    TRY(eval_logpost(ctx, h, n_chains, (double *)ll.dev, (double *)lp.dev));
    TRY(finish_out(ctx, &ll));
    TRY(finish_out(ctx, &lp));
    if (ll.host || lp.host || dh == ctx->d_in) CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MT_OK;
}

mt_status mt_ray_terms(mt_ctx *ctx, int n_chains, const void *heights, double *opacity_out,
                       double *term_out)
{
    TRY(need(ctx, true));
    if (ctx->linear) return fail(ctx, MT_EINVAL, "mt_ray_terms reports the marched forward model");
    if (n_chains < 1 || n_chains > 65535 || !heights)
        return fail(ctx, MT_EINVAL, "need 1 <= n_chains <= 65535 and heights");
    const size_t np = n_per_chain(ctx);
    const size_t nr = (size_t)n_chains * ctx->pb.n_rays;
    const void *dh;
    TRY(dev_in(ctx, heights, (size_t)n_chains * np * elem_size(ctx), &dh));
    OutBuf o, t;
    TRY(dev_out(ctx, opacity_out, nr * 8, &ctx->d_out, &ctx->out_cap, &o));
    TRY(dev_out(ctx, term_out, nr * 8, &ctx->d_out2, &ctx->out2_cap, &t));
    TRY(ensure_partials(ctx, n_chains));
    HRef h{dh, (long long)np, nullptr, 0, 0};
    TRY(prior_and_heights(ctx, h, n_chains, nullptr, &h));
    CK(ctx, launch_march(ctx->pb, ctx->mode, h, n_chains, ctx->d_part, (double *)o.dev,
                         (double *)t.dev, ctx->stream));
    TRY(finish_out(ctx, &o));
    TRY(finish_out(ctx, &t));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MT_OK;
}

mt_status mt_grad(mt_ctx *ctx, int n_chains, const void *heights, double *grad_out,
                  double *logpost_out)
{
    TRY(need(ctx, true));
    TRY(grad_ok(ctx));
    if (n_chains < 1 || n_chains > 65535 || !heights || !grad_out)
        return fail(ctx, MT_EINVAL, "need 1 <= n_chains <= 65535, heights and grad_out");
    const size_t np = n_per_chain(ctx);
    const void *dh;
    TRY(dev_in(ctx, heights, (size_t)n_chains * np * elem_size(ctx), &dh));
    OutBuf g, lp;
    TRY(dev_out(ctx, grad_out, (size_t)n_chains * np * 8, &ctx->d_out, &ctx->out_cap, &g));
    TRY(dev_out(ctx, logpost_out, (size_t)n_chains * 8, &ctx->d_out2, &ctx->out2_cap, &lp));
    TRY(grow(ctx, &ctx->d_tmp, &ctx->tmp_cap, (size_t)n_chains * 16));
    double *t_ll = (double *)ctx->d_tmp, *t_lp = t_ll + n_chains;
    HRef h{dh, (long long)np, nullptr, 0, 0};
    TRY(eval_grad(ctx, h, n_chains, (double *)g.dev, lp.dev ? t_ll : nullptr, lp.dev ? t_lp : nullptr));
    if (lp.dev) CK(ctx, launch_add(n_chains, t_ll, t_lp, (double *)lp.dev, ctx->stream));
    TRY(finish_out(ctx, &g));
    TRY(finish_out(ctx, &lp));
    if (g.host || lp.host || dh == ctx->d_in) CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MT_OK;
}

mt_status mt_init_chains(mt_ctx *ctx, int n_chains, const void *heights0, uint64_t seed)
{
    TRY(need(ctx, true));
    if (n_chains < 1 || n_chains > 65535 || !heights0)
        return fail(ctx, MT_EINVAL, "need 1 <= n_chains <= 65535 and heights0");
    const size_t np = n_per_chain(ctx), es = elem_size(ctx);
    if (n_chains != ctx->C) {
        drop_chains(ctx);
        void *h = nullptr;
        CK(ctx, dev_alloc(ctx, (void **)&h, 2 * (size_t)n_chains * np * es));
        ctx->d_H = h;
        TRY(dalloc(ctx, &ctx->d_cur, n_chains));
        TRY(dalloc(ctx, &ctx->d_psel, n_chains));
        TRY(dalloc(ctx, &ctx->d_ll, n_chains));
        TRY(dalloc(ctx, &ctx->d_lp, n_chains));
        TRY(dalloc(ctx, &ctx->d_llp, n_chains));
        TRY(dalloc(ctx, &ctx->d_lpp, n_chains));
        TRY(dalloc(ctx, &ctx->d_logu, n_chains));
        TRY(dalloc(ctx, &ctx->d_acc, n_chains));
        TRY(dalloc(ctx, &ctx->d_accl, n_chains));
        ctx->C = n_chains;
    }
    drop_graph(ctx);
    ctx->g_valid = false;
    ctx->adapt_pending = ctx->adapt_n > 0;  // new chains adapt their step sizes from the start
    ctx->seed = seed;
    CK(ctx, cudaMemcpyAsync(ctx->d_H, heights0, (size_t)n_chains * np * es, cudaMemcpyDefault,
                            ctx->stream));
    CK(ctx, cudaMemsetAsync(ctx->d_cur, 0, n_chains, ctx->stream));
    CK(ctx, cudaMemsetAsync(ctx->d_psel, 1, n_chains, ctx->stream));
    CK(ctx, cudaMemsetAsync(ctx->d_acc, 0, 8 * (size_t)n_chains, ctx->stream));
    CK(ctx, cudaMemsetAsync(ctx->d_accl, 0, 4 * (size_t)n_chains, ctx->stream));
    CK(ctx, cudaMemsetAsync(ctx->d_step, 0, 8, ctx->stream));
    HRef h{ctx->d_H, (long long)np, nullptr, 0, 0};
    TRY(eval_logpost(ctx, h, n_chains, ctx->d_ll, ctx->d_lp));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MT_OK;
}

// Gradients of the current states, for MALA (computed once, then carried).
static mt_status ensure_chain_grads(mt_ctx *ctx)
{
    if (ctx->g_valid) return MT_OK;
    const size_t np = n_per_chain(ctx);
    if (!ctx->d_G) TRY(dalloc(ctx, &ctx->d_G, 2 * (size_t)ctx->C * np));
    if (!ctx->d_extra) TRY(dalloc(ctx, &ctx->d_extra, (size_t)ctx->C));
    // gradients of the current heights into G[cur]; the current log-likelihoods
    // are refreshed by the gradient's forward pass, which the proposals' use too
    HRef hc{ctx->d_H, (long long)np, ctx->d_cur, (long long)(ctx->C * np), 0};
    TRY(grow(ctx, &ctx->d_out, &ctx->out_cap, (size_t)ctx->C * np * 8));
    TRY(eval_grad(ctx, hc, ctx->C, (double *)ctx->d_out, ctx->d_ll, nullptr));
    CK(ctx, launch_scatter_sel(ctx->C, (long long)np, (const double *)ctx->d_out, ctx->d_cur,
                               ctx->d_G, ctx->stream));
    ctx->g_valid = true;
    return MT_OK;
}

// The proposals' (slot 1 - cur) log-prior into d_lpp, forward march with
// d ll / d O_p (log-likelihood partials in d_part), adjoint, and their
// log-posterior gradient into G[1 - cur]: heights with the CAR prior, or
// latents through the copula transform and its reverse pass.
static mt_status enqueue_proposal_eval(mt_ctx *ctx, HRef hp)
{
    if (!ctx->copula) {
        CK(ctx, launch_prior(ctx->pb, ctx->mode, hp, ctx->d_mu, ctx->C, ctx->d_lpp, ctx->stream));
        TRY(enqueue_forward_adjoint(ctx, hp, ctx->C));
        CK(ctx, launch_grad_finish_sel(ctx->pb, ctx->mode, hp, ctx->d_mu, ctx->C,
                                       (const unsigned long long *)ctx->d_gacc, ctx->d_G, ctx->d_cur,
                                       ctx->stream));
        return MT_OK;
    }
    HRef hh;
    TRY(prior_and_heights(ctx, hp, ctx->C, ctx->d_lpp, &hh));
    TRY(enqueue_forward_adjoint(ctx, hh, ctx->C));
    CK(ctx, launch_copula_vjp(ctx->pb, hp, hh, ctx->d_terr, (const unsigned long long *)ctx->d_gacc, ctx->d_G,
                              ctx->d_cur, ctx->C, ctx->stream));
    return MT_OK;
}

static mt_status enqueue_mala(mt_ctx *ctx, double eps, int off)
{
    const size_t np = n_per_chain(ctx);
    const long long bs = (long long)ctx->C * np;
    EvPair es;
    if (ctx->timing) ev_begin(ctx, 1, &es);
    const double *ec = ctx->adapt_n > 0 ? ctx->d_eps : nullptr;
    CK(ctx, launch_propose_mala(ctx->pb, ctx->mode, ctx->d_H, bs, ctx->d_G, ctx->d_cur, ctx->C, eps, ec,
                                ctx->seed, ctx->d_step, off, ctx->stream));
    HRef hp{ctx->d_H, (long long)np, ctx->d_cur, bs, 1};
    EvPair ep;
    if (ctx->timing) ev_begin(ctx, 0, &ep);
    TRY(enqueue_proposal_eval(ctx, hp));  // prior, log-likelihood and gradient of the proposals
    if (ctx->timing) ev_end(ctx, 0, &ep);
    CK(ctx, launch_mala_hastings(ctx->pb, ctx->mode, ctx->d_H, bs, ctx->d_G, ctx->d_cur, ctx->C, eps, ec,
                                 ctx->d_extra, ctx->stream));
    CK(ctx, launch_accept_fused(ctx->pb, part_mode(ctx), ctx->C, ctx->d_part, ctx->d_lpp, ctx->d_extra,
                                ctx->d_ll, ctx->d_lp, ctx->d_llp, ctx->d_cur, ctx->d_psel,
                                ctx->d_acc, ctx->d_accl, ctx->d_logu, ctx->seed, ctx->d_step, off,
                                ctx->stream, ec ? ctx->d_alpha : nullptr));
    if (ec)
        CK(ctx, launch_adapt(ctx->C, ctx->adapt_target, ctx->adapt_n, 0, ctx->d_alpha, ctx->d_da, ctx->d_eps,
                             ctx->stream));
    if (ctx->timing) ev_end(ctx, 1, &es);
    return MT_OK;
}

static mt_status ensure_hmc(mt_ctx *ctx)
{
    const size_t n = (size_t)ctx->C * n_per_chain(ctx);
    if (!ctx->d_P) TRY(dalloc(ctx, &ctx->d_P, n));
    if (!ctx->d_Q64) TRY(dalloc(ctx, &ctx->d_Q64, n));
    if (!ctx->d_k0) TRY(dalloc(ctx, &ctx->d_k0, (size_t)ctx->C));
    return MT_OK;
}

// Warm-up adaptation buffers; on the first gradient-sampler run after
// mt_set_adapt (or after new chains) every chain starts at eps0 (and, with
// the metric adapted, at the unit metric with empty accumulators).
static mt_status ensure_adapt(mt_ctx *ctx, double eps0)
{
    const size_t C = (size_t)ctx->C, nm = C * n_per_chain(ctx);
    if (!ctx->d_eps || !ctx->d_da || !ctx->d_alpha) {
        drop_graph(ctx);
        TRY(dalloc(ctx, &ctx->d_eps, C));
        TRY(dalloc(ctx, &ctx->d_da, (size_t)kDAStride * C));
        TRY(dalloc(ctx, &ctx->d_alpha, C));
        CK(ctx, cudaMemsetAsync(ctx->d_alpha, 0, C * 8, ctx->stream));
        ctx->adapt_pending = true;
    }
    if (ctx->metric_on && (!ctx->d_minv || !ctx->d_wmean || !ctx->d_wm2)) {
        drop_graph(ctx);
        TRY(dalloc(ctx, &ctx->d_minv, nm));
        TRY(dalloc(ctx, &ctx->d_wmean, nm));
        TRY(dalloc(ctx, &ctx->d_wm2, nm));
        ctx->adapt_pending = true;
    }
    if (ctx->adapt_pending) {
        CK(ctx, launch_adapt_init(ctx->C, eps0, ctx->d_da, ctx->d_eps, ctx->stream));
        if (ctx->metric_on) CK(ctx, launch_metric_init(nm, ctx->d_wmean, ctx->d_wm2, ctx->d_minv, ctx->stream));
        ctx->adapt_pending = false;
    }
    return MT_OK;
}

// One HMC step: momentum and the first drift, then per leapfrog step the
// proposal's evaluation (prior, forward march, adjoint, gradient) and a
// kick + drift, a final half kick with the kinetic-energy difference, and
// the accept (the last evaluation, at the trajectory's end, gave the
// proposal's log-prior and log-likelihood partials).
static mt_status enqueue_hmc(mt_ctx *ctx, double eps, int off)
{
    const size_t np = n_per_chain(ctx);
    const long long bs = (long long)ctx->C * np;
    EvPair es;
    if (ctx->timing) ev_begin(ctx, 1, &es);
    const double *ec = ctx->adapt_n > 0 ? ctx->d_eps : nullptr;
    const bool metric = ec && ctx->metric_on;
    const double *mi = metric ? ctx->d_minv : nullptr;
    CK(ctx, launch_hmc_start(ctx->pb, ctx->mode, ctx->d_H, bs, ctx->d_G, ctx->d_cur, ctx->C, eps, ec, mi,
                             ctx->d_P, ctx->d_Q64, ctx->d_k0, ctx->seed, ctx->d_step, off, ctx->stream));
    HRef hp{ctx->d_H, (long long)np, ctx->d_cur, bs, 1};
    for (int i = 0; i < ctx->hmc_leap; ++i) {
        // the last evaluation, at the end of the trajectory, leaves the
        // proposal's log-prior in d_lpp and its log-likelihood partials
        TRY(enqueue_proposal_eval(ctx, hp));
        if (i + 1 < ctx->hmc_leap)
            CK(ctx, launch_hmc_kick_drift(ctx->pb, ctx->mode, ctx->d_H, bs, ctx->d_G, ctx->d_cur, ctx->C,
                                          eps, ec, mi, ctx->d_P, ctx->d_Q64, ctx->stream));
    }
    CK(ctx, launch_hmc_finish(ctx->pb, bs, ctx->d_G, ctx->d_cur, ctx->C, eps, ec, mi, ctx->d_P, ctx->d_k0,
                              ctx->d_extra, ctx->stream));
    CK(ctx, launch_accept_fused(ctx->pb, part_mode(ctx), ctx->C, ctx->d_part, ctx->d_lpp, ctx->d_extra,
                                ctx->d_ll, ctx->d_lp, ctx->d_llp, ctx->d_cur, ctx->d_psel,
                                ctx->d_acc, ctx->d_accl, ctx->d_logu, ctx->seed, ctx->d_step, off,
                                ctx->stream, ec ? ctx->d_alpha : nullptr));
    if (metric)  // the post-step states into the slow window's accumulators
        CK(ctx, launch_metric(ctx->pb, ctx->mode, ctx->d_H, bs, ctx->d_cur, ctx->C, ctx->adapt_n,
                              ctx->metric_shrink, ctx->d_da, ctx->d_wmean, ctx->d_wm2, ctx->d_minv,
                              ctx->stream));
    if (ec)
        CK(ctx, launch_adapt(ctx->C, ctx->adapt_target, ctx->adapt_n, metric ? 1 : 0, ctx->d_alpha, ctx->d_da,
                             ctx->d_eps, ctx->stream));
    if (ctx->timing) ev_end(ctx, 1, &es);
    return MT_OK;
}

static mt_status ensure_nuts(mt_ctx *ctx)
{
    NutsBufs &b = ctx->nuts;
    const size_t n = (size_t)ctx->C * n_per_chain(ctx);
    if (b.qL && b.sc) return MT_OK;
    drop_graph(ctx);
    for (double **p : {&b.qL, &b.pL, &b.gL, &b.qR, &b.pR, &b.gR, &b.ph, &b.gsel, &b.gsub}) TRY(dalloc(ctx, p, n));
    TRY(dalloc(ctx, &b.sc, (size_t)kNS * ctx->C));
    const size_t es = elem_size(ctx);
    for (void **p : {&b.hsel, &b.hsub}) {
        dfree(ctx, *p);
        CK(ctx, dev_alloc(ctx, (void **)p, n * es + 16));
    }
    return MT_OK;
}

// One capped-NUTS iteration: momentum and the trajectory's start, then per
// depth j its 2^j leapfrog steps (half kick + drift, the new state's prior,
// forward march + adjoint, gradient, log-likelihood, second half kick with
// the state's weight and the subtree's sample), the merge into the
// trajectory's sample, and the move of the chain to it.
static mt_status enqueue_nuts(mt_ctx *ctx, double eps, int off)
{
    const size_t np = n_per_chain(ctx);
    const long long bs = (long long)ctx->C * np;
    EvPair es;
    if (ctx->timing) ev_begin(ctx, 1, &es);
    const double *ec = ctx->adapt_n > 0 ? ctx->d_eps : nullptr;
    const bool metric = ec && ctx->metric_on;
    const double *mi = metric ? ctx->d_minv : nullptr;
    const NutsBufs &nb = ctx->nuts;
    CK(ctx, launch_nuts_start(ctx->pb, ctx->mode, ctx->d_H, bs, ctx->d_G, ctx->d_cur, ctx->C, mi, ctx->d_ll,
                              ctx->d_lp, nb, ctx->seed, ctx->d_step, off, ctx->stream));
    HRef hp{ctx->d_H, (long long)np, ctx->d_cur, bs, 1};
    int leaf = 0;
    for (int j = 0; j < ctx->nuts_depth; ++j) {
        for (int k = 0; k < (1 << j); ++k, ++leaf) {
            CK(ctx, launch_nuts_drift(ctx->pb, ctx->mode, ctx->d_H, bs, ctx->d_cur, ctx->C, eps, ec, mi, nb,
                                      ctx->seed, ctx->d_step, off, j, ctx->stream));
            TRY(enqueue_proposal_eval(ctx, hp));
            CK(ctx, launch_reduce_ll(ctx->pb, part_mode(ctx), ctx->C, ctx->d_part, ctx->d_llp, ctx->stream));
            CK(ctx, launch_nuts_leaf(ctx->pb, ctx->mode, ctx->d_H, bs, ctx->d_G, ctx->d_cur, ctx->C, eps, ec, mi,
                                     ctx->d_llp, ctx->d_lpp, nb, ctx->seed, ctx->d_step, off, j, leaf,
                                     ctx->stream));
        }
        CK(ctx, launch_nuts_merge(ctx->pb, ctx->mode, ctx->C, nb, ctx->seed, ctx->d_step, off, j, ctx->stream));
    }
    CK(ctx, launch_nuts_finish(ctx->pb, ctx->mode, ctx->d_H, bs, ctx->d_G, ctx->d_cur, ctx->d_psel, ctx->C,
                               ctx->d_ll, ctx->d_lp, ctx->d_llp, ctx->d_lpp, ctx->d_acc, ctx->d_accl, ctx->d_logu,
                               ec ? ctx->d_alpha : nullptr, nb, leaf, ctx->stream));
    if (metric)
        CK(ctx, launch_metric(ctx->pb, ctx->mode, ctx->d_H, bs, ctx->d_cur, ctx->C, ctx->adapt_n,
                              ctx->metric_shrink, ctx->d_da, ctx->d_wmean, ctx->d_wm2, ctx->d_minv,
                              ctx->stream));
    if (ec)
        CK(ctx, launch_adapt(ctx->C, ctx->adapt_target, ctx->adapt_n, metric ? 1 : 0, ctx->d_alpha, ctx->d_da,
                             ctx->d_eps, ctx->stream));
    if (ctx->timing) ev_end(ctx, 1, &es);
    return MT_OK;
}

static mt_status enqueue_step(mt_ctx *ctx, int kernel, double step, int off)
{
    const size_t np = n_per_chain(ctx);
    const long long bs = (long long)ctx->C * np;
    if (kernel == MT_KERNEL_MALA) return enqueue_mala(ctx, step, off);
    if (kernel == MT_KERNEL_HMC) return enqueue_hmc(ctx, step, off);
    if (kernel == MT_KERNEL_NUTS) return enqueue_nuts(ctx, step, off);
    if (kernel != MT_KERNEL_RW) return fail(ctx, MT_EINVAL, "kernel %d not available", kernel);
    EvPair es;
    if (ctx->timing) ev_begin(ctx, 1, &es);
    CK(ctx, launch_propose_rw(ctx->pb, ctx->mode, ctx->d_H, bs, ctx->d_cur, ctx->C, step, ctx->seed,
                              ctx->d_step, off, ctx->stream));
    HRef hp{ctx->d_H, (long long)np, ctx->d_cur, bs, 1};
    TRY(prior_and_heights(ctx, hp, ctx->C, ctx->d_lpp, &hp));
    EvPair ep;
    if (ctx->timing) {
        ev_begin(ctx, 0, &ep);
        count_work(ctx, ctx->C);
    }
    TRY(ray_kernel(ctx, hp, ctx->C));
    if (ctx->timing) ev_end(ctx, 0, &ep);
    CK(ctx, launch_accept_fused(ctx->pb, part_mode(ctx), ctx->C, ctx->d_part, ctx->d_lpp, nullptr,
                                ctx->d_ll, ctx->d_lp, ctx->d_llp, ctx->d_cur, ctx->d_psel,
                                ctx->d_acc, ctx->d_accl, ctx->d_logu, ctx->seed, ctx->d_step, off,
                                ctx->stream));
    if (ctx->timing) ev_end(ctx, 1, &es);
    return MT_OK;
}

mt_status mt_run(mt_ctx *ctx, int kernel, double step, int n_super, int n_within)
{
    TRY(need(ctx, true));
    if (ctx->C < 1) return fail(ctx, MT_ESTATE, "mt_init_chains first");
    if (kernel != MT_KERNEL_RW && kernel != MT_KERNEL_MALA && kernel != MT_KERNEL_HMC &&
        kernel != MT_KERNEL_NUTS)
        return fail(ctx, MT_EINVAL, "kernel %d", kernel);
    if (!(step >= 0.0) || n_super < 0 || n_within < 1 || n_within > 4096)
        return fail(ctx, MT_EINVAL, "need step >= 0, n_super >= 0, 1 <= n_within <= 4096");
    if (ctx->copula) TRY(ensure_derived(ctx, ctx->C));
    TRY(ensure_lin(ctx, ctx->C));
    if (kernel == MT_KERNEL_MALA || kernel == MT_KERNEL_HMC || kernel == MT_KERNEL_NUTS) {
        TRY(grad_ok(ctx));
        if (!(step > 0.0)) return fail(ctx, MT_EINVAL, "MALA / HMC / NUTS need a step size eps > 0");
        if (ctx->metric_on && ctx->adapt_n > 0 && kernel == MT_KERNEL_MALA)
            return fail(ctx, MT_EINVAL, "the adapted metric is for HMC: mt_set_metric_adapt(ctx, 0, ...) for MALA");
        if (ctx->metric_on && ctx->adapt_n > 0 && ctx->adapt_n < 20)
            return fail(ctx, MT_EINVAL, "metric adaptation needs n_adapt >= 20 warm-up steps");
        TRY(ensure_chain_grads(ctx));
        TRY(ensure_grad_bufs(ctx, ctx->C));
        if (kernel == MT_KERNEL_HMC) TRY(ensure_hmc(ctx));
        if (kernel == MT_KERNEL_NUTS) TRY(ensure_nuts(ctx));
        if (ctx->adapt_n > 0) TRY(ensure_adapt(ctx, step));
    }
    TRY(ensure_partials(ctx, ctx->C));
    // random-walk steps move the states without their gradients
    if (kernel == MT_KERNEL_RW && n_super > 0) ctx->g_valid = false;
    if (ctx->timing) {
        for (int s = 0; s < n_super; ++s) {
            for (int i = 0; i < n_within; ++i) TRY(enqueue_step(ctx, kernel, step, i));
            CK(ctx, launch_advance(ctx->d_step, n_within, ctx->stream));
        }
        return MT_OK;
    }
    if (!(ctx->gexec && ctx->g_kernel == kernel && ctx->g_step == step && ctx->g_nw == n_within &&
          ctx->g_C == ctx->C)) {
        drop_graph(ctx);
        cudaGraph_t g = nullptr;
        CK(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        mt_status st = MT_OK;
        for (int i = 0; i < n_within && st == MT_OK; ++i) st = enqueue_step(ctx, kernel, step, i);
        if (st == MT_OK) {
            cudaError_t e = launch_advance(ctx->d_step, n_within, ctx->stream);
            if (e != cudaSuccess) st = fail(ctx, MT_ECUDA, "advance: %s", cudaGetErrorString(e));
        }
        cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
        if (st != MT_OK) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return st;
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, MT_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        }
        e = cudaGraphInstantiate(&ctx->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ctx->gexec = nullptr;
            cudaGetLastError();
            return fail(ctx, MT_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        }
        ctx->g_kernel = kernel;
        ctx->g_step = step;
        ctx->g_nw = n_within;
        ctx->g_C = ctx->C;
    }
    // one NVTX range per super-step on the host timeline (a profiler that
    // traces NVTX shows the graph launch and its kernels under it)
    static const char *names[] = {"mt_run RW super-step", "mt_run MALA super-step", "mt_run HMC super-step",
                                  "mt_run NUTS super-step"};
    for (int s = 0; s < n_super; ++s) {
        nvtxRangePushA(names[kernel]);
        const cudaError_t e = cudaGraphLaunch(ctx->gexec, ctx->stream);
        nvtxRangePop();
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, MT_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
        }
    }
    return MT_OK;
}

mt_status mt_get_state(mt_ctx *ctx, void *heights_out, double *loglik_out, double *logprior_out,
                       int64_t *accepts_out, int64_t *step_out)
{
    TRY(need(ctx, false));
    if (ctx->C < 1) return fail(ctx, MT_ESTATE, "mt_init_chains first");
    const size_t np = n_per_chain(ctx), C = ctx->C;
    if (heights_out) {
        OutBuf o;
        TRY(dev_out(ctx, heights_out, C * np * elem_size(ctx), &ctx->d_out, &ctx->out_cap, &o));
        HRef h{ctx->d_H, (long long)np, ctx->d_cur, (long long)(C * np), 0};
        CK(ctx, launch_gather(ctx->mode, h, (int)C, (long long)np, o.dev, ctx->stream));
        TRY(finish_out(ctx, &o));
    }
    if (loglik_out)
        CK(ctx, cudaMemcpyAsync(loglik_out, ctx->d_ll, C * 8, cudaMemcpyDefault, ctx->stream));
    if (logprior_out)
        CK(ctx, cudaMemcpyAsync(logprior_out, ctx->d_lp, C * 8, cudaMemcpyDefault, ctx->stream));
    if (accepts_out)
        CK(ctx, cudaMemcpyAsync(accepts_out, ctx->d_acc, C * 8, cudaMemcpyDefault, ctx->stream));
    int64_t stp = 0;
    CK(ctx, cudaMemcpyAsync(&stp, ctx->d_step, 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (step_out) *step_out = stp;
    return MT_OK;
}

mt_status mt_get_last_step(mt_ctx *ctx, void *proposal_out, double *loglik_out,
                           double *logprior_out, int32_t *accepted_out, double *logu_out)
{
    TRY(need(ctx, false));
    if (ctx->C < 1) return fail(ctx, MT_ESTATE, "mt_init_chains first");
    const size_t np = n_per_chain(ctx), C = ctx->C;
    if (proposal_out) {
        OutBuf o;
        TRY(dev_out(ctx, proposal_out, C * np * elem_size(ctx), &ctx->d_out, &ctx->out_cap, &o));
        HRef h{ctx->d_H, (long long)np, ctx->d_psel, (long long)(C * np), 0};
        CK(ctx, launch_gather(ctx->mode, h, (int)C, (long long)np, o.dev, ctx->stream));
        TRY(finish_out(ctx, &o));
    }
    if (loglik_out)
        CK(ctx, cudaMemcpyAsync(loglik_out, ctx->d_llp, C * 8, cudaMemcpyDefault, ctx->stream));
    if (logprior_out)
        CK(ctx, cudaMemcpyAsync(logprior_out, ctx->d_lpp, C * 8, cudaMemcpyDefault, ctx->stream));
    if (accepted_out)
        CK(ctx, cudaMemcpyAsync(accepted_out, ctx->d_accl, C * 4, cudaMemcpyDefault, ctx->stream));
    if (logu_out)
        CK(ctx, cudaMemcpyAsync(logu_out, ctx->d_logu, C * 8, cudaMemcpyDefault, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MT_OK;
}

mt_status mt_set_state(mt_ctx *ctx, const void *heights, int64_t step)
{
    TRY(need(ctx, true));
    if (ctx->C < 1) return fail(ctx, MT_ESTATE, "mt_init_chains first");
    if (!heights || step < 0) return fail(ctx, MT_EINVAL, "need heights and step >= 0");
    const size_t np = n_per_chain(ctx), es = elem_size(ctx);
    CK(ctx, cudaMemcpyAsync(ctx->d_H, heights, (size_t)ctx->C * np * es, cudaMemcpyDefault,
                            ctx->stream));
    CK(ctx, cudaMemsetAsync(ctx->d_cur, 0, ctx->C, ctx->stream));
    CK(ctx, cudaMemcpyAsync(ctx->d_step, &step, 8, cudaMemcpyHostToDevice, ctx->stream));
    ctx->g_valid = false;
    HRef h{ctx->d_H, (long long)np, nullptr, 0, 0};
    TRY(eval_logpost(ctx, h, ctx->C, ctx->d_ll, ctx->d_lp));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MT_OK;
}

mt_status mt_sync(mt_ctx *ctx, double timeout_s)
{
    if (!ctx) return fail(nullptr, MT_EINVAL, "null context");
    CK(ctx, cudaSetDevice(ctx->device));
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(ctx->stream);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) {
            cudaGetLastError();
            return fail(ctx, MT_ECUDA, "stream: %s", cudaGetErrorString(e));
        }
        const double el =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (timeout_s > 0.0 && el > timeout_s)
            return fail(ctx, MT_ETIMEDOUT, "work still in flight after %.3f s", el);
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    int flag = 0;
    CK(ctx, cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (flag) {
        CK(ctx, cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
        return fail(ctx, MT_EDEVFLAG,
                    "a kernel latched device status %d (1: a Poisson draw ran out of attempts; 2: a "
                    "ray's samples left the grid; 4: a cell index out of range, MT_BOUNDS_CHECK builds)",
                    flag);
    }
    return MT_OK;
}

mt_status mt_set_timing(mt_ctx *ctx, int on)
{
    if (!ctx) return fail(nullptr, MT_EINVAL, "null context");
    CK(ctx, cudaSetDevice(ctx->device));
    ctx->timing = on != 0;
    drop_graph(ctx);
    if (ctx->timing && !ctx->d_work) {
        TRY(dalloc(ctx, &ctx->d_work, 1));
        CK(ctx, cudaMemsetAsync(ctx->d_work, 0, 8, ctx->stream));
    }
    ctx->pb.work = ctx->timing ? ctx->d_work : nullptr;
    return MT_OK;
}

mt_status mt_get_work(mt_ctx *ctx, double *evaluated, double *total, int reset)
{
    if (!ctx) return fail(nullptr, MT_EINVAL, "null context");
    CK(ctx, cudaSetDevice(ctx->device));
    unsigned long long e = 0;
    if (ctx->d_work) {
        CK(ctx, cudaMemcpyAsync(&e, ctx->d_work, 8, cudaMemcpyDeviceToHost, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
    }
    if (evaluated) *evaluated = (double)e;
    if (total) *total = ctx->work_total;
    if (reset) {
        if (ctx->d_work) CK(ctx, cudaMemsetAsync(ctx->d_work, 0, 8, ctx->stream));
        ctx->work_total = 0.0;
    }
    return MT_OK;
}

mt_status mt_get_timing(mt_ctx *ctx, int id, double *total_ms, int64_t *launches, int reset)
{
    if (!ctx) return fail(nullptr, MT_EINVAL, "null context");
    if (id < 0 || id > 1) return fail(ctx, MT_EINVAL, "timing id %d", id);
    CK(ctx, cudaSetDevice(ctx->device));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < 2; ++k) {
        for (auto &p : ctx->ev_open[k]) {
            float ms = 0.f;
            CK(ctx, cudaEventElapsedTime(&ms, p.a, p.b));
            ctx->t_ms[k] += ms;
            ctx->t_n[k] += 1;
            ctx->ev_pool.push_back(p.a);
            ctx->ev_pool.push_back(p.b);
        }
        ctx->ev_open[k].clear();
    }
    if (total_ms) *total_ms = ctx->t_ms[id];
    if (launches) *launches = ctx->t_n[id];
    if (reset) {
        ctx->t_ms[id] = 0.0;
        ctx->t_n[id] = 0;
    }
    return MT_OK;
}

mt_status mt_get_sizes(const mt_ctx *ctx, int *n_layers, int *n_rows, int *n_cols, int *n_sensors,
                       int *n_pixels, int *n_chains)
{
    if (!ctx) return fail(nullptr, MT_EINVAL, "null context");
    if (n_layers) *n_layers = ctx->L;
    if (n_rows) *n_rows = ctx->R;
    if (n_cols) *n_cols = ctx->Q;
    if (n_sensors) *n_sensors = ctx->S;
    if (n_pixels) *n_pixels = ctx->P;
    if (n_chains) *n_chains = ctx->C;
    return MT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- diagnostics
mt_status mt_nested_rhat(mt_ctx *ctx, int n_draws, int n_chains, const void *draws, int n_super,
                         double *rhat_out, double *rhat_max_out)
{
    if (!ctx) return fail(nullptr, MT_EINVAL, "null context");
    if (!ctx->have_grid) return fail(ctx, MT_ESTATE, "mt_set_grid has not been called");
    if (n_draws < 1 || n_super < 2 || n_super > 65535 || n_chains < n_super || n_chains % n_super ||
        !draws)
        return fail(ctx, MT_EINVAL,
                    "mt_nested_rhat: need n_draws >= 1, 2 <= n_super <= 65535 dividing n_chains, "
                    "and draws");
    CK(ctx, cudaSetDevice(ctx->device));
    const size_t P = n_per_chain(ctx);
    const void *dd;
    TRY(dev_in(ctx, draws, (size_t)n_draws * n_chains * P * elem_size(ctx), &dd));
    OutBuf o;
    TRY(dev_out(ctx, rhat_out, P * 8, &ctx->d_out, &ctx->out_cap, &o));
    TRY(grow(ctx, &ctx->d_diag, &ctx->diag_cap, (2 * (size_t)n_super * P + 1) * 8));
    double *sm = (double *)ctx->d_diag, *wk = sm + (size_t)n_super * P;
    unsigned long long *mx = (unsigned long long *)(wk + (size_t)n_super * P);
    CK(ctx, cudaMemsetAsync(mx, 0, 8, ctx->stream));
    CK(ctx, launch_nested_rhat(ctx->mode, dd, n_draws, n_chains, (int)P, n_super, sm, wk,
                               (double *)o.dev, mx, ctx->stream));
    TRY(finish_out(ctx, &o));
    if (rhat_max_out)
        CK(ctx, cudaMemcpyAsync(rhat_max_out, mx, 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MT_OK;
}

mt_status mt_interface_std(mt_ctx *ctx, int n_samples, const void *samples, int n_z, double *std_out)
{
    if (!ctx) return fail(nullptr, MT_EINVAL, "null context");
    if (!ctx->have_grid) return fail(ctx, MT_ESTATE, "mt_set_grid has not been called");
    if (n_samples < 1 || n_z < 1 || n_z > 4096 || !samples || !std_out)
        return fail(ctx, MT_EINVAL,
                    "mt_interface_std: need n_samples >= 1, 1 <= n_z <= 4096, samples and std_out");
    CK(ctx, cudaSetDevice(ctx->device));
    const size_t P = n_per_chain(ctx), N = (size_t)ctx->R * ctx->Q;
    const void *ds;
    TRY(dev_in(ctx, samples, (size_t)n_samples * P * elem_size(ctx), &ds));
    OutBuf o;
    TRY(dev_out(ctx, std_out, (size_t)ctx->L * n_z * N * 8, &ctx->d_out, &ctx->out_cap, &o));
    std::vector<double> z(n_z);
    const double dz = ctx->box[2] / n_z;
    for (int k = 0; k < n_z; ++k) z[k] = k * dz;
    TRY(grow(ctx, &ctx->d_diag, &ctx->diag_cap, (size_t)n_z * 8));
    CK(ctx, cudaMemcpyAsync(ctx->d_diag, z.data(), (size_t)n_z * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, launch_interface_std(ctx->mode, ds, n_samples, ctx->L, (int)N, n_z,
                                 (const double *)ctx->d_diag, (double *)o.dev, ctx->stream));
    TRY(finish_out(ctx, &o));
    CK(ctx, cudaStreamSynchronize(ctx->stream));  // z is a local host buffer
    return MT_OK;
}

// ---------------------------------------------------------------- copula prior
mt_status mt_set_prior(mt_ctx *ctx, int kind)
{
    if (!ctx) return fail(nullptr, MT_EINVAL, "null context");
    if (!ctx->have_grid) return fail(ctx, MT_ESTATE, "mt_set_grid has not been called");
    if (kind != MT_PRIOR_CAR && kind != MT_PRIOR_COPULA)
        return fail(ctx, MT_EINVAL, "mt_set_prior: kind %d", kind);
    CK(ctx, cudaSetDevice(ctx->device));
    if (kind == MT_PRIOR_COPULA) {
        if (ctx->L < 2) return fail(ctx, MT_EINVAL, "the copula prior needs >= 2 surfaces (the top is the terrain)");
        const size_t smem = copula_smem_bytes(ctx->pb, ctx->mode);
        if (smem + MT_SMEM_STATIC > MT_MAX_SMEM)
            return fail(ctx, MT_EINVAL, "grid %d x %d too large for the copula transform (%zu bytes of shared memory)",
                        ctx->R, ctx->Q, smem);
        const size_t N = (size_t)ctx->R * ctx->Q, es = elem_size(ctx);
        std::vector<double> t(ctx->mu.begin() + (ctx->L - 1) * N, ctx->mu.begin() + ctx->L * N);
        std::vector<float> tf(N);
        for (size_t i = 0; i < N; ++i) tf[i] = (float)t[i];
        if (ctx->d_terr) dev_free(ctx, ctx->d_terr);
        ctx->d_terr = nullptr;
        CK(ctx, dev_alloc(ctx, (void **)&ctx->d_terr, N * es));
        CK(ctx, cudaMemcpyAsync(ctx->d_terr, es == 8 ? (const void *)t.data() : (const void *)tf.data(),
                                N * es, cudaMemcpyHostToDevice, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
    }
    drop_chains(ctx);
    ctx->copula = kind == MT_PRIOR_COPULA;
    return MT_OK;
}

mt_status mt_copula_heights(mt_ctx *ctx, int n, const void *latent, void *heights_out)
{
    if (!ctx) return fail(nullptr, MT_EINVAL, "null context");
    if (!ctx->copula) return fail(ctx, MT_ESTATE, "mt_set_prior(ctx, MT_PRIOR_COPULA) first");
    if (n < 1 || n > 65535 || !latent || !heights_out)
        return fail(ctx, MT_EINVAL, "need 1 <= n <= 65535, latent and heights_out");
    CK(ctx, cudaSetDevice(ctx->device));
    const size_t bytes = (size_t)n * n_per_chain(ctx) * elem_size(ctx);
    const void *dl;
    TRY(dev_in(ctx, latent, bytes, &dl));
    OutBuf o;
    TRY(dev_out(ctx, heights_out, bytes, &ctx->d_out, &ctx->out_cap, &o));
    HRef h{dl, (long long)n_per_chain(ctx), nullptr, 0, 0};
    CK(ctx, launch_copula(ctx->pb, ctx->mode, h, ctx->d_terr, o.dev, n, ctx->stream));
    TRY(finish_out(ctx, &o));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MT_OK;
}

mt_status mt_set_hmc(mt_ctx *ctx, int n_leapfrog)
{
    if (!ctx) return fail(nullptr, MT_EINVAL, "null context");
    if (n_leapfrog < 1 || n_leapfrog > 1024) return fail(ctx, MT_EINVAL, "n_leapfrog %d not in [1, 1024]", n_leapfrog);
    if (ctx->hmc_leap != n_leapfrog) drop_graph(ctx);
    ctx->hmc_leap = n_leapfrog;
    return MT_OK;
}

mt_status mt_set_adapt(mt_ctx *ctx, double target_accept, int n_adapt)
{
    if (!ctx) return fail(nullptr, MT_EINVAL, "null context");
    if (!(target_accept > 0.0 && target_accept < 1.0) || n_adapt < 0)
        return fail(ctx, MT_EINVAL, "mt_set_adapt: need 0 < target_accept < 1 and n_adapt >= 0");
    CK(ctx, cudaSetDevice(ctx->device));
    drop_graph(ctx);
    ctx->adapt_target = target_accept;
    ctx->adapt_n = n_adapt;
    ctx->adapt_pending = n_adapt > 0;
    if (n_adapt == 0) {
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        dfree(ctx, ctx->d_eps);
        dfree(ctx, ctx->d_da);
        dfree(ctx, ctx->d_alpha);
        dfree(ctx, ctx->d_minv);
        dfree(ctx, ctx->d_wmean);
        dfree(ctx, ctx->d_wm2);
    }
    return MT_OK;
}

mt_status mt_set_nuts(mt_ctx *ctx, int max_depth)
{
    if (!ctx) return fail(nullptr, MT_EINVAL, "null context");
    if (max_depth < 1 || max_depth > 10) return fail(ctx, MT_EINVAL, "max_depth %d not in [1, 10]", max_depth);
    if (ctx->nuts_depth != max_depth) drop_graph(ctx);
    ctx->nuts_depth = max_depth;
    return MT_OK;
}

mt_status mt_set_metric_adapt(mt_ctx *ctx, int on, double shrink)
{
    if (!ctx) return fail(nullptr, MT_EINVAL, "null context");
    if ((on != 0 && on != 1) || !(shrink >= 0.0))
        return fail(ctx, MT_EINVAL, "mt_set_metric_adapt: need on in {0, 1} and shrink >= 0");
    CK(ctx, cudaSetDevice(ctx->device));
    drop_graph(ctx);
    ctx->metric_on = on != 0;
    ctx->metric_shrink = shrink;
    ctx->adapt_pending = ctx->adapt_n > 0;  // the warm-up starts over
    if (!on) {
        CK(ctx, cudaStreamSynchronize(ctx->stream));
        dfree(ctx, ctx->d_minv);
        dfree(ctx, ctx->d_wmean);
        dfree(ctx, ctx->d_wm2);
    }
    return MT_OK;
}

mt_status mt_get_metric(mt_ctx *ctx, double *inv_metric_out)
{
    TRY(need(ctx, false));
    if (ctx->C < 1) return fail(ctx, MT_ESTATE, "mt_init_chains first");
    if (!inv_metric_out) return fail(ctx, MT_EINVAL, "need inv_metric_out");
    if (!ctx->metric_on || ctx->adapt_n == 0 || ctx->adapt_pending || !ctx->d_minv)
        return fail(ctx, MT_ESTATE, "no adapted metric: mt_set_metric_adapt, mt_set_adapt, then an HMC mt_run");
    const size_t n = (size_t)ctx->C * n_per_chain(ctx);
    CK(ctx, cudaMemcpyAsync(inv_metric_out, ctx->d_minv, n * 8, cudaMemcpyDefault, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MT_OK;
}

mt_status mt_get_adapt(mt_ctx *ctx, double *eps_out, double *accept_prob_out)
{
    TRY(need(ctx, false));
    if (ctx->C < 1) return fail(ctx, MT_ESTATE, "mt_init_chains first");
    if (ctx->adapt_n == 0 || ctx->adapt_pending || !ctx->d_eps)
        return fail(ctx, MT_ESTATE, "no adapted step sizes: mt_set_adapt, then a MALA / HMC mt_run");
    const size_t C = ctx->C;
    if (eps_out) CK(ctx, cudaMemcpyAsync(eps_out, ctx->d_eps, C * 8, cudaMemcpyDefault, ctx->stream));
    if (accept_prob_out)
        CK(ctx, cudaMemcpyAsync(accept_prob_out, ctx->d_alpha, C * 8, cudaMemcpyDefault, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    return MT_OK;
}

// ---------------------------------------------------------------- linearised forward model
mt_status mt_set_forward(mt_ctx *ctx, int kind, int n_z, const double *h_ref)
{
    if (!ctx) return fail(nullptr, MT_EINVAL, "null context");
    if (!(ctx->have_grid && ctx->have_sensors && ctx->have_pixels))
        return fail(ctx, MT_ESTATE, "mt_set_forward needs grid, sensors and pixels");
    if (kind != MT_FORWARD_MARCH && kind != MT_FORWARD_LINEAR)
        return fail(ctx, MT_EINVAL, "mt_set_forward: kind %d", kind);
    CK(ctx, cudaSetDevice(ctx->device));
    drop_graph(ctx);
    if (kind == MT_FORWARD_MARCH) {
        ctx->linear = false;
        if (ctx->C > 0 && ctx->have_counts) {  // live chains: re-evaluate under the march
            const size_t np = n_per_chain(ctx);
            HRef h{ctx->d_H, (long long)np, ctx->d_cur, (long long)(ctx->C * np), 0};
            TRY(eval_logpost(ctx, h, ctx->C, ctx->d_ll, ctx->d_lp));
            CK(ctx, cudaStreamSynchronize(ctx->stream));
        }
        ctx->g_valid = false;
        return MT_OK;
    }
    if (n_z < 1 || n_z > 4096) return fail(ctx, MT_EINVAL, "n_z %d not in [1, 4096]", n_z);
    const size_t np = n_per_chain(ctx);
    ctx->lin_href.assign(h_ref ? h_ref : ctx->mu.data(), (h_ref ? h_ref : ctx->mu.data()) + np);
    std::vector<double> sens(3 * (size_t)ctx->S), dirs(3 * (size_t)ctx->P);
    CK(ctx, cudaMemcpyAsync(sens.data(), ctx->d_sensors, sens.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaMemcpyAsync(dirs.data(), ctx->d_dirs, dirs.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    refresh_prob(ctx);
    std::vector<int> row, col;
    std::vector<double> val, R0;
    lin_build_lengths(ctx->pb, sens, dirs, n_z, row, col, val);
    lin_density_host(ctx->pb, ctx->lin_href.data(), n_z, R0);
    const size_t nr = (size_t)ctx->pb.n_rays, nnz = col.size();
    std::vector<double> lam0(nr);
    for (size_t p = 0; p < nr; ++p) {
        double O = 0.0;
        for (int e = row[p]; e < row[p + 1]; ++e) O += val[e] * R0[col[e]];
        lam0[p] = ctx->cfg.I0 * exp(-O / ctx->cfg.atten);
    }
    const size_t es = elem_size(ctx);
    std::vector<float> valf;
    if (es == 4) valf.assign(val.begin(), val.end());
    const size_t nvox = R0.size();
    for (void **p : {(void **)&ctx->d_lrow, (void **)&ctx->d_lcol, &ctx->d_lval, &ctx->d_R0,
                     (void **)&ctx->d_lam0, (void **)&ctx->d_amc, (void **)&ctx->d_lcptr, (void **)&ctx->d_lcrow,
                     &ctx->d_lcval}) {
        if (*p) dev_free(ctx, *p);
        *p = nullptr;
    }
    CK(ctx, dev_alloc(ctx, (void **)&ctx->d_lrow, row.size() * 4));
    CK(ctx, dev_alloc(ctx, (void **)&ctx->d_lcol, nnz * 4 + 16));
    CK(ctx, dev_alloc(ctx, (void **)&ctx->d_lval, nnz * es + 16));
    CK(ctx, dev_alloc(ctx, (void **)&ctx->d_R0, nvox * es));
    CK(ctx, dev_alloc(ctx, (void **)&ctx->d_lam0, nr * 8));
    CK(ctx, dev_alloc(ctx, (void **)&ctx->d_amc, nr * 8));
    CK(ctx, cudaMemcpyAsync(ctx->d_lrow, row.data(), row.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaMemcpyAsync(ctx->d_lcol, col.data(), nnz * 4, cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaMemcpyAsync(ctx->d_lval, es == 4 ? (const void *)valf.data() : (const void *)val.data(),
                            nnz * es, cudaMemcpyHostToDevice, ctx->stream));
    // the same path lengths by voxel, for gradients
    std::vector<int> cptr, crow;
    std::vector<double> cval;
    lin_transpose((int)nr, (int)nvox, row, col, val, cptr, crow, cval);
    std::vector<float> cvalf;
    if (es == 4) cvalf.assign(cval.begin(), cval.end());
    CK(ctx, dev_alloc(ctx, (void **)&ctx->d_lcptr, cptr.size() * 4));
    CK(ctx, dev_alloc(ctx, (void **)&ctx->d_lcrow, nnz * 4 + 16));
    CK(ctx, dev_alloc(ctx, (void **)&ctx->d_lcval, nnz * es + 16));
    CK(ctx, cudaMemcpyAsync(ctx->d_lcptr, cptr.data(), cptr.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaMemcpyAsync(ctx->d_lcrow, crow.data(), nnz * 4, cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaMemcpyAsync(ctx->d_lcval, es == 4 ? (const void *)cvalf.data() : (const void *)cval.data(),
                            nnz * es, cudaMemcpyHostToDevice, ctx->stream));
    // reference densities with the device's own arithmetic (so that the
    // densities of the reference itself differ from them by exactly 0)
    {
        std::vector<float> hf;
        if (es == 4) hf.assign(ctx->lin_href.begin(), ctx->lin_href.end());
        TRY(grow(ctx, &ctx->d_in, &ctx->in_cap, np * es));
        CK(ctx, cudaMemcpyAsync(ctx->d_in, es == 4 ? (const void *)hf.data() : (const void *)ctx->lin_href.data(),
                                np * es, cudaMemcpyHostToDevice, ctx->stream));
        HRef hr{ctx->d_in, (long long)np, nullptr, 0, 0};
        CK(ctx, launch_lin_reference(ctx->pb, ctx->mode, hr, n_z, ctx->d_R0, ctx->stream));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
    }
    CK(ctx, cudaMemcpyAsync(ctx->d_lam0, lam0.data(), nr * 8, cudaMemcpyHostToDevice, ctx->stream));
    ctx->lin_nz = n_z;
    ctx->linear = true;
    if (ctx->have_counts)
        CK(ctx, launch_lin_amc((int)nr, ctx->d_lam0, ctx->d_cnt, ctx->d_amc, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));  // host vectors go out of scope
    if (ctx->C > 0 && ctx->have_counts) {  // live chains: re-evaluate under the new forward model
        HRef h{ctx->d_H, (long long)np, ctx->d_cur, (long long)(ctx->C * np), 0};
        TRY(eval_logpost(ctx, h, ctx->C, ctx->d_ll, ctx->d_lp));
        CK(ctx, cudaStreamSynchronize(ctx->stream));
    }
    ctx->g_valid = false;
    return MT_OK;
}
