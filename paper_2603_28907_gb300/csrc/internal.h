// internal.h -- types shared by the translation units of libmt.so.
//
// The problem descriptor Prob is passed by value to every kernel.  Layouts:
//   heights (HBM)  [chain][layer][row][col], column fastest (C ABI layout);
//   heights (smem) FP32 modes: per-surface planes of (h - ref_l, dx) pairs,
//                  [layer][row][col]; FP64 / BF16: node-major [row][col][layer],
//                  each node padded to a 16/8/4-byte vector;
//   ray table      structure of arrays over ray = sensor * P + pixel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/mt.h"

#define MT_MAX_L 8
#define MT_MAX_SMEM 232448  // opt-in shared memory per block on sm_100/sm_103
// static shared memory a kernel may use on top of its dynamic allocation
#define MT_SMEM_STATIC 4096
// ray slots per CTA of the ray kernels (the FP32 march's CTAs hold one chain
// and this many rays; the chain's CTA partials follow from it)
#ifndef MT_RAYS_PER_CTA
#define MT_RAYS_PER_CTA 6144
#endif

namespace mt {

enum { MODE_F64 = 0, MODE_F32 = 1, MODE_F32C = 2, MODE_BF16 = 3, MODE_F32A = 4 };
// the FP32 modes marched over (h, dx) planes
constexpr bool is_dx_mode(int m) { return m == MODE_F32 || m == MODE_F32C || m == MODE_F32A; }
enum { STREAM_GEOM = 0, STREAM_DATA = 1, STREAM_INIT = 2, STREAM_PROP = 3, STREAM_ACC = 4,
       STREAM_MALA = 5, STREAM_HMC = 6, STREAM_NUTS_P = 7, STREAM_NUTS_U = 8 };

struct Prob {
    int L, R, Q, S, P, G, n_rays, N;  // N = R*Q nodes per surface
    double box[3];
    double gamma, I0, Lambda, inv_Lambda;
    double tau, car_r, delta;
    float kg;                  // log2(e) / gamma (1 for the hard indicator)
    float gm_hi_x, gm_hi_y;    // upper clamp of the shifted cell coordinates (< n - 3/2)
    double rho_top;            // density of the top unit
    double drho[MT_MAX_L];     // rho_l - rho_{l+1}: density step across surface l
    float drho_f[MT_MAX_L];
    // ray table (n_rays entries each)
    const float4 *o4;          // FP32 sample-0 cell coordinates {gx - 1/2, gy - 1/2, 0, 0}
    const float4 *s4;          // FP32 per-sample step {dgx, dgy, kg*dz hi, kg*dz lo}
    const float *kz0;          // [2][L][n_rays] kg * (z_0 - ref_l) as FP32 hi, lo
    // Ray table of the FP32 modes' march (k_march), kept apart so that its
    // sample positions carry no per-ray rounding offset:
    const float4 *xa4;         // {ox, oy, sxh, syh}: sample-0 cell coordinate minus 1/2,
                               // relative to the start cell; per-sample step, high part
    const float4 *xb4;         // {sxl, syl, szh, szl}: low parts of the x, y steps; z step
                               // (log2 units, FP64 kg) on the grid zgrid and its remainder
    const int2 *xc2;           // start cell {c0x, c0y}
    const float *kz1;          // [2][L][n_rays] kg64 * (z_0 - ref_l) on the grid zgrid, remainder
    const float *kzm;          // [2][L][n_rays] z_0 - ref_l in metres on the grid zgrid_m, and
                               // kg64 times the remainder (log2 units)
    const float2 *szm;         // [n_rays] z step in metres on the grid zgrid_m, kg64 times the remainder
    float kgl;                 // kg64 - kg (FP32 remainder of log2(e) / gamma)
    float psi_kc;              // kappa * 2^-28: calibration of the march's logistic
                               // (launch_psi_calib); 0 = none
    double kg64;               // log2(e) / gamma in FP64 (1 for the hard indicator)
    double zgrid;              // grid of the z high parts: 2^(e - 24) with |z| < 2^e
    double zgrid_m;            // the same for z - ref_l in metres
    float ref[MT_MAX_L];       // per-surface reference height of the FP32 paths
    float2 drho_ff[MT_MAX_L];  // float-float of drho
    const double *o_d;         // [3] FP64 sample-0 position {gx, gy, z}
    const double *s_d;         // [3] FP64 per-sample step
    const double *dt;          // sample spacing along the ray (m)
    const double *a;           // ln(I0 / C) (0 where C = 0)
    const float2 *a_ff;        // float-float of a
    const float2 *dt_ff;       // float-float of dt
    const int32_t *cnt;        // observed counts
    double sumK;               // sum over rays of C ln C - C - lgamma(C + 1)
    unsigned long long *work;  // timing mode: [0] surface-samples evaluated by the FP32
                               // march (the rest were exactly saturated), else nullptr
    float *gnodes;             // grids too large for shared memory: per-chain (h, dx)
                               // planes in HBM, [chain][l][node] float2; else nullptr
    int full_windows;          // FP32 march evaluates every sample (verification switch)
    const int *perm;           // march order of the rays (ray table sorted by vertical
                               // step, then start height); nullptr = ray order
    const float2 *mu_ff;       // [L][N] float-float of the prior mean (FP32-mode prior)
    float lz_f;                // largest float <= box[2]
    float2 delta_ff;           // float-float of the minimum thickness
    float2 grho_ff;            // float-float of G * rho_top
    float2 invL_ff;            // float-float of 1 / Lambda
    int *flag;                 // device status word (bit 4: a cell index out of range, in
                               // builds with MT_BOUNDS_CHECK)
    float *dO;                 // FP32 modes: the march also writes d ll / d O_p = (lambda_p -
                               // C_p) / Lambda per ray, [chain][ray]; the adjoint reads it
                               // (nullptr: not written)
};

// Where chain c's heights live: base + sel[c] * sel_stride + c * chain_stride
// (elements), with sel[c] replaced by 1 - sel[c] when sel_flip is set.
struct HRef {
    const void *base;
    long long chain_stride;
    const uint8_t *sel;
    long long sel_stride;
    int sel_flip;
};

// What a context holds for a call that must not allocate (filled by ctx_view,
// which also checks that grid, sensors, pixels and counts are set).
// Host side of the linearised forward model (linear.cu).
void lin_build_lengths(const Prob &pb, const std::vector<double> &sensors,
                       const std::vector<double> &dirs, int nz, std::vector<int> &row,
                       std::vector<int> &col, std::vector<double> &val);
void lin_density_host(const Prob &pb, const double *H, int nz, std::vector<double> &R);

struct CtxView {
    Prob pb;
    int mode;
    int device;
    const double *mu;
    cudaStream_t stream;
};
mt_status ctx_view(mt_ctx *ctx, CtxView *v);
// mt_create with the context's device memory taken from a stream-ordered
// pool (allocated and released on the context's stream; the server's
// request contexts), or from cudaMalloc when pool is nullptr.
mt_status ctx_create_pooled(mt_ctx **out, int device, const mt_config *cfg, void *cuda_stream,
                            cudaMemPool_t pool);
mt_status ctx_fail(mt_ctx *ctx, mt_status st, const char *msg);

// Launchers (stream-ordered, return cudaGetLastError()).
cudaError_t launch_raytab(const Prob &pb, const double *d_sensors, const double *d_dirs,
                          float4 *o4, float4 *s4, float *kz0, double *o_d, double *s_d, double *dt,
                          float2 *dt_ff, int *flag, cudaStream_t st);
// The FP32 march's ray table (Prob::xa4, xb4, xc2, kz1); pb.zgrid, pb.kg64
// and pb.ref must be set.
cudaError_t launch_raytab_march(const Prob &pb, const double *d_sensors, const double *d_dirs,
                                float4 *xa4, float4 *xb4, int2 *xc2, float *kz1, float *kzm, float2 *szm,
                                int *flag, cudaStream_t st);
// kappa of the march's logistic on this device (one double at out).
cudaError_t launch_psi_calib(double *out, cudaStream_t st);
cudaError_t launch_counts_prep(const Prob &pb, double *a, float2 *a_ff, double *sumK,
                               cudaStream_t st);
cudaError_t launch_gen_counts(const Prob &pb, const double *h_nodes, uint64_t seed, int mode,
                              int32_t *counts, double *lambda, int *flag, cudaStream_t st);
int march_rays_per_block(const Prob &pb);
size_t march_smem_bytes(const Prob &pb, int mode);
bool march_fits_smem(const Prob &pb, int mode);  // records + static part within a block's limit
// One surface's plane plus a float-float sum per ray slot (FP32 modes' phased march)
size_t march_phased_smem_bytes(const Prob &pb);
bool march_fits_phased(const Prob &pb, int mode);
cudaError_t launch_march(const Prob &pb, int mode, HRef h, int n_chains, void *partial,
                         double *ray_O, double *ray_term, cudaStream_t st);
cudaError_t launch_reduce_ll(const Prob &pb, int mode, int n_chains, const void *partial,
                             double *ll_out, cudaStream_t st);
cudaError_t launch_prior(const Prob &pb, int mode, HRef h, const double *mu, int n_chains,
                         double *lp_out, cudaStream_t st);
cudaError_t launch_propose_rw(const Prob &pb, int mode, void *hbuf, long long buf_stride,
                              const uint8_t *cur, int n_chains, double sigma, uint64_t seed,
                              const int64_t *step_base, int step_off, cudaStream_t st);
cudaError_t launch_advance(int64_t *step, int n, cudaStream_t st);
size_t adjoint_smem_bytes(const Prob &pb, bool with_acc);
// The adjoint's scatter of pb.dO (written by an FP32-mode march of the same
// heights) into gacc [n_chains][L][N] (zeroed by the caller; units 2^-24).
// pb.dO holds n_chains * n_rays floats followed by n_chains ints of scratch.
cudaError_t launch_adjoint(const Prob &pb, HRef h, int n_chains, unsigned long long *gacc,
                           cudaStream_t st);
cudaError_t launch_grad_finish(const Prob &pb, int mode, HRef h, const double *mu, int n_chains,
                               const unsigned long long *gacc, double *grad, cudaStream_t st);
cudaError_t launch_add(int n, const double *a, const double *b, double *out, cudaStream_t st);
cudaError_t launch_grad_finish_sel(const Prob &pb, int mode, HRef h, const double *mu, int n_chains,
                                   const unsigned long long *gacc, double *G, const uint8_t *cur,
                                   cudaStream_t st);
cudaError_t launch_scatter_sel(int n_chains, long long n, const double *src, const uint8_t *cur,
                               double *G, cudaStream_t st);
// The gradient samplers take the step size eps, or per chain eps_c[c] when
// eps_c is not null (step-size adaptation).
cudaError_t launch_propose_mala(const Prob &pb, int mode, void *hbuf, long long buf_stride,
                                const double *gbuf, const uint8_t *cur, int n_chains, double eps,
                                const double *eps_c, uint64_t seed, const int64_t *step_base,
                                int step_off, cudaStream_t st);
// HMC with a diagonal inverse metric minv [C][n] (nullptr: unit).
cudaError_t launch_hmc_start(const Prob &pb, int mode, void *hbuf, long long buf_stride,
                             const double *gbuf, const uint8_t *cur, int n_chains, double eps,
                             const double *eps_c, const double *minv, double *pbuf, double *qbuf,
                             double *k0, uint64_t seed, const int64_t *step_base, int step_off,
                             cudaStream_t st);
cudaError_t launch_hmc_kick_drift(const Prob &pb, int mode, void *hbuf, long long buf_stride,
                                  const double *gbuf, const uint8_t *cur, int n_chains, double eps,
                                  const double *eps_c, const double *minv, double *pbuf, double *qbuf,
                                  cudaStream_t st);
cudaError_t launch_hmc_finish(const Prob &pb, long long buf_stride, const double *gbuf,
                              const uint8_t *cur, int n_chains, double eps, const double *eps_c,
                              const double *minv, double *pbuf, const double *k0, double *extra,
                              cudaStream_t st);
cudaError_t launch_mala_hastings(const Prob &pb, int mode, const void *hbuf, long long buf_stride,
                                 const double *gbuf, const uint8_t *cur, int n_chains, double eps,
                                 const double *eps_c, double *extra, cudaStream_t st);
// Capped NUTS (mcmc.cu): the trajectory's two ends (FP64 position, momentum,
// gradient) and the half-kicked momentum, [C][n] each; the trajectory's and
// the current subtree's samples (heights in the storage type, gradients);
// per-chain scalars sc [C][kNS].
constexpr int kNS = 12;
struct NutsBufs {
    double *qL, *pL, *gL, *qR, *pR, *gR, *ph;
    void *hsel, *hsub;
    double *gsel, *gsub, *sc;
};
cudaError_t launch_nuts_start(const Prob &pb, int mode, const void *hbuf, long long bs, const double *gbuf,
                              const uint8_t *cur, int n_chains, const double *minv, const double *ll,
                              const double *lp, const NutsBufs &nb, uint64_t seed, const int64_t *step_base,
                              int step_off, cudaStream_t st);
cudaError_t launch_nuts_drift(const Prob &pb, int mode, void *hbuf, long long bs, const uint8_t *cur,
                              int n_chains, double eps, const double *eps_c, const double *minv,
                              const NutsBufs &nb, uint64_t seed, const int64_t *step_base, int step_off, int j,
                              cudaStream_t st);
cudaError_t launch_nuts_leaf(const Prob &pb, int mode, const void *hbuf, long long bs, const double *gbuf,
                             const uint8_t *cur, int n_chains, double eps, const double *eps_c,
                             const double *minv, const double *llp, const double *lpp, const NutsBufs &nb,
                             uint64_t seed, const int64_t *step_base, int step_off, int j, int leaf,
                             cudaStream_t st);
cudaError_t launch_nuts_merge(const Prob &pb, int mode, int n_chains, const NutsBufs &nb, uint64_t seed,
                              const int64_t *step_base, int step_off, int j, cudaStream_t st);
cudaError_t launch_nuts_finish(const Prob &pb, int mode, void *hbuf, long long bs, double *gbuf,
                               const uint8_t *cur, uint8_t *prop_sel, int n_chains, double *ll, double *lp,
                               double *llp, double *lpp, int64_t *accepts, int32_t *acc_last, double *logu,
                               double *alpha, const NutsBufs &nb, int n_leaves, cudaStream_t st);
// Warm-up adaptation (mcmc.cu): dual-averaging state da [C][6], step sizes
// eps [C]; with metric != 0 the windowed diagonal-metric schedule (Welford
// mean / m2 and the inverse metric minv, [C][n] each).
constexpr int kDAStride = 6;
cudaError_t launch_adapt_init(int n_chains, double eps0, double *da, double *eps, cudaStream_t st);
cudaError_t launch_adapt(int n_chains, double target, int n_adapt, int metric, const double *alpha,
                         double *da, double *eps, cudaStream_t st);
cudaError_t launch_metric_init(size_t n, double *mean, double *m2, double *minv, cudaStream_t st);
cudaError_t launch_metric(const Prob &pb, int mode, const void *hbuf, long long buf_stride,
                          const uint8_t *cur, int n_chains, int n_adapt, double shrink,
                          const double *da, double *mean, double *m2, double *minv, cudaStream_t st);
cudaError_t launch_gather(int mode, HRef h, int n_chains, long long n_per_chain, void *out,
                          cudaStream_t st);
cudaError_t launch_nested_rhat(int mode, const void *draws, int N, int C, int P, int K, double *sm,
                               double *wk, double *rhat, unsigned long long *max_bits, cudaStream_t st);
size_t interface_smem(int n_z);
size_t copula_smem_bytes(const Prob &pb, int mode);
cudaError_t launch_lin(const Prob &pb, int mode, HRef h, int n_chains, int nz, const int *row,
                       const int *col, const void *val, const void *R0, void *dR, const double *lam0,
                       const double *amc, double *fine, double *partial, cudaStream_t st,
                       void *fO = nullptr);
// Gradient of the linearised log-likelihood into the fixed-point accumulators
// gacc [n][L][N] (fO: d ll / d O_p from launch_lin, [ray][Cp]; gR [voxel][Cp]
// and gcell [L][cell][Cp] scratch; cptr / crow / cval the path lengths by
// voxel, from lin_transpose).
cudaError_t launch_lin_grad(const Prob &pb, int mode, HRef h, int n_chains, int nz, const int *cptr,
                            const int *crow, const void *cval, const void *fO, void *gR, void *gcell,
                            unsigned long long *gacc, cudaStream_t st);
void lin_transpose(int n_rays, int nvox, const std::vector<int> &row, const std::vector<int> &col,
                   const std::vector<double> &val, std::vector<int> &cptr, std::vector<int> &crow,
                   std::vector<double> &cval);
cudaError_t launch_lin_reference(const Prob &pb, int mode, HRef h, int nz, void *R0, cudaStream_t st);
size_t lin_fine_partials(const Prob &pb, int n_chains);
cudaError_t launch_lin_amc(int n, const double *lam0, const int32_t *cnt, double *amc, cudaStream_t st);
cudaError_t launch_copula(const Prob &pb, int mode, HRef lat, const void *terrain, void *H, int n_chains,
                          cudaStream_t st);
// Reverse of the copula transform (FP32 latents): the latent gradient from the
// heights' log-likelihood gradient (fixed point, 2^-24) into G[1 - cur[c]][c]
// (cur != nullptr) or G[c], plus the latent log-prior's gradient.
size_t copula_vjp_smem_bytes(const Prob &pb);
cudaError_t launch_copula_vjp(const Prob &pb, HRef lat, HRef hts, const void *terrain,
                              const unsigned long long *gacc, double *G, const uint8_t *cur, int n_chains,
                              cudaStream_t st);
cudaError_t launch_prior_latent(const Prob &pb, int mode, HRef lat, int n_chains, double *lp_out,
                                cudaStream_t st);
cudaError_t launch_interface_std(int mode, const void *samples, int S, int L, int N, int n_z,
                                 const double *z, double *out, cudaStream_t st);

}  // namespace mt
