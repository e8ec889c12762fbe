/*
 * mt.h -- C ABI of libmt.so: muon-tomography log-posterior of layered
 * block-cave geometries, evaluated for many MCMC chains at once on one GB300
 * (sm_103a), with the batched Metropolis update.
 *
 * The calls follow the paper's statement of the problem ("GPU-accelerated
 * Bayesian inference for block-cave geometry recovery via muon tomography"):
 * sensors at known positions in a box-shaped domain (Sec. 2.1.1), pixels as
 * the directions of a solid-angle partition (Sec. 2.1.1), one observed count
 * per pixel (Eq. def_likelihood), a layer model H on an n_rows x n_cols grid
 * with known unit densities (Sec. 2.1.3), and a posterior over H sampled by
 * MCMC that needs only density ratios (Sec. 2.2).
 *
 * Conventions shared by every call
 *  - Every call returns mt_status; the library never aborts, never calls
 *    __trap and never prints.  mt_last_error() gives a message for the last
 *    failing call on that context (library-owned, valid until the next call).
 *  - Coordinates are metres in a box [0,Lx]x[0,Ly]x[0,Lz]; a height is z above
 *    the box floor.  Heights are row-major [chain][layer][row][col], column
 *    (x) fastest; node (r, c) sits at x = c*Lx/(n_cols-1), y = r*Ly/(n_rows-1)
 *    and heights between nodes are bilinear.  Surfaces are ordered bottom to
 *    top; unit u (0..n_layers) lies between surface u-1 and surface u.
 *  - Host arrays passed in are copied; the caller keeps ownership.  Pointers
 *    documented "host or device" may be either (the library asks the CUDA
 *    driver which); device pointers must be on the context's device and are
 *    only borrowed for the duration of the call, on the context's stream.
 *  - Calls are asynchronous on the context's stream unless they write to a
 *    host pointer, in which case they return after the result is on the host.
 *  - Device-side failures (a Poisson draw that ran out of attempts) are
 *    latched in a device status word; mt_sync() reports them as MT_EDEVFLAG.
 *  - A geometry that breaks the ordering is not an error: its log-prior is
 *    -inf and a proposal with it is always rejected.
 *  - One context is used by one host thread at a time.
 */
#ifndef MT_H
#define MT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MT_API __attribute__((visibility("default")))
#else
#define MT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mt_ctx mt_ctx; /* opaque, owned by the library */

typedef enum {
    MT_OK = 0,
    MT_EINVAL = -1,     /* bad argument (size, pointer, range)              */
    MT_ENOMEM = -2,     /* device or host allocation failed                 */
    MT_ESTATE = -3,     /* call order: grid / sensors / pixels / counts /
                           chains not set yet                               */
    MT_ECUDA = -4,      /* a CUDA runtime call failed                       */
    MT_ETIMEDOUT = -5,  /* mt_sync deadline passed, work still in flight    */
    MT_EDEVFLAG = -6,   /* a kernel latched a failure in the status word    */
    MT_ECANCELED = -7   /* a served request was cancelled (mt_server_cancel) */
} mt_status;

/* Arithmetic of the ray march and the per-chain reduction.
 *  MT_PREC_F64  : heights, march, flux and reductions in FP64.
 *  MT_PREC_F32  : FP32 heights and march: each sample's cell fraction and
 *                 sigmoid argument formed from exact products and exact
 *                 differences (heights minus z on fine grids), so they
 *                 round at the scale of one cell and of the distance to the
 *                 surface; each sample's indicator an exact integer in
 *                 units of 2^-28; the logistic from 2^|a| split exactly
 *                 into 2^round(|a|) and a polynomial of the fraction, and a
 *                 reciprocal refined by one Newton step (no bias beyond
 *                 rounding); float-float per-ray flux term and CTA sums,
 *                 FP64 per-chain reduction.  Per-chain log-likelihoods
 *                 within 1e-3 of FP64 (9e-5 on average, 6e-4 at worst over
 *                 2e5 proposals at the scenario size).
 *  MT_PREC_F32C : as MT_PREC_F32 with the per-chain reduction in
 *                 float-float: no FP64 in the ray kernel.
 *  MT_PREC_F32A : as MT_PREC_F32 with the logistic from the SFU's ex2 / rcp
 *                 approximations, their mean error calibrated per device at
 *                 context creation: ~17 % faster; per-chain log-likelihoods
 *                 within ~4e-4 of FP64 on average but up to ~3.4e-3 for
 *                 chains far from the data at the scenario size (the
 *                 approximations' error pattern survives the calibration
 *                 for one-sided transitions).
 *  MT_PREC_BF16 : FP32 chain state; the ray kernel holds each surface as
 *                 BF16 offsets h - ref_l from a reference height ref_l (the
 *                 surface's mean prior height rounded to FP32, or
 *                 Lz (l+1)/(L+1) when that mean is 0) and widens them to FP32
 *                 when read; its march evaluates every sample with the
 *                 SFU's logistic, indicators as integers in units of 2^-23,
 *                 and FP64 per-ray and per-chain sums.  The FP32 modes use
 *                 the same offsets in FP32.
 * Heights passed to and returned by the library are double for MT_PREC_F64
 * and float for every other mode. */
enum { MT_PREC_F64 = 0, MT_PREC_F32 = 1, MT_PREC_F32C = 2, MT_PREC_BF16 = 3, MT_PREC_F32A = 4 };

/* Proposal kernels for mt_run. */
enum { MT_KERNEL_RW = 0, MT_KERNEL_MALA = 1, MT_KERNEL_HMC = 2, MT_KERNEL_NUTS = 3 };

/* Observed-count generation for mt_generate_data. */
enum { MT_COUNTS_POISSON = 0, MT_COUNTS_ROUND = 1 };

typedef struct {
    int precision;     /* MT_PREC_*                                           */
    int n_grid;        /* samples per ray G >= 1: t_k = (k+1/2) t_exit / G    */
    double gamma;      /* sigmoid scale in metres (Eq. def_sigmoid); 0 selects
                          the Heaviside eta with eta(0) = 1/2                 */
    double I0;         /* expected count at zero opacity (1e4)                */
    double atten;      /* attenuation length Lambda in mwe (150):
                          lambda = I0 exp(-O / Lambda)                        */
    double tau;        /* prior precision scale (1/m^2)                        */
    double car_r;      /* CAR spatial dependence r in [0,1) (Eq. def_CAR_precision) */
    double min_thick;  /* minimum thickness delta > 0 between surfaces (m)    */
} mt_config;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to run on (borrowed; NULL = the library creates and owns one).  *out is set
 * on success.  Errors: MT_EINVAL (bad config), MT_ECUDA, MT_ENOMEM.
 * Verification switch: if the environment variable MT_FULL_WINDOWS is set to
 * a value other than "0" when the context is created, its FP32 ray kernels
 * evaluate every sample instead of skipping the exactly saturated ones; the
 * results are bit-identical, only slower. */
MT_API mt_status mt_create(mt_ctx **out, int device, const mt_config *cfg, void *cuda_stream);

/* Release every device buffer, graph and event of the context. NULL is a no-op. */
MT_API mt_status mt_destroy(mt_ctx *ctx);

/* Message for the last failing call on ctx (or on mt_create when ctx is NULL). */
MT_API const char *mt_last_error(const mt_ctx *ctx);

/* Layer model (Sec. 2.1.3): n_layers surfaces (1..8) on an n_rows x n_cols
 * grid (each >= 2), box = {Lx, Ly, Lz} > 0, unit_density[n_layers+1] in g/cc
 * bottom to top (Eq. def_LM_density_grid), prior_mean[n_layers][n_rows][n_cols]
 * (host, may be NULL = zero).  Resets sensors/pixels/counts/chains state that
 * depends on the grid. */
MT_API mt_status mt_set_grid(mt_ctx *ctx, int n_layers, int n_rows, int n_cols, const double box[3],
                      const double *unit_density, const double *prior_mean);

/* Sensor positions (Sec. 2.1.1), host [n_sensors][3], each strictly inside the box. */
MT_API mt_status mt_set_sensors(mt_ctx *ctx, int n_sensors, const double *pos);

/* Pixel directions (Sec. 2.1.1), host [n_pixels][3] unit vectors (|d| within
 * 1e-6 of 1), shared by every sensor; ray (s, p) has index s*n_pixels + p. */
MT_API mt_status mt_set_pixels(mt_ctx *ctx, int n_pixels, const double *dirs);

/* Observed counts C_p >= 0 (Eq. def_likelihood), host or device
 * int32 [n_sensors][n_pixels].  Needs grid, sensors and pixels. */
MT_API mt_status mt_set_counts(mt_ctx *ctx, const int32_t *counts);

/* Synthetic observations from a true geometry: lambda_p from the FP64 march
 * of h_true (host [L][R][Q] double), then C_p ~ Poisson(lambda_p) drawn from
 * Philox4x32-10 stream 1 with key `seed` (count_mode MT_COUNTS_POISSON), or
 * C_p = round-half-even(lambda_p) (MT_COUNTS_ROUND, the paper's Sec. 4).
 * The counts become the context's observed counts.  counts_out / lambda_out
 * (host or device, [S][P], nullable) receive copies. */
MT_API mt_status mt_generate_data(mt_ctx *ctx, const double *h_true, uint64_t seed, int count_mode,
                           int32_t *counts_out, double *lambda_out);

/* Log-likelihood (Eq. def_likelihood, summed over every sensor and pixel) and
 * log-prior of n_chains geometries.  heights: host or device
 * [n_chains][L][R][Q] (double for MT_PREC_F64, float otherwise).
 * loglik_out / logprior_out: host or device double [n_chains], nullable. */
MT_API mt_status mt_logpost(mt_ctx *ctx, int n_chains, const void *heights, double *loglik_out,
                     double *logprior_out);

/* mt_logpost without any device allocation, for callers that cannot
 * allocate: a host that hands out all device memory through its own
 * fixed-budget allocator, or a latency-critical serving loop in which a
 * cudaMalloc / cudaFree (cudaFree synchronises the whole device) must never
 * happen after start-up.  The paper has no counterpart of this call.
 *  - heights, loglik_out and logprior_out (nullable) must be device memory on
 *    the context's device; host pointers are rejected with MT_EINVAL because
 *    staging them would need an allocation.
 *  - The per-(chain, CTA) partial sums live in one 1 MiB array inside the
 *    library (held by every GPU that loads it until the process exits), so
 *    n_chains * ceil(S*P / 6144) * 8 bytes must fit in 1 MiB (11915 chains
 *    of a 16 x 4096-ray problem); larger calls fail with MT_EINVAL.
 *  - The first call on each device looks up the array's device address and
 *    keeps it for the process (so the device's primary context must live as
 *    long as the process: no device reset in between); make that first call
 *    before any stream capture.
 *  - All calls share the array: two calls whose kernels overlap on the GPU
 *    (on different streams or contexts) race and both may return garbage.
 *    Calls on one stream are ordered and safe.
 * Results equal mt_logpost's bit for bit (the same kernels in the same
 * order).  Asynchronous on the context's stream. */
MT_API mt_status mt_logpost_noalloc(mt_ctx *ctx, int n_chains, const void *heights,
                                    double *loglik_out, double *logprior_out);

/* Per-ray opacity O (mwe) and Poisson log-pmf term of n_chains geometries,
 * host or device double [n_chains][S][P] each (nullable): the per-ray values
 * that mt_logpost sums, for element-wise checks. */
MT_API mt_status mt_ray_terms(mt_ctx *ctx, int n_chains, const void *heights, double *opacity_out,
                       double *term_out);

/* Gradient of the log-posterior with respect to every node height
 * (differentiable forward model, Sec. 2.1.4; the hand-written adjoint of the
 * ray march plus -tau Q (h - mu) from the prior): grad_out host or device
 * double [n_chains][L][R][Q]; logpost_out (nullable) double [n_chains].
 * FP32 march arithmetic with 64-bit fixed-point (2^-24) accumulation, so the
 * result is reproducible bit for bit.  Under the copula prior the states and
 * the gradient are latents: the heights' log-likelihood gradient goes back
 * through the stick-breaking, Phi, the Sigma_11(r) normalisation and the
 * spectral filter (z and r gradients, r in the first L-1 entries of plane
 * L-1, the rest of that plane 0), plus -z from the latent log-prior (FP32).
 * Needs gamma > 0 and an FP32 precision mode (MT_EINVAL otherwise); heights
 * (or latents) as for mt_logpost. */
MT_API mt_status mt_grad(mt_ctx *ctx, int n_chains, const void *heights, double *grad_out,
                  double *logpost_out);

/* Start n_chains chains at heights0 (host or device, storage type of the
 * precision) with Philox key `seed`; evaluates their log-posterior.  The step
 * counter restarts at 0. */
MT_API mt_status mt_init_chains(mt_ctx *ctx, int n_chains, const void *heights0, uint64_t seed);

/* Run n_super x n_within Metropolis steps on every chain (Sec. 2.2).
 * kernel MT_KERNEL_RW: H' = H + step * xi; MT_KERNEL_MALA: Langevin proposal
 * H' = H + (eps^2/2) grad(H) + eps xi with eps = step, the gradient from the
 * adjoint (FP32 precision modes, gamma > 0), and the Hastings correction
 * ln q(H|H') - ln q(H'|H) in the accept test; MT_KERNEL_HMC: Hamiltonian
 * Monte Carlo (Sec. 3.1) with a leapfrog trajectory of mt_set_hmc's
 * n_leapfrog steps of size eps = step: momentum p0 = xi / sqrt(m) with
 * xi ~ N(0, I) and m the diagonal inverse metric (1 unless adapted, see
 * mt_set_metric_adapt), p = p0 + eps/2 g, then n_leapfrog times
 * H' += eps m p and p += eps g(H') (eps/2 after the last), the trajectory
 * carried in FP64 and each gradient taken at the stored (rounded) heights;
 * accept term log pi(H') - log pi(H) + K(p0) - K(p), K = p^T m p / 2 (same
 * requirements as MALA); MT_KERNEL_NUTS: the capped NUTS trajectory of
 * mt_set_nuts.  Step k of chain c draws xi from Philox stream 3 (RW), 5
 * (MALA), 6 (HMC) or 7 (NUTS),
 * counter {j, k, c}, and its acceptance uniform from stream 4, counter
 * {0, k, c}.  The n_within steps of a super-step are one CUDA graph replay;
 * the host only sees super-step boundaries.  Asynchronous. */
MT_API mt_status mt_run(mt_ctx *ctx, int kernel, double step, int n_super, int n_within);

/* Leapfrog steps per HMC proposal (1 .. 1024; default 8).  MT_EINVAL outside. */
MT_API mt_status mt_set_hmc(mt_ctx *ctx, int n_leapfrog);

/* Maximum tree depth D of MT_KERNEL_NUTS (1 .. 10; default 8, the paper's
 * cap of 256 steps: 2^8 - 1 = 255 leapfrog steps).  MT_KERNEL_NUTS runs the
 * trajectory NUTS builds when it reaches its cap (Sec. 3.1: the paper caps
 * NUTS at 256 steps and reports that almost every iteration reaches the
 * cap; Hoffman & Gelman 2014): momentum p0 = xi / sqrt(m) (xi from Philox
 * stream 7, counter {pair, step, chain}; m the diagonal inverse metric, 1
 * without mt_set_metric_adapt); for depth j = 0 .. D-1 a direction v_j
 * (stream 8, index j: backwards if its uniform is below 1/2) and 2^j
 * leapfrog steps of size v_j eps from that end of the trajectory; each new
 * state has log-weight ll + lp - p^T M^-1 p / 2 and replaces its subtree's
 * sample when log u < w - W_sub (uniform index 64 + its leaf number, W_sub
 * the subtree's log-sum of weights including it); after each subtree its
 * sample replaces the trajectory's when log u < W_sub - W (index 32 + j),
 * and W accumulates W_sub.  The chain moves to the trajectory's sample; no
 * U-turn stop, no separate accept.  mt_get_last_step reports the sample as
 * the proposal and accepted = whether the chain moved; the step-size
 * adaptation uses the mean of min(1, e^(H_0 - H)) over the 2^D - 1 new
 * states.  Requirements as for HMC.  MT_EINVAL outside 1 .. 10. */
MT_API mt_status mt_set_nuts(mt_ctx *ctx, int max_depth);

/* Step-size adaptation of the gradient samplers (Sec. 3.1: during warm-up
 * the step size is tuned toward a target acceptance probability, 0.8 in the
 * paper) by per-chain dual averaging of log eps (Hoffman & Gelman 2014,
 * Sec. 3.2.1; gamma = 0.05, t0 = 10, kappa = 0.75, mu = log(10 eps0)).
 * n_adapt > 0 turns per-chain step sizes on: the next MALA, HMC or NUTS
 * mt_run starts every chain at eps0 = its `step`, and its first n_adapt
 * gradient-sampler steps (counted across runs) each update chain c's eps
 * from that step's acceptance probability alpha = min(1, e^Delta) (0 outside
 * the prior's support; for NUTS the trajectory's acceptance statistic, see
 * mt_set_nuts); after the n_adapt-th every chain keeps its averaged step
 * size eps_bar, and later MALA / HMC / NUTS runs use it and ignore `step`.  New chains
 * (mt_init_chains) restart the adaptation.  n_adapt = 0 turns it off (the
 * scalar `step` again).  target_accept in (0, 1), n_adapt >= 0, else
 * MT_EINVAL.  Random-walk steps neither use nor change the step sizes. */
MT_API mt_status mt_set_adapt(mt_ctx *ctx, double target_accept, int n_adapt);

/* Diagonal preconditioner of HMC adapted in the same warm-up (Sec. 3.1: the
 * warm-up tunes a diagonal preconditioner together with the step size).
 * With on = 1 the n_adapt warm-up steps armed by mt_set_adapt (n_adapt >= 20,
 * HMC and NUTS; MALA runs are refused while it is on) follow a windowed
 * schedule: an initial buffer, slow windows of doubling length and a
 * terminal buffer (75 / 25 / 50 steps, or 15 % / 75 % / 10 % of n_adapt when
 * those do not fit; the last slow window is stretched to the terminal buffer
 * when the next one would cross it).  During each slow window every chain
 * accumulates the mean and variance of each height of its post-step states
 * (Welford, FP64); at the window's end its inverse metric becomes
 * (n/(n+5)) var + shrink 5/(n+5) (n the window length) and the step-size
 * averaging restarts from mu = log(10 eps).  HMC then draws momenta
 * p ~ N(0, M) with M = diag(1 / inverse metric), drifts H += eps M^-1 p and
 * takes the kinetic energy p^T M^-1 p / 2; the adapted metric is kept after
 * the warm-up.  on = 0: unit metric.  shrink >= 0 (m^2; 1e-3 is the usual
 * default of that schedule).  Re-arms the warm-up (the next HMC run starts
 * it over).  MT_EINVAL on bad arguments. */
MT_API mt_status mt_set_metric_adapt(mt_ctx *ctx, int on, double shrink);

/* Each chain's diagonal inverse metric, host or device double
 * [n_chains][L][R][Q].  Synchronous.  MT_ESTATE before the first HMC run of
 * an armed warm-up with the metric adapted. */
MT_API mt_status mt_get_metric(mt_ctx *ctx, double *inv_metric_out);

/* The per-chain step sizes the next MALA / HMC / NUTS step uses and the
 * acceptance probability of each chain's last adapted step, host or device
 * double [n_chains] each (nullable).  Synchronous.  MT_ESTATE before the
 * first MALA / HMC / NUTS run after mt_set_adapt (or with adaptation off). */
MT_API mt_status mt_get_adapt(mt_ctx *ctx, double *eps_out, double *accept_prob_out);

/* Copy the chains' current state out (each pointer host or device, nullable):
 * heights [C][L][R][Q] storage type, loglik/logprior double [C], accepts
 * int64 [C] (accepted proposals so far), *step_out = steps taken. */
MT_API mt_status mt_get_state(mt_ctx *ctx, void *heights_out, double *loglik_out, double *logprior_out,
                       int64_t *accepts_out, int64_t *step_out);

/* Diagnostics of the most recent step (nullable, host or device):
 * proposal [C][L][R][Q] storage type, its loglik/logprior double [C],
 * accepted int32 [C] (1 = accepted), logu double [C] (ln of the uniform). */
MT_API mt_status mt_get_last_step(mt_ctx *ctx, void *proposal_out, double *loglik_out,
                           double *logprior_out, int32_t *accepted_out, double *logu_out);

/* Resume: overwrite the current heights (host or device) and set the step
 * counter; log-posteriors are re-evaluated.  Acceptance counters are kept. */
MT_API mt_status mt_set_state(mt_ctx *ctx, const void *heights, int64_t step);

/* Wait for the context's stream, at most timeout_s seconds (<= 0: no limit).
 * MT_ETIMEDOUT if work is still in flight at the deadline (the context stays
 * usable); MT_EDEVFLAG if a kernel latched a failure (the flag is cleared). */
MT_API mt_status mt_sync(mt_ctx *ctx, double timeout_s);

/* Kernel timing: when on, the library brackets each launch of the ray kernel
 * (id 0) and each whole Metropolis step (id 1) with CUDA events on its stream
 * and does not use graphs.  mt_get_timing returns the summed milliseconds and
 * the launch count since the last reset (reset = 1 clears them). */
MT_API mt_status mt_set_timing(mt_ctx *ctx, int on);
MT_API mt_status mt_get_timing(mt_ctx *ctx, int id, double *total_ms, int64_t *launches, int reset);

/* Work of the FP32 ray kernel launched while timing was on: *total = the
 * method's surface-samples (chains x rays x n_grid x n_layers), *evaluated =
 * those whose logistic was computed; the others lay so far from their surface
 * (|s - z| >= 29.25 gamma / log2(e)) that their integer indicator (units of
 * 2^-28) is exactly 0 or 2^28 and was added without evaluation (the result
 * is bit-identical).
 * reset = 1 clears both. */
MT_API mt_status mt_get_work(mt_ctx *ctx, double *evaluated, double *total, int reset);

/* Sizes of the loaded problem (any pointer nullable). */
MT_API mt_status mt_get_sizes(const mt_ctx *ctx, int *n_layers, int *n_rows, int *n_cols,
                       int *n_sensors, int *n_pixels, int *n_chains);

/* ------------------------------------------------------------------------
 * Prior.
 *
 * MT_PRIOR_CAR (the default): chain states are heights; the log-prior is the
 * CAR quadratic form -tau/2 sum_l (h_l - mu_l)^T (4I - rA)(h_l - mu_l) with
 * the hard ordering / bounds constraints (see mt_config).
 *
 * MT_PRIOR_COPULA: the paper's prior (Sec. 2.2.1).  Chain states are latents
 * laid out like heights [L][R][Q]: planes 0 .. L-2 hold standard-normal
 * fields z_l, the first L-1 entries of plane L-1 hold the spatial-dependence
 * parameters r_l (prior U(0, 1)); the rest of plane L-1 is ignored.  Heights:
 * x_l = Q(r_l)^-1/2 z_l with Q(r) = 4I - rA on the periodic grid (Eq.
 * def_CAR_precision; the symmetric square root, applied with 2-D discrete
 * Fourier transforms, where the paper uses a Cholesky factor: both give x the
 * law N(0, Q^-1)), u_l = Phi(x_l / sqrt(Sigma_11)) (Eq. CAR_cdf_transform),
 * H_l = H_{l-1} + u_l (T - H_{l-1}) with H_{-1} = 0 (Eq. indep_columns), and
 * the top surface L-1 is the known terrain T = the prior mean's top plane.
 * Log-prior in latent coordinates: -1/2 sum z^2 if every r_l is in (0, 1),
 * else -inf.  mt_logpost, mt_ray_terms, mt_init_chains, mt_set_state and
 * mt_get_state then take and return latents; random-walk, MALA, HMC and
 * capped-NUTS steps move the latents (their gradient comes back through the
 * transform, see mt_grad).  mt_logpost_noalloc needs the CAR prior.
 * Switching drops the chains; mt_set_grid resets the prior to MT_PRIOR_CAR.
 * Errors: MT_EINVAL (kind, fewer than 2 surfaces, grids whose transform does
 * not fit in shared memory: 4 R Q values of the height dtype), MT_ESTATE. */
#define MT_PRIOR_CAR 0
#define MT_PRIOR_COPULA 1
MT_API mt_status mt_set_prior(mt_ctx *ctx, int kind);

/* Heights [n][L][R][Q] (host or device, height dtype) of n latent states
 * (same layout and dtype) under the copula prior.  MT_ESTATE unless the
 * copula prior is set. */
MT_API mt_status mt_copula_heights(mt_ctx *ctx, int n, const void *latent, void *heights_out);

/* ------------------------------------------------------------------------
 * Forward model.
 *
 * MT_FORWARD_MARCH (the default): every ray is marched at n_grid samples.
 * MT_FORWARD_LINEAR: the paper's linearised model (Sec. 2.1.2, Eqs.
 * expected_counts_linearized / _approx) on a voxel density grid (Sec. 2.1.4,
 * Eq. def_LM_density_grid_smooth): voxels are the (R-1) x (Q-1) cells of the
 * surface grid times n_z levels of height box[2] / n_z; a voxel's density is
 * rho_top + sum_l (rho_l - rho_{l+1}) varsigma(h_l - z_k) with h_l the mean of
 * the cell's four corner heights and z_k the level's centre; L_pv = the
 * length of ray p inside voxel v (built once on the host in FP64, stored in
 * the height dtype); lambda_hat_p = lambda_p(R0) (1 - sum_v L_pv (R_v - R0_v)
 * / Lambda) with R0 the densities of h_ref ([L][R][Q] host FP64; NULL = the
 * prior mean).  The Poisson log-likelihood is -inf when some lambda_hat_p <=
 * 0.  mt_logpost, random-walk steps, gradients (mt_grad: the chain rule
 * d ll / d O_p = (C_p / lambda_hat_p - 1) (-lambda_p(R0) / Lambda), the path
 * lengths by voxel, the cell-centre sigmoids' derivatives, 1/4 to each
 * corner node; gamma > 0) and so MALA, HMC and capped NUTS then use it;
 * mt_ray_terms and mt_logpost_noalloc need the march.  Live chains are
 * re-evaluated.  mt_set_grid / mt_set_sensors / mt_set_pixels reset the
 * model to the march.
 * Errors: MT_EINVAL (kind, n_z outside 1..4096), MT_ESTATE (grid, sensors or
 * pixels missing). */
#define MT_FORWARD_MARCH 0
#define MT_FORWARD_LINEAR 1
MT_API mt_status mt_set_forward(mt_ctx *ctx, int kind, int n_z, const double *h_ref);

/* ------------------------------------------------------------------------
 * Chain diagnostics.
 *
 * Nested R-hat (Sec. 3.2: chains grouped into super-chains that share a
 * start, to detect chains stuck near it; statistic of Margossian et al. 2024)
 * of every height over stored draws.  draws: [n_draws][n_chains][L][R][Q],
 * host or device, FP64 in MT_PREC_F64 and FP32 otherwise (what
 * mt_get_state returns).  Chains c = k*M .. k*M + M - 1 form super-chain k,
 * M = n_chains / n_super.  Per height: B = variance of the super-chain means
 * (divisor n_super - 1); W = mean over super-chains of the variance of their
 * chain means (divisor M - 1, 0 if M = 1) plus the mean within-chain variance
 * (divisor n_draws - 1, 0 if n_draws = 1); R = sqrt(1 + B / W), 1 if
 * B = W = 0.  rhat_out: [L*R*Q] (host or device, nullable); rhat_max_out:
 * host, nullable.  FP64.  Errors: MT_EINVAL (n_draws < 1, n_super < 2 or not
 * dividing n_chains, null draws), MT_ESTATE (no grid). */
MT_API mt_status mt_nested_rhat(mt_ctx *ctx, int n_draws, int n_chains, const void *draws, int n_super,
                                double *rhat_out, double *rhat_max_out);

/* Tomographic standard deviation of the below-interface indicators
 * B^l_{ijk}(H) = eta(H_{l,i,j} - z_k), eta(0) = 1/2 (Eq.
 * def_below_interface_indicator; Sec. 4, Fig. tomography_std_poisson) over
 * n_samples height sets: voxel columns at the surface nodes, levels
 * z_k = k * box[2] / n_z, k = 0 .. n_z - 1 (box as given to mt_set_grid;
 * heights are measured from the box floor).  Population standard deviation
 * sqrt(mean(B^2) - mean(B)^2), in [0, 1/2].  samples: [n_samples][L][R][Q],
 * host or device, dtype as for mt_nested_rhat; std_out: [L][n_z][R][Q]
 * doubles, host or device.  Errors: MT_EINVAL (n_samples < 1, n_z outside
 * 1..4096, null pointers), MT_ESTATE (no grid). */
MT_API mt_status mt_interface_std(mt_ctx *ctx, int n_samples, const void *samples, int n_z,
                                  double *std_out);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of inversion requests on one GPU.
 *
 * A request is a whole inversion (Sec. 2: problem, data, prior and an MCMC
 * run): grid, sensors, pixels, counts (or a true geometry to draw them from),
 * chain starts and a step budget.  The server admits queued requests in
 * arrival order while their estimated device memory fits the budget and a
 * slot is free; each admitted request keeps its chains resident in its own
 * context and stream, and gets its next super-step (one graph replay of
 * n_within steps) as soon as the previous one finishes, so the work of
 * different requests overlaps on the device.  Finished requests free their
 * memory and slot for the next ones.  A request's result depends only on its
 * own inputs and seeds: it is the same alone and in any mix.
 * ---------------------------------------------------------------------- */
typedef struct mt_server mt_server; /* opaque, owned by the library */

typedef struct {
    mt_config cfg;
    int n_layers, n_rows, n_cols;
    const double *box;            /* [3] */
    const double *unit_density;   /* [n_layers + 1] */
    const double *prior_mean;     /* [L][R][Q] or NULL */
    int n_sensors;
    const double *sensors;        /* [S][3] */
    int n_pixels;
    const double *dirs;           /* [P][3] unit vectors */
    const int32_t *counts;        /* [S][P], or NULL: Poisson counts drawn from h_true */
    const double *h_true;         /* [L][R][Q], used when counts is NULL */
    uint64_t data_seed;
    int n_chains;
    const void *heights0;         /* [C][L][R][Q], storage type of cfg.precision */
    uint64_t seed;                /* Philox key of the chains */
    int kernel;                   /* MT_KERNEL_RW or MT_KERNEL_MALA */
    double step;                  /* random-walk sigma or MALA eps */
    int n_super, n_within;        /* super-steps and steps per super-step */
} mt_request;

typedef struct {
    int status;                   /* MT_OK or the request's error */
    int n_supersteps;
    double submit_s, admit_s, done_s;          /* server clock, seconds */
    double superstep_ms_p50, superstep_ms_p99; /* CUDA-event time per super-step */
    /* device clock (CUDA events, ms from an event the server records at
     * creation): start of the request's first super-step, end of its last,
     * and the sum of its super-steps' durations.  Two requests whose
     * [gpu_start_ms, gpu_end_ms] spans intersect had work on the device at
     * the same time. */
    double gpu_start_ms, gpu_end_ms, gpu_busy_ms;
} mt_request_info;

typedef struct {
    int64_t n_done, n_pending, n_active;
    double superstep_ms_p50, superstep_ms_p99; /* over all finished requests */
    double ttp_s_p50, ttp_s_p99;               /* time to posterior: submit -> done */
    double chain_ray_evals_per_s;              /* finished work / (last done - first admit) */
    size_t bytes_in_use;                       /* estimated device memory of active requests */
    /* the server's device-memory pool: bytes it held once creation had
     * filled it, and now; equal while no request needed more than the pool
     * held, i.e. no request's memory came from the driver */
    size_t pool_bytes_at_start, pool_bytes_now;
} mt_server_stats_t;

/* Start a server on `device` with a device-memory budget (bytes) and at most
 * max_active requests in flight.  A host thread runs the scheduler.
 * Creation reserves the device memory requests draw from: a stream-ordered
 * pool that keeps up to the budget and is filled here with min(budget,
 * 32 GiB); each request's contexts allocate from it and give it back on their
 * own stream, so admitting and finishing a request neither calls cudaMalloc /
 * cudaFree nor synchronises the device.  The max_active streams and events
 * the requests run on are created here too and reused. */
MT_API mt_status mt_server_create(mt_server **out, int device, size_t hbm_budget_bytes,
                                  int max_active);

/* Queue a request (host arrays, copied).  MT_ENOMEM if it alone needs more than
 * the budget; MT_EINVAL for an incomplete request or a kernel other than
 * MT_KERNEL_RW / MT_KERNEL_MALA.  *id_out names it. */
MT_API mt_status mt_server_submit(mt_server *s, const mt_request *req, int64_t *id_out);

/* Wait for request `id` (timeout_s <= 0: no limit; MT_ETIMEDOUT otherwise) and
 * copy its final chains out (host pointers, nullable): heights [C][L][R][Q],
 * loglik / logprior double [C], accepts int64 [C]; info (nullable) gets its
 * timing.  Returns the request's own error if it failed. */
MT_API mt_status mt_server_wait(mt_server *s, int64_t id, double timeout_s, void *heights_out,
                                double *loglik_out, double *logprior_out, int64_t *accepts_out,
                                mt_request_info *info);

/* Cancel request `id`: a queued request is dropped at once; a running one
 * stops at its next super-step boundary (no kernel is interrupted) and
 * releases its device memory.  Either way mt_server_wait then returns
 * MT_ECANCELED.  MT_ESTATE if the request had already finished, MT_EINVAL
 * for an unknown id. */
MT_API mt_status mt_server_cancel(mt_server *s, int64_t id);

/* Aggregate latency and throughput of the requests finished so far. */
MT_API mt_status mt_server_stats(mt_server *s, mt_server_stats_t *out);

/* Stop the scheduler (requests still queued or running end with MT_ESTATE,
 * waking their waiters) and free all. */
MT_API mt_status mt_server_destroy(mt_server *s);

MT_API const char *mt_server_last_error(const mt_server *s);

#ifdef __cplusplus
}
#endif

#endif /* MT_H */
