// mcmc.cu -- per-chain kernels around the ray march: random-walk proposal,
// log-prior, fixed-order reduction + Metropolis accept, state gather.
//
// The Metropolis step needs only the ratio of posterior densities (Sec. 2.2):
// accept iff the proposal's prior is finite and ln u < (ll' + lp') - (ll + lp).
// Chain state is double-buffered: cur[c] says which of the two height buffers
// holds chain c; a proposal is written to the other one and an accept just
// flips cur[c], so no heights are copied.
#include <math.h>

#include "march.cuh"
#include "philox.cuh"

namespace mt {

// ---------------------------------------------------------------- prior
// lp = -tau/2 sum_l (h_l - mu_l)^T Q (h_l - mu_l), Q = diag(A 1) - r A on the
// periodic 4-neighbour grid (Eq. def_CAR_precision, Fig. neighbors), and -inf
// unless every height is in [0, Lz] and every thickness is >= delta (Sec.
// 2.1.3, strictly positive thicknesses).  With e = h - mu, the quadratic form
// is sum_nodes e (4 e - r (e_up + e_down + e_right + e_left))
//   = 4 sum e^2 - 2 r sum_nodes e (e_right + e_up)
// (each neighbour pair appears twice in the first sum; the identity also holds
// where a side of 2 or 1 nodes makes the wrap-around neighbours coincide).
// One block per chain; each thread walks nodes i, i + 256, ... with its
// (layer, row, col) stepped incrementally.
constexpr int kPriorThreads = 256;

struct NodeWalk {
    int l, r, c, dr, dc;
    __device__ NodeWalk(int i, int N, int Q) : l(i / N), r((i % N) / Q), c(i % Q), dr(kPriorThreads / Q), dc(kPriorThreads % Q) {}
    __device__ void next(int R, int Q)
    {
        c += dc;
        r += dr;
        if (c >= Q) {
            c -= Q;
            ++r;
        }
        while (r >= R) {
            r -= R;
            ++l;
        }
    }
};

// FP64 heights (F64 mode): FP64 arithmetic.
__global__ void __launch_bounds__(kPriorThreads) k_prior_f64(Prob pb, HRef h, const double *mu, double *lp_out)
{
    const int c = blockIdx.x;
    const double *Hc = chain_ptr<double>(h, c);
    const int N = pb.N, Q = pb.Q, R = pb.R, n = pb.L * N;
    double q1 = 0.0, q2 = 0.0;
    int bad = 0;
    NodeWalk wk(threadIdx.x, N, Q);
    for (int i = threadIdx.x; i < n; i += kPriorThreads, wk.next(R, Q)) {
        const int base = wk.l * N, rt = wk.c + 1 == Q ? 0 : wk.c + 1, up = wk.r + 1 == R ? 0 : wk.r + 1;
        const double hv = Hc[i];
        if (!(hv >= 0.0 && hv <= pb.box[2])) bad = 1;
        if (wk.l > 0 && !(hv - Hc[i - N] >= pb.delta)) bad = 1;
        const int iR = base + wk.r * Q + rt, iU = base + up * Q + wk.c;
        const double e = hv - mu[i];
        const double t = (Hc[iR] - mu[iR]) + (Hc[iU] - mu[iU]);
        q1 = fma(e, e, q1);
        q2 = fma(e, t, q2);
    }
    const double quad = block_sum(4.0 * q1 - 2.0 * pb.car_r * q2);
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) lp_out[c] = bad ? -INFINITY : -0.5 * pb.tau * quad;
}

// e = h - mu as a float-float (h a float, mu = mu_ff.x + mu_ff.y).
__device__ __forceinline__ FF ff_dev(float hv, float2 m)
{
    return ff_add(ff_two_sum(hv, -m.x), FF{-m.y, 0.f});
}

// FP32 heights: float-float arithmetic on the FP32 pipes (relative error
// ~2^-44 of the quadratic form; FP64 runs at a small fraction of the FP32
// rate here).  Bounds and thicknesses are decided exactly: h <= Lz as
// h <= the largest float <= Lz, and h_l - h_{l-1} (exact as a float-float
// two-sum) against delta as a float-float.
__global__ void __launch_bounds__(kPriorThreads) k_prior_f32(Prob pb, HRef h, double *lp_out)
{
    const int c = blockIdx.x;
    const float *Hc = chain_ptr<float>(h, c);
    const float2 *mu = pb.mu_ff;
    const int N = pb.N, Q = pb.Q, R = pb.R, n = pb.L * N;
    FF q1 = {0.f, 0.f}, q2 = {0.f, 0.f};
    int bad = 0;
    NodeWalk wk(threadIdx.x, N, Q);
    for (int i = threadIdx.x; i < n; i += kPriorThreads, wk.next(R, Q)) {
        const int base = wk.l * N, rt = wk.c + 1 == Q ? 0 : wk.c + 1, up = wk.r + 1 == R ? 0 : wk.r + 1;
        const float hv = Hc[i];
        if (!(hv >= 0.0f && hv <= pb.lz_f)) bad = 1;
        if (wk.l > 0) {
            const FF d = ff_two_sum(hv, -Hc[i - N]);
            if (d.hi < pb.delta_ff.x || (d.hi == pb.delta_ff.x && d.lo < pb.delta_ff.y)) bad = 1;
        }
        const int iR = base + wk.r * Q + rt, iU = base + up * Q + wk.c;
        const FF e = ff_dev(hv, mu[i]);
        const FF t = ff_add(ff_dev(Hc[iR], mu[iR]), ff_dev(Hc[iU], mu[iU]));
        q1 = ff_add(q1, ff_mul(e, e));
        q2 = ff_add(q2, ff_mul(e, t));
    }
    q1 = block_sum(q1);
    __syncthreads();  // block_sum reuses its shared buffer
    q2 = block_sum(q2);
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        const double quad = 4.0 * ((double)q1.hi + (double)q1.lo) - 2.0 * pb.car_r * ((double)q2.hi + (double)q2.lo);
        lp_out[c] = bad ? -INFINITY : -0.5 * pb.tau * quad;
    }
}

cudaError_t launch_prior(const Prob &pb, int mode, HRef h, const double *mu, int n_chains,
                         double *lp_out, cudaStream_t st)
{
    if (mode == MODE_F64) k_prior_f64<<<n_chains, kPriorThreads, 0, st>>>(pb, h, mu, lp_out);
    else k_prior_f32<<<n_chains, kPriorThreads, 0, st>>>(pb, h, lp_out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- proposal
// Random walk H' = H + sigma xi; the normal pair (xi_2j, xi_2j+1) comes from
// Philox stream PROP, counter {j, step, chain} by Box-Muller.
template <typename H>
__global__ void __launch_bounds__(256)
k_propose_rw(int n, H *hbuf, long long buf_stride, const uint8_t *cur, double sigma, uint64_t seed,
             const int64_t *step_base, int step_off)
{
    const int c = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * j >= n) return;
    const uint32_t step = (uint32_t)(*step_base + step_off);
    const uint4 w = draw4(seed, STREAM_PROP, (uint32_t)c, step, (uint32_t)j);
    const int cs = cur[c];
    const H *src = hbuf + (long long)cs * buf_stride + (long long)c * n;
    H *dst = hbuf + (long long)(1 - cs) * buf_stride + (long long)c * n;
    if constexpr (sizeof(H) == 8) {
        const double u1 = u01_f64(w.x, w.y), u2 = u01_f64(w.z, w.w);
        const double rad = sqrt(-2.0 * log(u1));
        double sn, cn;
        sincospi(2.0 * u2, &sn, &cn);
        dst[2 * j] = src[2 * j] + sigma * (rad * cn);
        if (2 * j + 1 < n) dst[2 * j + 1] = src[2 * j + 1] + sigma * (rad * sn);
    } else {
        const float u1 = u01_to_f32(w.x, w.y), u2 = u01_to_f32(w.z, w.w);
        const float rad = sqrtf(-2.0f * logf(u1));
        float sn, cn;
        sincospif(2.0f * u2, &sn, &cn);
        const float sg = (float)sigma;
        dst[2 * j] = fmaf(sg, rad * cn, src[2 * j]);
        if (2 * j + 1 < n) dst[2 * j + 1] = fmaf(sg, rad * sn, src[2 * j + 1]);
    }
}

cudaError_t launch_propose_rw(const Prob &pb, int mode, void *hbuf, long long buf_stride,
                              const uint8_t *cur, int n_chains, double sigma, uint64_t seed,
                              const int64_t *step_base, int step_off, cudaStream_t st)
{
    const int n = pb.L * pb.N;
    dim3 grid((n / 2 + 1 + 255) / 256, n_chains);
    if (mode == MODE_F64)
        k_propose_rw<double><<<grid, 256, 0, st>>>(n, (double *)hbuf, buf_stride, cur, sigma, seed,
                                                   step_base, step_off);
    else
        k_propose_rw<float><<<grid, 256, 0, st>>>(n, (float *)hbuf, buf_stride, cur, sigma, seed,
                                                  step_base, step_off);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- MALA
// Langevin proposal H' = H + (eps^2/2) grad(H) + eps xi, xi from Philox stream
// MALA, counter {j, step, chain}; grad holds the log-posterior gradient of the
// current state (double, [2][C][n], buffer chosen by cur like the heights).
template <typename H>
__global__ void __launch_bounds__(256)
k_propose_mala(int n, H *hbuf, long long buf_stride, const double *gbuf, const uint8_t *cur,
               double eps0, const double *eps_c, uint64_t seed, const int64_t *step_base, int step_off)
{
    const int c = blockIdx.y;
    const double eps = eps_c ? eps_c[c] : eps0;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (2 * j >= n) return;
    const uint32_t step = (uint32_t)(*step_base + step_off);
    const uint4 w = draw4(seed, STREAM_MALA, (uint32_t)c, step, (uint32_t)j);
    const int cs = cur[c];
    const long long off = (long long)cs * buf_stride + (long long)c * n;
    const long long dst = (long long)(1 - cs) * buf_stride + (long long)c * n;
    const double u1 = u01_f64(w.x, w.y), u2 = u01_f64(w.z, w.w);
    const double rad = sqrt(-2.0 * log(u1));
    double sn, cn;
    sincospi(2.0 * u2, &sn, &cn);
    const double half = 0.5 * eps * eps;
    hbuf[dst + 2 * j] = (H)((double)hbuf[off + 2 * j] + half * gbuf[off + 2 * j] + eps * (rad * cn));
    if (2 * j + 1 < n)
        hbuf[dst + 2 * j + 1] =
            (H)((double)hbuf[off + 2 * j + 1] + half * gbuf[off + 2 * j + 1] + eps * (rad * sn));
}

cudaError_t launch_propose_mala(const Prob &pb, int mode, void *hbuf, long long buf_stride,
                                const double *gbuf, const uint8_t *cur, int n_chains, double eps,
                                const double *eps_c, uint64_t seed, const int64_t *step_base,
                                int step_off, cudaStream_t st)
{
    const int n = pb.L * pb.N;
    dim3 grid((n / 2 + 1 + 255) / 256, n_chains);
    if (mode == MODE_F64)
        k_propose_mala<double><<<grid, 256, 0, st>>>(n, (double *)hbuf, buf_stride, gbuf, cur, eps,
                                                     eps_c, seed, step_base, step_off);
    else
        k_propose_mala<float><<<grid, 256, 0, st>>>(n, (float *)hbuf, buf_stride, gbuf, cur, eps,
                                                    eps_c, seed, step_base, step_off);
    return cudaGetLastError();
}

// Hastings term ln q(H | H') - ln q(H' | H) with q(b | a) = N(a + (eps^2/2) g(a), eps^2 I),
// from the stored heights and gradients in FP64; one block per chain.
template <typename H>
__global__ void __launch_bounds__(256)
k_mala_hastings(int n, const H *hbuf, long long buf_stride, const double *gbuf, const uint8_t *cur,
                double eps0, const double *eps_c, double *extra)
{
    const int c = blockIdx.x;
    const double eps = eps_c ? eps_c[c] : eps0;
    const int cs = cur[c];
    const long long a = (long long)cs * buf_stride + (long long)c * n;       // current
    const long long b = (long long)(1 - cs) * buf_stride + (long long)c * n; // proposal
    const double half = 0.5 * eps * eps;
    double fwd = 0.0, rev = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double ha = (double)hbuf[a + i], hb = (double)hbuf[b + i];
        const double rf = hb - ha - half * gbuf[a + i];
        const double rr = ha - hb - half * gbuf[b + i];
        fwd += rf * rf;
        rev += rr * rr;
    }
    fwd = block_sum(fwd);
    __syncthreads();
    rev = block_sum(rev);
    if (threadIdx.x == 0) extra[c] = (fwd - rev) / (2.0 * eps * eps);
}

cudaError_t launch_mala_hastings(const Prob &pb, int mode, const void *hbuf, long long buf_stride,
                                 const double *gbuf, const uint8_t *cur, int n_chains, double eps,
                                 const double *eps_c, double *extra, cudaStream_t st)
{
    const int n = pb.L * pb.N;
    if (mode == MODE_F64)
        k_mala_hastings<double><<<n_chains, 256, 0, st>>>(n, (const double *)hbuf, buf_stride, gbuf,
                                                          cur, eps, eps_c, extra);
    else
        k_mala_hastings<float><<<n_chains, 256, 0, st>>>(n, (const float *)hbuf, buf_stride, gbuf,
                                                         cur, eps, eps_c, extra);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- HMC
// Hamiltonian Monte Carlo with a leapfrog trajectory (Sec. 3.1, the building
// block of the paper's NUTS).  Momentum p0 = xi / sqrt(m), xi ~ N(0, I) from
// Philox stream HMC, counter {pair j, step, chain}, m the diagonal inverse
// metric (1 unless adapted); p = p0 + eps/2 g(q0); n_leap times:
// q += eps m p, then p += eps g(q) (eps/2 after the last drift).
// The trajectory q is carried in FP64 (qbuf); the proposal buffer holds it
// rounded to the height dtype, which is where the gradient and the
// log-density are evaluated.  Gradients: G[1 - cur] (the proposal's), G[cur]
// (the current state's), FP64 like the momentum.  The accept term is
// K(p0) - K(p), K = p^T m p / 2.
template <typename H>
__global__ void __launch_bounds__(256)
k_hmc_start(int n, H *hbuf, long long bs, const double *gbuf, const uint8_t *cur, double eps0,
            const double *eps_c, const double *minv, double *pbuf, double *qbuf, double *k0, uint64_t seed,
            const int64_t *step_base, int step_off)
{
    const int c = blockIdx.x;
    const double eps = eps_c ? eps_c[c] : eps0;
    const uint32_t step = (uint32_t)(*step_base + step_off);
    const int cs = cur[c];
    const long long a = (long long)cs * bs + (long long)c * n;
    const long long b = (long long)(1 - cs) * bs + (long long)c * n;
    double kin = 0.0;
    for (int j = threadIdx.x; 2 * j < n; j += blockDim.x) {
        const uint4 w = draw4(seed, STREAM_HMC, (uint32_t)c, step, (uint32_t)j);
        const double u1 = u01_f64(w.x, w.y), u2 = u01_f64(w.z, w.w);
        const double rad = sqrt(-2.0 * log(u1));
        double sn, cn;
        sincospi(2.0 * u2, &sn, &cn);
        const double xi[2] = {rad * cn, rad * sn};
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int i = 2 * j + t;
            if (i >= n) break;
            kin += 0.5 * xi[t] * xi[t];  // K(p0) = p0^2 minv / 2 with p0 = xi / sqrt(minv)
            const double mi = minv ? minv[(size_t)c * n + i] : 1.0;
            const double p = (minv ? xi[t] / sqrt(mi) : xi[t]) + 0.5 * eps * gbuf[a + i];
            const double q = (double)hbuf[a + i] + eps * (mi * p);
            pbuf[(size_t)c * n + i] = p;
            qbuf[(size_t)c * n + i] = q;
            hbuf[b + i] = (H)q;
        }
    }
    kin = block_sum(kin);
    if (threadIdx.x == 0) k0[c] = kin;
}

template <typename H>
__global__ void __launch_bounds__(256)
k_hmc_kick_drift(int n, H *hbuf, long long bs, const double *gbuf, const uint8_t *cur, double eps0,
                 const double *eps_c, const double *minv, double *pbuf, double *qbuf)
{
    const int c = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double eps = eps_c ? eps_c[c] : eps0;
    const long long b = (long long)(1 - cur[c]) * bs + (long long)c * n;
    const size_t k = (size_t)c * n + i;
    const double p = pbuf[k] + eps * gbuf[b + i];
    const double q = qbuf[k] + eps * ((minv ? minv[k] : 1.0) * p);
    pbuf[k] = p;
    qbuf[k] = q;
    hbuf[b + i] = (H)q;
}

__global__ void __launch_bounds__(256)
k_hmc_finish(int n, long long bs, const double *gbuf, const uint8_t *cur, double eps0,
             const double *eps_c, const double *minv, const double *pbuf, const double *k0, double *extra)
{
    const int c = blockIdx.x;
    const double eps = eps_c ? eps_c[c] : eps0;
    const long long b = (long long)(1 - cur[c]) * bs + (long long)c * n;
    double kin = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double p = pbuf[(size_t)c * n + i] + 0.5 * eps * gbuf[b + i];
        kin += 0.5 * (minv ? minv[(size_t)c * n + i] : 1.0) * p * p;
    }
    kin = block_sum(kin);
    if (threadIdx.x == 0) extra[c] = k0[c] - kin;
}

cudaError_t launch_hmc_start(const Prob &pb, int mode, void *hbuf, long long buf_stride,
                             const double *gbuf, const uint8_t *cur, int n_chains, double eps,
                             const double *eps_c, const double *minv, double *pbuf, double *qbuf,
                             double *k0, uint64_t seed, const int64_t *step_base, int step_off,
                             cudaStream_t st)
{
    const int n = pb.L * pb.N;
    if (mode == MODE_F64)
        k_hmc_start<double><<<n_chains, 256, 0, st>>>(n, (double *)hbuf, buf_stride, gbuf, cur, eps, eps_c,
                                                      minv, pbuf, qbuf, k0, seed, step_base, step_off);
    else
        k_hmc_start<float><<<n_chains, 256, 0, st>>>(n, (float *)hbuf, buf_stride, gbuf, cur, eps, eps_c,
                                                     minv, pbuf, qbuf, k0, seed, step_base, step_off);
    return cudaGetLastError();
}

cudaError_t launch_hmc_kick_drift(const Prob &pb, int mode, void *hbuf, long long buf_stride,
                                  const double *gbuf, const uint8_t *cur, int n_chains, double eps,
                                  const double *eps_c, const double *minv, double *pbuf, double *qbuf,
                                  cudaStream_t st)
{
    const int n = pb.L * pb.N;
    dim3 grid((n + 255) / 256, n_chains);
    if (mode == MODE_F64)
        k_hmc_kick_drift<double><<<grid, 256, 0, st>>>(n, (double *)hbuf, buf_stride, gbuf, cur, eps,
                                                       eps_c, minv, pbuf, qbuf);
    else
        k_hmc_kick_drift<float><<<grid, 256, 0, st>>>(n, (float *)hbuf, buf_stride, gbuf, cur, eps,
                                                      eps_c, minv, pbuf, qbuf);
    return cudaGetLastError();
}

cudaError_t launch_hmc_finish(const Prob &pb, long long buf_stride, const double *gbuf,
                              const uint8_t *cur, int n_chains, double eps, const double *eps_c,
                              const double *minv, double *pbuf, const double *k0, double *extra,
                              cudaStream_t st)
{
    k_hmc_finish<<<n_chains, 256, 0, st>>>(pb.L * pb.N, buf_stride, gbuf, cur, eps, eps_c, minv, pbuf, k0,
                                           extra);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- capped NUTS
// The trajectory NUTS (Sec. 3.1; Hoffman & Gelman 2014) builds when it runs
// to its cap of 2^D - 1 leapfrog steps, as the paper reports almost every
// iteration did: momentum p0 = xi / sqrt(m) (Philox stream NUTS_P, counter
// {pair, step, chain}); for depth j = 0 .. D-1 a direction v_j (stream
// NUTS_U, index j: -1 if u < 1/2) and 2^j leapfrog steps of size v_j eps from
// that end of the trajectory; every new state n gets log-weight
// w_n = -H_n = ll + lp - K(p) and may replace the subtree's sample
// (log u < w_n - W_sub after adding w_n, index 64 + leaf); after each subtree
// its sample replaces the trajectory's when log u < W_sub - W (index
// 32 + j), then W = logaddexp(W, W_sub).  The chain moves to the trajectory's
// sample.  Ends (FP64 position, momentum, gradient) per side, [C][n] each;
// per-chain scalars sc[kNS * c + ...].
enum { NS_W = 0, NS_WSUB, NS_H0, NS_LLSEL, NS_LPSEL, NS_LLSUB, NS_LPSUB, NS_STAT, NS_MOVED };

__device__ __forceinline__ double nuts_u(uint64_t seed, int c, uint32_t step, uint32_t index)
{
    const uint4 w = draw4(seed, STREAM_NUTS_U, (uint32_t)c, step, index);
    return u01_f64(w.x, w.y);
}

__device__ __forceinline__ double logaddexp_d(double a, double b)
{
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    const double m = fmax(a, b);
    return m + log(exp(a - m) + exp(b - m));
}

template <typename H>
__global__ void __launch_bounds__(256)
k_nuts_start(int n, const H *hbuf, long long bs, const double *gbuf, const uint8_t *cur, const double *minv,
             const double *ll, const double *lp, NutsBufs nb, uint64_t seed, const int64_t *step_base,
             int step_off)
{
    const int c = blockIdx.x;
    const uint32_t step = (uint32_t)(*step_base + step_off);
    const long long a = (long long)cur[c] * bs + (long long)c * n;
    double kin = 0.0;
    for (int j = threadIdx.x; 2 * j < n; j += blockDim.x) {
        const uint4 w = draw4(seed, STREAM_NUTS_P, (uint32_t)c, step, (uint32_t)j);
        const double u1 = u01_f64(w.x, w.y), u2 = u01_f64(w.z, w.w);
        const double rad = sqrt(-2.0 * log(u1));
        double sn, cn;
        sincospi(2.0 * u2, &sn, &cn);
        const double xi[2] = {rad * cn, rad * sn};
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int i = 2 * j + t;
            if (i >= n) break;
            const size_t k = (size_t)c * n + i;
            kin += 0.5 * xi[t] * xi[t];  // K(p0) with p0 = xi / sqrt(m)
            const double p0 = minv ? xi[t] / sqrt(minv[k]) : xi[t];
            const double q = (double)hbuf[a + i], g = gbuf[a + i];
            nb.qL[k] = q;
            nb.qR[k] = q;
            nb.pL[k] = p0;
            nb.pR[k] = p0;
            nb.gL[k] = g;
            nb.gR[k] = g;
            reinterpret_cast<H *>(nb.hsel)[k] = hbuf[a + i];
            nb.gsel[k] = g;
        }
    }
    kin = block_sum(kin);
    if (threadIdx.x == 0) {
        double *sc = nb.sc + kNS * c;
        const double H0 = -(ll[c] + lp[c]) + kin;
        sc[NS_H0] = H0;
        sc[NS_W] = -H0;
        sc[NS_WSUB] = -INFINITY;
        sc[NS_LLSEL] = ll[c];
        sc[NS_LPSEL] = lp[c];
        sc[NS_STAT] = 0.0;
        sc[NS_MOVED] = 0.0;
    }
}

// Half kick with the end's gradient and a drift, from the end on side v_j;
// the rounded position goes to the proposal slot (evaluated next).
template <typename H>
__global__ void __launch_bounds__(256)
k_nuts_drift(int n, H *hbuf, long long bs, const uint8_t *cur, double eps0, const double *eps_c,
             const double *minv, NutsBufs nb, uint64_t seed, const int64_t *step_base, int step_off, int j)
{
    const int c = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t step = (uint32_t)(*step_base + step_off);
    const int v = nuts_u(seed, c, step, (uint32_t)j) < 0.5 ? -1 : 1;
    const double e = (double)v * (eps_c ? eps_c[c] : eps0);
    const size_t k = (size_t)c * n + i;
    double *q64 = v > 0 ? nb.qR : nb.qL;
    const double *p = v > 0 ? nb.pR : nb.pL, *g = v > 0 ? nb.gR : nb.gL;
    const double p_half = p[k] + 0.5 * e * g[k];
    const double q = q64[k] + e * ((minv ? minv[k] : 1.0) * p_half);
    q64[k] = q;
    nb.ph[k] = p_half;
    hbuf[(long long)(1 - cur[c]) * bs + (long long)c * n + i] = (H)q;
}

// Second half kick with the new gradient (G[1 - cur]), the new state's
// energy and weight, the acceptance statistic and the subtree's sample.
template <typename H>
__global__ void __launch_bounds__(256)
k_nuts_leaf(int n, const H *hbuf, long long bs, const double *gbuf, const uint8_t *cur, double eps0,
            const double *eps_c, const double *minv, const double *llp, const double *lpp, NutsBufs nb,
            uint64_t seed, const int64_t *step_base, int step_off, int j, int leaf)
{
    __shared__ int take_s;
    const int c = blockIdx.x;
    const uint32_t step = (uint32_t)(*step_base + step_off);
    const int v = nuts_u(seed, c, step, (uint32_t)j) < 0.5 ? -1 : 1;
    const double e = (double)v * (eps_c ? eps_c[c] : eps0);
    const long long b = (long long)(1 - cur[c]) * bs + (long long)c * n;
    double *p_end = v > 0 ? nb.pR : nb.pL, *g_end = v > 0 ? nb.gR : nb.gL;
    double kin = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const size_t k = (size_t)c * n + i;
        const double g = gbuf[b + i];
        const double p = nb.ph[k] + 0.5 * e * g;
        p_end[k] = p;
        g_end[k] = g;
        kin += 0.5 * (minv ? minv[k] : 1.0) * p * p;
    }
    kin = block_sum(kin);
    if (threadIdx.x == 0) {
        double *sc = nb.sc + kNS * c;
        const double Hn = -(llp[c] + lpp[c]) + kin;
        const bool fin = isfinite(Hn);
        const double w = fin ? -Hn : -INFINITY;
        if (fin) sc[NS_STAT] += fmin(1.0, exp(sc[NS_H0] - Hn));
        const double Wn = logaddexp_d(sc[NS_WSUB], w);
        const double lu = log(nuts_u(seed, c, step, 64u + (uint32_t)leaf));
        const int take = fin && lu < w - Wn;
        sc[NS_WSUB] = Wn;
        if (take) {
            sc[NS_LLSUB] = llp[c];
            sc[NS_LPSUB] = lpp[c];
        }
        take_s = take;
    }
    __syncthreads();
    if (take_s) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            const size_t k = (size_t)c * n + i;
            reinterpret_cast<H *>(nb.hsub)[k] = hbuf[b + i];
            nb.gsub[k] = gbuf[b + i];
        }
    }
}

// The subtree's sample replaces the trajectory's (biased progressive
// sampling); W is updated by k_nuts_merge_w after every block has read it.
template <typename H>
__global__ void __launch_bounds__(256)
k_nuts_merge(int n, NutsBufs nb, uint64_t seed, const int64_t *step_base, int step_off, int j)
{
    const int c = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t step = (uint32_t)(*step_base + step_off);
    double *sc = nb.sc + kNS * c;
    const double Ws = sc[NS_WSUB], W = sc[NS_W];
    const double lu = log(nuts_u(seed, c, step, 32u + (uint32_t)j));
    if (!(Ws > -INFINITY && lu < Ws - W)) return;
    if (i < n) {
        const size_t k = (size_t)c * n + i;
        reinterpret_cast<H *>(nb.hsel)[k] = reinterpret_cast<const H *>(nb.hsub)[k];
        nb.gsel[k] = nb.gsub[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc[NS_LLSEL] = sc[NS_LLSUB];
        sc[NS_LPSEL] = sc[NS_LPSUB];
        sc[NS_MOVED] = 1.0;
    }
}

__global__ void k_nuts_merge_w(int n_chains, double *scs)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chains) return;
    double *sc = scs + kNS * c;
    sc[NS_W] = logaddexp_d(sc[NS_W], sc[NS_WSUB]);
    sc[NS_WSUB] = -INFINITY;
}

// The chain moves to the trajectory's sample (heights, gradient,
// log-likelihood and log-prior); the step's record: proposal = that sample,
// accepted = whether it moved, and the acceptance statistic for adaptation.
template <typename H>
__global__ void __launch_bounds__(256)
k_nuts_finish(int n, H *hbuf, long long bs, double *gbuf, const uint8_t *cur, uint8_t *prop_sel, double *ll,
              double *lp, double *llp, double *lpp, int64_t *accepts, int32_t *acc_last, double *logu,
              double *alpha, NutsBufs nb, int n_leaves)
{
    const int c = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const long long a = (long long)cur[c] * bs + (long long)c * n;
    if (i < n) {
        const size_t k = (size_t)c * n + i;
        hbuf[a + i] = reinterpret_cast<const H *>(nb.hsel)[k];
        gbuf[a + i] = nb.gsel[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double *sc = nb.sc + kNS * c;
        const int moved = sc[NS_MOVED] != 0.0;
        ll[c] = sc[NS_LLSEL];
        lp[c] = sc[NS_LPSEL];
        llp[c] = sc[NS_LLSEL];
        lpp[c] = sc[NS_LPSEL];
        accepts[c] += moved;
        acc_last[c] = moved;
        logu[c] = 0.0;
        prop_sel[c] = cur[c];
        if (alpha) alpha[c] = sc[NS_STAT] / (double)n_leaves;
    }
}

cudaError_t launch_nuts_start(const Prob &pb, int mode, const void *hbuf, long long bs, const double *gbuf,
                              const uint8_t *cur, int n_chains, const double *minv, const double *ll,
                              const double *lp, const NutsBufs &nb, uint64_t seed, const int64_t *step_base,
                              int step_off, cudaStream_t st)
{
    const int n = pb.L * pb.N;
    if (mode == MODE_F64)
        k_nuts_start<double><<<n_chains, 256, 0, st>>>(n, (const double *)hbuf, bs, gbuf, cur, minv, ll, lp, nb,
                                                       seed, step_base, step_off);
    else
        k_nuts_start<float><<<n_chains, 256, 0, st>>>(n, (const float *)hbuf, bs, gbuf, cur, minv, ll, lp, nb,
                                                      seed, step_base, step_off);
    return cudaGetLastError();
}

cudaError_t launch_nuts_drift(const Prob &pb, int mode, void *hbuf, long long bs, const uint8_t *cur,
                              int n_chains, double eps, const double *eps_c, const double *minv,
                              const NutsBufs &nb, uint64_t seed, const int64_t *step_base, int step_off, int j,
                              cudaStream_t st)
{
    const int n = pb.L * pb.N;
    dim3 grid((n + 255) / 256, n_chains);
    if (mode == MODE_F64)
        k_nuts_drift<double><<<grid, 256, 0, st>>>(n, (double *)hbuf, bs, cur, eps, eps_c, minv, nb, seed,
                                                   step_base, step_off, j);
    else
        k_nuts_drift<float><<<grid, 256, 0, st>>>(n, (float *)hbuf, bs, cur, eps, eps_c, minv, nb, seed,
                                                  step_base, step_off, j);
    return cudaGetLastError();
}

cudaError_t launch_nuts_leaf(const Prob &pb, int mode, const void *hbuf, long long bs, const double *gbuf,
                             const uint8_t *cur, int n_chains, double eps, const double *eps_c,
                             const double *minv, const double *llp, const double *lpp, const NutsBufs &nb,
                             uint64_t seed, const int64_t *step_base, int step_off, int j, int leaf,
                             cudaStream_t st)
{
    const int n = pb.L * pb.N;
    if (mode == MODE_F64)
        k_nuts_leaf<double><<<n_chains, 256, 0, st>>>(n, (const double *)hbuf, bs, gbuf, cur, eps, eps_c, minv,
                                                      llp, lpp, nb, seed, step_base, step_off, j, leaf);
    else
        k_nuts_leaf<float><<<n_chains, 256, 0, st>>>(n, (const float *)hbuf, bs, gbuf, cur, eps, eps_c, minv,
                                                     llp, lpp, nb, seed, step_base, step_off, j, leaf);
    return cudaGetLastError();
}

cudaError_t launch_nuts_merge(const Prob &pb, int mode, int n_chains, const NutsBufs &nb, uint64_t seed,
                              const int64_t *step_base, int step_off, int j, cudaStream_t st)
{
    const int n = pb.L * pb.N;
    dim3 grid((n + 255) / 256, n_chains);
    if (mode == MODE_F64) k_nuts_merge<double><<<grid, 256, 0, st>>>(n, nb, seed, step_base, step_off, j);
    else k_nuts_merge<float><<<grid, 256, 0, st>>>(n, nb, seed, step_base, step_off, j);
    k_nuts_merge_w<<<(n_chains + 127) / 128, 128, 0, st>>>(n_chains, nb.sc);
    return cudaGetLastError();
}

cudaError_t launch_nuts_finish(const Prob &pb, int mode, void *hbuf, long long bs, double *gbuf,
                               const uint8_t *cur, uint8_t *prop_sel, int n_chains, double *ll, double *lp,
                               double *llp, double *lpp, int64_t *accepts, int32_t *acc_last, double *logu,
                               double *alpha, const NutsBufs &nb, int n_leaves, cudaStream_t st)
{
    const int n = pb.L * pb.N;
    dim3 grid((n + 255) / 256, n_chains);
    if (mode == MODE_F64)
        k_nuts_finish<double><<<grid, 256, 0, st>>>(n, (double *)hbuf, bs, gbuf, cur, prop_sel, ll, lp, llp, lpp,
                                                    accepts, acc_last, logu, alpha, nb, n_leaves);
    else
        k_nuts_finish<float><<<grid, 256, 0, st>>>(n, (float *)hbuf, bs, gbuf, cur, prop_sel, ll, lp, llp, lpp,
                                                   accepts, acc_last, logu, alpha, nb, n_leaves);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- reduce
// ll[c] = sum over data of the Poisson constants + the CTA partials of chain c
// added in CTA order (deterministic).
__device__ __forceinline__ double chain_loglik(int mode, const void *partial, int n_blk, int c,
                                               double sumK)
{
    if (mode == MODE_F32C) {
        const float2 *p = reinterpret_cast<const float2 *>(partial) + (size_t)c * n_blk;
        FF s = {0.f, 0.f};
        for (int b = 0; b < n_blk; ++b) s = ff_add(s, FF{p[b].x, p[b].y});
        return sumK + ((double)s.hi + (double)s.lo);
    }
    const double *p = reinterpret_cast<const double *>(partial) + (size_t)c * n_blk;
    double s = 0.0;
    for (int b = 0; b < n_blk; ++b) s += p[b];
    return sumK + s;
}

__global__ void k_reduce_ll(int mode, int n_chains, int n_blk, const void *partial, double sumK,
                            double *ll_out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n_chains) ll_out[c] = chain_loglik(mode, partial, n_blk, c, sumK);
}

cudaError_t launch_reduce_ll(const Prob &pb, int mode, int n_chains, const void *partial,
                             double *ll_out, cudaStream_t st)
{
    const int n_blk = (pb.n_rays + march_rays_per_block(pb) - 1) / march_rays_per_block(pb);
    k_reduce_ll<<<(n_chains + 127) / 128, 128, 0, st>>>(mode, n_chains, n_blk, partial, pb.sumK,
                                                        ll_out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- accept
__global__ void k_accept(int n_chains, int mode, const void *partial, int n_blk, double sumK,
                         const double *lp_prop, const double *extra, double *ll, double *lp,
                         double *ll_prop_out, uint8_t *cur, uint8_t *prop_sel, int64_t *accepts,
                         int32_t *acc_last, double *logu_out, uint64_t seed,
                         const int64_t *step_base, int step_off, double *alpha_out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chains) return;
    const double lln = chain_loglik(mode, partial, n_blk, c, sumK);
    const double lpn = lp_prop[c];
    const uint32_t step = (uint32_t)(*step_base + step_off);
    const uint4 w = draw4(seed, STREAM_ACC, (uint32_t)c, step, 0u);
    const double logu = log(u01_f64(w.x, w.y));
    double delta = (lln + lpn) - (ll[c] + lp[c]);
    if (extra) delta += extra[c];
    const int acc = (lpn > -INFINITY) && (logu < delta);
    // acceptance probability min(1, e^delta) of the proposal (0 where it is
    // outside the prior's support or delta is not a number)
    if (alpha_out) alpha_out[c] = (lpn > -INFINITY && delta == delta) ? (delta >= 0.0 ? 1.0 : exp(delta)) : 0.0;
    const uint8_t cs = cur[c];
    prop_sel[c] = (uint8_t)(1 - cs);
    if (acc) {
        cur[c] = (uint8_t)(1 - cs);
        ll[c] = lln;
        lp[c] = lpn;
        accepts[c] += 1;
    }
    acc_last[c] = acc;
    ll_prop_out[c] = lln;
    logu_out[c] = logu;
}

cudaError_t launch_accept_fused(const Prob &pb, int mode, int n_chains, const void *partial,
                                const double *lp_prop, const double *extra, double *ll,
                                double *lp, double *ll_prop_out, uint8_t *cur, uint8_t *prop_sel,
                                int64_t *accepts, int32_t *acc_last, double *logu_out,
                                uint64_t seed, const int64_t *step_base, int step_off,
                                cudaStream_t st, double *alpha_out)
{
    const int n_blk = (pb.n_rays + march_rays_per_block(pb) - 1) / march_rays_per_block(pb);
    k_accept<<<(n_chains + 127) / 128, 128, 0, st>>>(n_chains, mode, partial, n_blk, pb.sumK,
                                                     lp_prop, extra, ll, lp, ll_prop_out, cur,
                                                     prop_sel, accepts, acc_last, logu_out, seed,
                                                     step_base, step_off, alpha_out);
    return cudaGetLastError();
}

__global__ void k_advance(int64_t *step, int n)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *step += n;
}

cudaError_t launch_advance(int64_t *step, int n, cudaStream_t st)
{
    k_advance<<<1, 32, 0, st>>>(step, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- warm-up adaptation
// Per-chain dual averaging of log eps toward a target acceptance probability
// delta (Sec. 3.1: the step size is tuned in the warm-up toward 0.8; the
// scheme is Hoffman & Gelman's, J. Mach. Learn. Res. 15 (2014), Sec. 3.2.1,
// with gamma = 0.05, t0 = 10, kappa = 0.75 and mu = log(10 eps0)).  After the
// m-th dual-averaging step with acceptance probability alpha_m:
//   Hbar_m = (1 - 1/(m + t0)) Hbar_{m-1} + (delta - alpha_m) / (m + t0)
//   log eps_m = mu - sqrt(m) / gamma * Hbar_m
//   log epsbar_m = m^-kappa log eps_m + (1 - m^-kappa) log epsbar_{m-1}
// (Hbar_0 = 0, log epsbar_0 = 0); the next step runs with eps_m, and after
// the last of the W adapted steps every chain keeps epsbar.
//
// With the metric adapted too (HMC; Sec. 3.1: the warm-up also tunes a
// diagonal preconditioner), the adapted steps t = 0 .. W-1 are split into an
// initial buffer, slow windows of doubling length and a terminal buffer
// (75 / 25 / 50 steps, or 15 % / 75 % / 10 % of W when those do not fit; the
// last slow window is stretched to the terminal buffer when the next one
// would cross it).  In a slow window every chain accumulates the mean and M2
// of each coordinate of its post-step state (Welford); at the window's last
// step its inverse metric becomes (n/(n+5)) var + s 5/(n+5) (var = M2/(n-1),
// n the window length, s the shrinkage target), the accumulators restart and
// the dual averaging restarts from mu = log(10 eps), Hbar = 0,
// log epsbar = 0, m = 0.
//
// State per chain: da[6c .. 6c+5] = {log epsbar, Hbar, mu, m, t, unused}
// (kDAStride = 6).

// Slow window of adapted step t (of W): returns whether t lies in one, with
// the window's first step and whether t is its last.
__host__ __device__ inline bool slow_window(int W, int t, int &start, bool &last)
{
    int init = 75, term = 50, base = 25;
    if (init + base + term > W) {
        init = (int)(0.15 * W);
        term = (int)(0.1 * W);
        base = W - (init + term);
    }
    const int stop = W - term;
    if (t < init || t >= stop || base < 1) return false;
    int s0 = init, size = base;
    while (s0 < stop) {
        int end = s0 + size;
        if (end + 2 * size > stop) end = stop;
        if (t < end) {
            start = s0;
            last = t == end - 1;
            return true;
        }
        s0 = end;
        size *= 2;
    }
    return false;
}

__global__ void k_adapt_init(int n_chains, double eps0, double *da, double *eps)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chains) return;
    eps[c] = eps0;
    double *d = da + kDAStride * c;
    d[0] = 0.0;
    d[1] = 0.0;
    d[2] = log(10.0 * eps0);
    d[3] = 0.0;
    d[4] = 0.0;
    d[5] = 0.0;
}

__global__ void k_adapt(int n_chains, double target, int n_adapt, int metric, const double *alpha,
                        double *da, double *eps)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_chains) return;
    double *d = da + kDAStride * c;
    const int t = (int)d[4];
    if (t >= n_adapt) return;  // adaptation over: eps stays at epsbar
    const double m = d[3] + 1.0;
    const double t0 = 10.0, gamma = 0.05, kappa = 0.75;
    const double w = 1.0 / (m + t0);
    const double hbar = (1.0 - w) * d[1] + w * (target - alpha[c]);
    const double log_eps = d[2] - sqrt(m) / gamma * hbar;
    const double eta = pow(m, -kappa);
    const double log_bar = eta * log_eps + (1.0 - eta) * d[0];
    const double e = exp(t + 1 < n_adapt ? log_eps : log_bar);
    eps[c] = e;
    int s0;
    bool last = false;
    if (metric && slow_window(n_adapt, t, s0, last) && last) {
        d[0] = 0.0;  // the metric changed: dual averaging starts over from eps
        d[1] = 0.0;
        d[2] = log(10.0 * e);
        d[3] = 0.0;
    } else {
        d[0] = log_bar;
        d[1] = hbar;
        d[3] = m;
    }
    d[4] = (double)(t + 1);
}

// Welford accumulation of the chains' post-step states during slow windows
// and the inverse metric at each window's end; grid (coordinate blocks,
// chains).  Reads the step index t before k_adapt advances it.
template <typename H>
__global__ void __launch_bounds__(256)
k_metric(int n, const H *hbuf, long long bs, const uint8_t *cur, int n_adapt, double shrink,
         const double *da, double *mean, double *m2, double *minv)
{
    const int c = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int t = (int)da[kDAStride * c + 4];
    int s0;
    bool last = false;
    if (t >= n_adapt || !slow_window(n_adapt, t, s0, last)) return;
    const size_t k = (size_t)c * n + i;
    const double x = (double)hbuf[(long long)cur[c] * bs + (long long)c * n + i];
    const double cnt = (double)(t - s0 + 1);
    const double dx = x - mean[k];
    const double mu = mean[k] + dx / cnt;
    const double q = m2[k] + dx * (x - mu);
    if (last) {
        const double var = cnt > 1.0 ? q / (cnt - 1.0) : 0.0;
        minv[k] = (cnt / (cnt + 5.0)) * var + shrink * (5.0 / (cnt + 5.0));
        mean[k] = 0.0;
        m2[k] = 0.0;
    } else {
        mean[k] = mu;
        m2[k] = q;
    }
}

__global__ void k_metric_init(size_t n, double *mean, double *m2, double *minv)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        mean[i] = 0.0;
        m2[i] = 0.0;
        minv[i] = 1.0;
    }
}

cudaError_t launch_adapt_init(int n_chains, double eps0, double *da, double *eps, cudaStream_t st)
{
    k_adapt_init<<<(n_chains + 127) / 128, 128, 0, st>>>(n_chains, eps0, da, eps);
    return cudaGetLastError();
}

cudaError_t launch_adapt(int n_chains, double target, int n_adapt, int metric, const double *alpha,
                         double *da, double *eps, cudaStream_t st)
{
    k_adapt<<<(n_chains + 127) / 128, 128, 0, st>>>(n_chains, target, n_adapt, metric, alpha, da, eps);
    return cudaGetLastError();
}

cudaError_t launch_metric_init(size_t n, double *mean, double *m2, double *minv, cudaStream_t st)
{
    k_metric_init<<<1024, 256, 0, st>>>(n, mean, m2, minv);
    return cudaGetLastError();
}

cudaError_t launch_metric(const Prob &pb, int mode, const void *hbuf, long long buf_stride,
                          const uint8_t *cur, int n_chains, int n_adapt, double shrink,
                          const double *da, double *mean, double *m2, double *minv, cudaStream_t st)
{
    const int n = pb.L * pb.N;
    dim3 grid((n + 255) / 256, n_chains);
    if (mode == MODE_F64)
        k_metric<double><<<grid, 256, 0, st>>>(n, (const double *)hbuf, buf_stride, cur, n_adapt, shrink, da,
                                               mean, m2, minv);
    else
        k_metric<float><<<grid, 256, 0, st>>>(n, (const float *)hbuf, buf_stride, cur, n_adapt, shrink, da,
                                              mean, m2, minv);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- gather
template <typename H>
__global__ void k_gather(HRef h, long long n_per_chain, H *out)
{
    const int c = blockIdx.y;
    const H *src = chain_ptr<H>(h, c);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_per_chain;
         i += (long long)gridDim.x * blockDim.x)
        out[(long long)c * n_per_chain + i] = src[i];
}

cudaError_t launch_gather(int mode, HRef h, int n_chains, long long n_per_chain, void *out,
                          cudaStream_t st)
{
    dim3 grid((unsigned)((n_per_chain + 255) / 256 < 64 ? (n_per_chain + 255) / 256 : 64), n_chains);
    if (mode == MODE_F64) k_gather<double><<<grid, 256, 0, st>>>(h, n_per_chain, (double *)out);
    else k_gather<float><<<grid, 256, 0, st>>>(h, n_per_chain, (float *)out);
    return cudaGetLastError();
}

}  // namespace mt
