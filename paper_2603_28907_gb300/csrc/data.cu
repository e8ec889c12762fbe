// data.cu -- once-per-problem kernels: ray table, count constants and the
// synthetic observed counts.
#include <math.h>

#include "march.cuh"
#include "philox.cuh"

namespace mt {

// ---------------------------------------------------------------- ray table
// Ray (s, p) starts at sensor s and runs along pixel direction p (Sec. 2.1.1);
// only its part inside the box counts, t in [0, t_exit] with t_exit the
// nearest slab exit.  Samples sit at t_k = (k + 1/2) dt, dt = t_exit / G.
// Positions are stored as sample-0 point plus per-sample step, with x, y in
// cell units (x * (Q-1) / Lx, y * (R-1) / Ly).  The FP32 copy shifts x, y by
// -1/2 (centred cell split) and keeps z per surface, relative to the surface's
// reference height and scaled by kg = log2(e)/gamma.

// Make fmaf(k, s, o) lie in [lo, hi] for k = 0 .. G-1.  fmaf is monotone in
// k (the exact k*s + o is, and rounding preserves order), so the two ends
// decide.  The moves are a few ulps; returns false if they did not suffice.
__device__ bool fit_axis(float &o, float &s, int G, float lo, float hi)
{
    o = fminf(fmaxf(o, lo), hi);
    const float kl = (float)(G - 1);
    for (int it = 0; it < 64; ++it) {
        const float v1 = fmaf(kl, s, o);
        if (v1 >= lo && v1 <= hi) return true;
        if (it == 0 && G > 1) {
            const double target = v1 < lo ? (double)lo : (double)hi;
            s = __double2float_rz((target - (double)o) / (double)(G - 1));
        } else {
            s = nextafterf(s, 0.0f);
        }
    }
    return false;
}

__global__ void k_raytab(Prob pb, const double *sensors, const double *dirs, float4 *o4, float4 *s4,
                         float *kz0, double *o_d, double *s_d, double *dt_out, float2 *dt_ff,
                         int *flag)
{
    const int ray = blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= pb.n_rays) return;
    const int s = ray / pb.P, p = ray - s * pb.P;
    const double o[3] = {sensors[3 * s], sensors[3 * s + 1], sensors[3 * s + 2]};
    const double d[3] = {dirs[3 * p], dirs[3 * p + 1], dirs[3 * p + 2]};
    double te = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double ta = INFINITY;
        if (d[a] > 0.0) ta = (pb.box[a] - o[a]) / d[a];
        else if (d[a] < 0.0) ta = (0.0 - o[a]) / d[a];
        te = fmin(te, ta);
    }
    const double dt = te / (double)pb.G;
    const double sx = (double)(pb.Q - 1) / pb.box[0], sy = (double)(pb.R - 1) / pb.box[1];
    const double gx0 = (o[0] + 0.5 * dt * d[0]) * sx, gsx = dt * d[0] * sx;
    const double gy0 = (o[1] + 0.5 * dt * d[1]) * sy, gsy = dt * d[1] * sy;
    const double z0 = o[2] + 0.5 * dt * d[2], sz = dt * d[2];
    o_d[3 * ray] = gx0;
    o_d[3 * ray + 1] = gy0;
    o_d[3 * ray + 2] = z0;
    s_d[3 * ray] = gsx;
    s_d[3 * ray + 1] = gsy;
    s_d[3 * ray + 2] = sz;
    const double kg = (double)pb.kg;
    float ox = (float)(gx0 - 0.5), fsx = (float)gsx;
    float oy = (float)(gy0 - 0.5), fsy = (float)gsy;
    const bool ok = fit_axis(ox, fsx, pb.G, -0.5f, pb.gm_hi_x) & fit_axis(oy, fsy, pb.G, -0.5f, pb.gm_hi_y);
    if (!ok) {  // cannot happen for rays that start inside the box; keep the samples in range
        fsx = 0.f;
        fsy = 0.f;
        atomicOr(flag, 2);
    }
    // z in float-float, scaled by the FP32 kg the kernel multiplies heights by
    const double ksz = kg * sz;
    const float ksz_hi = (float)ksz;
    o4[ray] = make_float4(ox, oy, 0.f, 0.f);
    s4[ray] = make_float4(fsx, fsy, ksz_hi, (float)(ksz - (double)ksz_hi));
    for (int l = 0; l < pb.L; ++l) {
        const double kz = kg * (z0 - (double)pb.ref[l]);
        const float hi = (float)kz;
        kz0[(size_t)l * pb.n_rays + ray] = hi;
        kz0[(size_t)(pb.L + l) * pb.n_rays + ray] = (float)(kz - (double)hi);
    }
    dt_out[ray] = dt;
    const float hi = (float)dt;
    dt_ff[ray] = make_float2(hi, (float)(dt - (double)hi));
}

cudaError_t launch_raytab(const Prob &pb, const double *d_sensors, const double *d_dirs,
                          float4 *o4, float4 *s4, float *kz0, double *o_d, double *s_d, double *dt,
                          float2 *dt_ff, int *flag, cudaStream_t st)
{
    k_raytab<<<(pb.n_rays + 255) / 256, 256, 0, st>>>(pb, d_sensors, d_dirs, o4, s4, kz0, o_d, s_d,
                                                      dt, dt_ff, flag);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- FP32 march ray table
// The FP32 march forms sample k's cell coordinate as
//   g = fmaf(k, sh, fmaf(k, sl, o))   (relative to the ray's start cell c0)
// with o = gx0 - 1/2 - c0 in [-1/2, 1/2] and the step split sh + sl, so the
// position carries no per-ray FP32 offset (the sample-0 point and the step
// are exact to ~2^-48) and only the final rounding, which differs from
// sample to sample.  Its cell is c0 + round(g).  g is monotone in k, so the
// cells of the first and last sample decide whether all lie in [0, n - 2];
// where rounding at a face of the box would leave that range, o and sh move
// inward by a few ulps (this does not happen for rays that start inside the
// box away from a face).
// Cell of sample kf as the march computes it: the coordinate rounded to the
// nearest integer (x: coordinates relative to the cell's centre) or down
// (FLOOR, y: relative to the cell's lower edge), from the bits of
// g + 1.5 * 2^23.
__device__ __forceinline__ int rel_cell(float o, float sl, float sh, float kf, bool floor_axis)
{
    const float g = fmaf(kf, sh, fmaf(kf, sl, o));
    const float t = floor_axis ? __fadd_rd(g, 12582912.0f) : g + 12582912.0f;
    return __float_as_int(t) - 0x4B400000;
}

__device__ bool fit_axis_rel(float &o, float &sh, float sl, int c0, int n, int G, bool floor_axis)
{
    const float kl = (float)(G - 1);
    for (int it = 0; it < 64; ++it) {
        const int a = c0 + rel_cell(o, sl, sh, 0.0f, floor_axis), b = c0 + rel_cell(o, sl, sh, kl, floor_axis);
        const bool oka = a >= 0 && a <= n - 2, okb = b >= 0 && b <= n - 2;
        if (oka && okb) return true;
        if (!oka) o = nextafterf(o, a < 0 ? INFINITY : -INFINITY);
        if (!okb) sh = nextafterf(sh, b < 0 ? INFINITY : -INFINITY);
    }
    return false;
}

// z per surface in log2 units, kg64 (z - ref_l), split into a high part on
// the grid pb.zgrid and an FP32 remainder; likewise the per-sample step.
// Every sample's |kg64 (z - ref_l)| lies below half the bound the grid was
// chosen for, so hi + k * step_hi is exact in FP32 for all k < G.  (These
// place the exact-saturation windows and serve the adjoint.)  The march's
// own arithmetic takes z - ref_l in metres, its high part on the grid
// pb.zgrid_m (exact in the same way) and kg64 times the remainder (kzm, szm).
__global__ void k_raytab_march(Prob pb, const double *sensors, const double *dirs, float4 *xa4, float4 *xb4,
                               int2 *xc2, float *kz1, float *kzm, float2 *szm, int *flag)
{
    const int ray = blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= pb.n_rays) return;
    const int s = ray / pb.P, p = ray - s * pb.P;
    const double o[3] = {sensors[3 * s], sensors[3 * s + 1], sensors[3 * s + 2]};
    const double d[3] = {dirs[3 * p], dirs[3 * p + 1], dirs[3 * p + 2]};
    double te = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double ta = INFINITY;
        if (d[a] > 0.0) ta = (pb.box[a] - o[a]) / d[a];
        else if (d[a] < 0.0) ta = (0.0 - o[a]) / d[a];
        te = fmin(te, ta);
    }
    const double dt = te / (double)pb.G;
    const double sx = (double)(pb.Q - 1) / pb.box[0], sy = (double)(pb.R - 1) / pb.box[1];
    const double gx0 = (o[0] + 0.5 * dt * d[0]) * sx - 0.5, gsx = dt * d[0] * sx;
    const double gy0 = (o[1] + 0.5 * dt * d[1]) * sy, gsy = dt * d[1] * sy;  // y from the cell's lower edge
    const double z0 = o[2] + 0.5 * dt * d[2], sz = dt * d[2];
    const int c0x = min(max((int)rint(gx0), 0), pb.Q - 2), c0y = min(max((int)floor(gy0), 0), pb.R - 2);
    float ox = (float)(gx0 - (double)c0x), oy = (float)(gy0 - (double)c0y);
    float sxh = (float)gsx, syh = (float)gsy;
    const float sxl = (float)(gsx - (double)sxh), syl = (float)(gsy - (double)syh);
    const bool ok = fit_axis_rel(ox, sxh, sxl, c0x, pb.Q, pb.G, false) &
                    fit_axis_rel(oy, syh, syl, c0y, pb.R, pb.G, true);
    if (!ok) atomicOr(flag, 2);
    const double g = pb.zgrid;
    const double ksz = pb.kg64 * sz;
    const double szh = rint(ksz / g) * g;
    xa4[ray] = make_float4(ox, oy, sxh, syh);
    xb4[ray] = make_float4(ok ? sxl : 0.f, ok ? syl : 0.f, (float)szh, (float)(ksz - szh));
    if (!ok) xa4[ray] = make_float4(0.f, 0.f, 0.f, 0.f);  // keeps every sample in the start cell
    xc2[ray] = make_int2(c0x, c0y);
    const double gm = pb.zgrid_m;
    const double szh_m = rint(sz / gm) * gm;
    szm[ray] = make_float2((float)szh_m, (float)(pb.kg64 * (sz - szh_m)));
    for (int l = 0; l < pb.L; ++l) {
        const double kz = pb.kg64 * (z0 - (double)pb.ref[l]);
        const double hi = rint(kz / g) * g;
        kz1[(size_t)l * pb.n_rays + ray] = (float)hi;
        kz1[(size_t)(pb.L + l) * pb.n_rays + ray] = (float)(kz - hi);
        const double zm = z0 - (double)pb.ref[l];
        const double hm = rint(zm / gm) * gm;
        kzm[(size_t)l * pb.n_rays + ray] = (float)hm;
        kzm[(size_t)(pb.L + l) * pb.n_rays + ray] = (float)(pb.kg64 * (zm - hm));
    }
}

cudaError_t launch_raytab_march(const Prob &pb, const double *d_sensors, const double *d_dirs, float4 *xa4,
                                float4 *xb4, int2 *xc2, float *kz1, float *kzm, float2 *szm, int *flag,
                                cudaStream_t st)
{
    k_raytab_march<<<(pb.n_rays + 255) / 256, 256, 0, st>>>(pb, d_sensors, d_dirs, xa4, xb4, xc2, kz1, kzm, szm,
                                                            flag);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- logistic calibration
// The FP32 march forms psi = 1 / (1 + 2^a), a = |argument| >= 0, as
// rcp.approx((ex2.approx(a) + 1) c) with c = 2^-28.  Each approximation is
// within a few ulps, but their errors have a nonzero mean (on GB300:
// ex2.approx ~ +3.6e-8 relative, rcp.approx ~ +4e-9), and a transition that
// the box cuts on one side (a surface within a few gamma of the box top, a
// ray leaving through a wall) adds one side's psi values only, so that mean
// survives: with ~1e5 such rays a far-off chain's log-likelihood would move
// by ~1e-3.  This kernel measures the mean on the device the march runs on:
// over a in [0, 16) (2^16 points; beyond, psi < 2^-16 carries no weight) the
// relative error r(a) of the march's own instruction sequence against FP64,
// weighted by psi (a one-sided transition's sum of psi errors), and returns
// kappa = -sum psi r / sum psi (1 - psi): the march then uses
// (2^a (1 - kappa) + 1) c, whose psi moves by +kappa (1 - psi) relative
// (d psi / psi = -(1 - psi) d(2^a) / 2^a), which to first order cancels the
// psi-weighted mean error.  One block, fixed summation order: the same kappa
// on every call.
__global__ void __launch_bounds__(1024) k_psi_calib(double *out)
{
    const int n = 1 << 16;
    const float c = __uint_as_float(0x31800000u);  // 2^-28
    double num = 0.0, den = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float a = (float)(16.0 * ((double)i + 0.5) / (double)n);
        const float q = rcp_approx(fmaf(ex2_approx(a), c, c));  // psi 2^28, as in the march
        const double E = exp2((double)a);
        const double psi = 1.0 / (1.0 + E);
        const double r = (double)q * 0x1p-28 / psi - 1.0;
        num += psi * r;
        den += psi * (1.0 - psi);
    }
    num = block_sum(num);
    __syncthreads();
    den = block_sum(den);
    if (threadIdx.x == 0) out[0] = -num / den;
}

cudaError_t launch_psi_calib(double *out, cudaStream_t st)
{
    k_psi_calib<<<1, 1024, 0, st>>>(out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- counts
// a = ln(I0 / C) per ray (the centred Poisson term's offset), and the data
// constant sum_p (C ln C - C - ln C!) reduced in a fixed order by one block.
__global__ void k_counts_prep(Prob pb, double *a, float2 *a_ff)
{
    const int ray = blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= pb.n_rays) return;
    const int C = pb.cnt[ray];
    const double v = C > 0 ? log(pb.I0 / (double)C) : 0.0;
    a[ray] = v;
    const float hi = (float)v;
    a_ff[ray] = make_float2(hi, (float)(v - (double)hi));
}

__global__ void __launch_bounds__(1024) k_sumK(Prob pb, double *out)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < pb.n_rays; i += blockDim.x) s += poisson_K(pb.cnt[i]);
    s = block_sum(s);
    if (threadIdx.x == 0) *out = s;
}

cudaError_t launch_counts_prep(const Prob &pb, double *a, float2 *a_ff, double *sumK,
                               cudaStream_t st)
{
    k_counts_prep<<<(pb.n_rays + 255) / 256, 256, 0, st>>>(pb, a, a_ff);
    k_sumK<<<1, 1024, 0, st>>>(pb, sumK);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- Poisson
// Knuth's multiplication method for lambda < 10 and Hormann's PTRS
// (transformed rejection with squeeze, 1993) for lambda >= 10, with uniforms
// from Philox stream DATA, counter {ray, attempt, 0}.  Every floating-point
// step is an explicitly rounded operation so no contraction changes a draw.
// Attempts are bounded; running out latches *flag.
__device__ int32_t poisson_draw(double lam, uint64_t seed, uint32_t ray, int *flag)
{
    const int max_attempts = 256;
    if (lam < 10.0) {
        const double limit = exp(-lam);
        double prod = 1.0;
        int32_t k = 0;
        for (int j = 0; j < max_attempts; ++j) {
            const uint4 w = draw4(seed, STREAM_DATA, 0u, (uint32_t)j, ray);
            prod = __dmul_rn(prod, u01_f64(w.x, w.y));
            if (prod <= limit) return k;
            k = k + 1;
            prod = __dmul_rn(prod, u01_f64(w.z, w.w));
            if (prod <= limit) return k;
            k = k + 1;
        }
        atomicOr(flag, 1);
        return k;
    }
    const double slam = sqrt(lam);
    const double loglam = log(lam);
    const double b = __dadd_rn(0.931, __dmul_rn(2.53, slam));
    const double a = __dadd_rn(-0.059, __dmul_rn(0.02483, b));
    const double inv_alpha = __dadd_rn(1.1239, __ddiv_rn(1.1328, __dsub_rn(b, 3.4)));
    const double v_r = __dsub_rn(0.9277, __ddiv_rn(3.6224, __dsub_rn(b, 2.0)));
    for (int j = 0; j < max_attempts; ++j) {
        const uint4 w = draw4(seed, STREAM_DATA, 0u, (uint32_t)j, ray);
        const double U = __dsub_rn(u01_f64(w.x, w.y), 0.5);
        const double V = u01_f64(w.z, w.w);
        const double us = __dsub_rn(0.5, fabs(U));
        const double kf = floor(__dadd_rn(
            __dadd_rn(__dmul_rn(__dadd_rn(__ddiv_rn(__dmul_rn(2.0, a), us), b), U), lam), 0.43));
        if (us >= 0.07 && V <= v_r) return (int32_t)kf;
        if (kf < 0.0 || (us < 0.013 && V > us)) continue;
        const double lhs = __dsub_rn(__dadd_rn(log(V), log(inv_alpha)),
                                     log(__dadd_rn(__ddiv_rn(a, __dmul_rn(us, us)), b)));
        const double rhs = __dsub_rn(__dadd_rn(-lam, __dmul_rn(kf, loglam)), lgamma(__dadd_rn(kf, 1.0)));
        if (lhs <= rhs) return (int32_t)kf;
    }
    atomicOr(flag, 1);
    return 0;
}

// lambda_p of the true geometry from the FP64 march, then the count.
template <int L, bool HARD>
__global__ void __launch_bounds__(128)
k_gen_counts(Prob pb, const double *nodes, uint64_t seed, int mode, int32_t *counts,
             double *lambda, int *flag)
{
    const int ray = blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= pb.n_rays) return;
    const double S_ = march_ray_f64<L, HARD>(pb, nodes, ray);
    const double O = pb.dt[ray] * ((double)pb.G * pb.rho_top + S_);
    const double lam = pb.I0 * exp(-O / pb.Lambda);
    lambda[ray] = lam;
    counts[ray] = mode == 1 ? (int32_t)rint(lam) : poisson_draw(lam, seed, (uint32_t)ray, flag);
}

// [L][N] heights -> node-major layout of march.cuh, in global memory.
template <int L> __global__ void k_to_nodes(double *dst, const double *src, int N)
{
    stage_nodes<double, double, L>(dst, src, N);
}

size_t nodes_bytes_f64(int L, int N)
{
    const int raw = L * 8;
    const int bytes = raw <= 8 ? 8 : ((raw + 15) / 16) * 16;
    return (size_t)bytes * N;
}

template <int L, bool HARD>
static void gen_l(const Prob &pb, double *nodes, const double *h, uint64_t seed, int mode,
                  int32_t *counts, double *lambda, int *flag, cudaStream_t st)
{
    k_to_nodes<L><<<1, 256, 0, st>>>(nodes, h, pb.N);
    k_gen_counts<L, HARD><<<(pb.n_rays + 127) / 128, 128, 0, st>>>(pb, nodes, seed, mode, counts,
                                                                    lambda, flag);
}

// h_layers: [L][N] FP64 device array; scratch for the node layout follows it,
// rounded up to an even double (the caller allocates (L*N + 1) * 8 +
// nodes_bytes_f64 bytes from a 256-byte aligned base).
cudaError_t launch_gen_counts(const Prob &pb, const double *h_layers, uint64_t seed, int mode,
                              int32_t *counts, double *lambda, int *flag, cudaStream_t st)
{
    // node records use 16-byte loads: start them on an even double
    double *nodes = const_cast<double *>(h_layers) + (((size_t)pb.L * pb.N + 1) & ~(size_t)1);
    const bool hard = pb.gamma == 0.0;
#define GEN_CASE(LL)                                                                         \
    case LL:                                                                                 \
        if (hard) gen_l<LL, true>(pb, nodes, h_layers, seed, mode, counts, lambda, flag, st); \
        else gen_l<LL, false>(pb, nodes, h_layers, seed, mode, counts, lambda, flag, st);     \
        break;
    switch (pb.L) {
        GEN_CASE(1) GEN_CASE(2) GEN_CASE(3) GEN_CASE(4)
        GEN_CASE(5) GEN_CASE(6) GEN_CASE(7) GEN_CASE(8)
        default: return cudaErrorInvalidValue;
    }
#undef GEN_CASE
    return cudaGetLastError();
}

}  // namespace mt
