// march.cuh -- fused ray march + Poisson log-likelihood (the hot path).
//
// One CTA = one chain x one block of rays.  The chain's surfaces are staged
// node-major in shared memory; each thread marches whole rays (consecutive
// lanes = consecutive pixels of one sensor, so a warp's rays stay close).
//
// Per sample k of a ray (Sec. 2.1.1 opacity integral as a midpoint sum; Eqs.
// smooth_layer_indicators / def_LM_density_grid_smooth):
//   position      g = g0 + k*gs  (x, y in cell units, z scaled by log2(e)/gamma)
//   cell          the bilinear cell holding (x, y); its four corners of every
//                 surface are cached in registers and reloaded only when the
//                 ray enters a new cell
//   indicator     varsigma(s_l - z) for each surface l
//   density       rho(x) = rho_top + sum_l (rho_l - rho_{l+1}) varsigma(s_l - z),
//                 which equals sum_u W_u rho_u because the normaliser sum_u D_u
//                 telescopes to exactly 1
// Per ray: O = dt * sum_k rho_k, y = ln(I0/C) - O/Lambda and the Poisson term
// C y - C expm1(y) (Eq. def_likelihood without the constant C ln C - C - ln C!,
// which is summed once per data set).  Terms are reduced per CTA in a fixed
// order (warp shuffles, then warps in order) into one partial per (chain, CTA).
#pragma once

#include <cuda_bf16.h>

#include "internal.h"

// Threads per CTA of the FP32 modes' march (one CTA per SM: the planes take
// the shared memory) and the unroll of its surface loop: 768 threads leave 80
// registers per thread, enough to unroll four surfaces without spilling.
#ifndef MT_DX_THREADS
#define MT_DX_THREADS 768
#endif
#ifndef MT_SURF_UNROLL
#define MT_SURF_UNROLL 4
#endif

namespace mt {
constexpr int kSurfUnroll = MT_SURF_UNROLL;

// ---------------------------------------------------------------- types
template <int MODE> struct Types;
template <> struct Types<MODE_F64> { using S = double; using T = double; using H = double; };
template <> struct Types<MODE_F32> { using S = float; using T = float; using H = float; };
template <> struct Types<MODE_F32C> { using S = float; using T = float; using H = float; };
template <> struct Types<MODE_F32A> { using S = float; using T = float; using H = float; };
template <> struct Types<MODE_BF16> { using S = __nv_bfloat16; using T = float; using H = float; };

// Node-major shared-memory layout: the L heights of one node, padded to a
// 4-, 8- or multiple-of-16-byte record so they load as vectors.
template <typename S, int L> struct NodeLayout {
    static constexpr int raw = L * (int)sizeof(S);
    static constexpr int bytes = raw <= 4 ? 4 : raw <= 8 ? 8 : ((raw + 15) / 16) * 16;
    static constexpr int LP = bytes / (int)sizeof(S);
};

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ double to_d(double v) { return v; }

template <typename S> __device__ __forceinline__ S from_h(float v);
template <> __device__ __forceinline__ float from_h<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_h<__nv_bfloat16>(float v)
{
    return __float2bfloat16_rn(v);
}
template <typename S> __device__ __forceinline__ S from_hd(double v) { return v; }

template <typename H> __device__ __forceinline__ const H *chain_ptr(const HRef &h, int c)
{
    long long off = (long long)c * h.chain_stride;
    if (h.sel) {
        int s = h.sel[c];
        if (h.sel_flip) s = 1 - s;
        off += (long long)s * h.sel_stride;
    }
    return reinterpret_cast<const H *>(h.base) + off;
}

// Copy one chain [L][N] from HBM into node-major shared memory.
// FP32 / BF16 storage keeps h - ref[l] (ref = nullptr: absolute heights).
template <typename S, typename H, int L>
__device__ __forceinline__ void stage_nodes(S *sh, const H *Hc, int N, const float *ref = nullptr)
{
    using NL = NodeLayout<S, L>;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        alignas(16) S tmp[NL::LP];
#pragma unroll
        for (int l = 0; l < NL::LP; ++l) tmp[l] = (S)0.0f;
#pragma unroll
        for (int l = 0; l < L; ++l) {
            if constexpr (sizeof(S) == 8) tmp[l] = Hc[(size_t)l * N + i];
            else tmp[l] = from_h<S>(ref ? (float)Hc[(size_t)l * N + i] - ref[l] : (float)Hc[(size_t)l * N + i]);
        }
        char *dst = reinterpret_cast<char *>(sh) + (size_t)i * NL::bytes;
        if constexpr (NL::bytes == 4) {
            *reinterpret_cast<uint32_t *>(dst) = *reinterpret_cast<const uint32_t *>(tmp);
        } else if constexpr (NL::bytes == 8) {
            *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<const uint2 *>(tmp);
        } else {
#pragma unroll
            for (int q = 0; q < NL::bytes / 16; ++q)
                reinterpret_cast<uint4 *>(dst)[q] = reinterpret_cast<const uint4 *>(tmp)[q];
        }
    }
}

// FP32 node records, one plane per surface: plane l holds for every node
// {hm, dx} with h = H - ref_l, dx = h(r, c+1) - h(r, c) (0 in the last
// column) and hm = h + dx / 2, the height halfway along the row segment: the
// x-lerp at the cell fraction f in [-1/2, 1/2] around the midpoint is then
// hm + f dx, one multiply-add, and a cell needs the 8-byte records of its
// two left corners only.  A chain's planes take 8 L N bytes, [l][node].
template <typename H>
__device__ __forceinline__ float2 dx_record(const H *Hc, int N, int Q, float ref, int l, int i)
{
    const float h = (float)Hc[(size_t)l * N + i] - ref;
    const float d = (i % Q) == Q - 1 ? 0.f : ((float)Hc[(size_t)l * N + i + 1] - ref) - h;
    return make_float2(fmaf(0.5f, d, h), d);
}

template <typename H, int L>
__device__ __forceinline__ void stage_planes_dx(float2 *sh, const H *Hc, int N, int Q, const float *ref)
{
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
#pragma unroll
        for (int l = 0; l < L; ++l) sh[(size_t)l * N + i] = dx_record<H>(Hc, N, Q, ref[l], l, i);
    }
}

// The same planes scaled to sigmoid-argument units (log2, kg64 = log2(e) /
// gamma = kgh + kgl), for the adjoint: {-kg64 hm, -kg64 dx}, so that the
// lerp of the records is -kg64 (s_l - ref_l) directly.  hm is formed exactly
// (float-float two-sum) and each product by kg64 is rounded once.
template <typename H>
__device__ __forceinline__ float2 dx_record_scaled(const H *Hc, int N, int Q, float ref, float kgh, float kgl,
                                                   int l, int i)
{
    const float h = (float)Hc[(size_t)l * N + i] - ref;
    const float d = (i % Q) == Q - 1 ? 0.f : ((float)Hc[(size_t)l * N + i + 1] - ref) - h;
    const float hd = 0.5f * d, mh = h + hd, v = mh - h;
    const float ml = (h - (mh - v)) + (hd - v);  // h + d / 2 = mh + ml exactly
    const float p = kgh * mh;
    float e = fmaf(kgh, mh, -p);
    e = fmaf(kgh, ml, e);
    e = fmaf(kgl, mh, e);
    const float pd = kgh * d;
    const float ed = fmaf(kgl, d, fmaf(kgh, d, -pd));
    return make_float2(-(p + e), -(pd + ed));
}

template <typename H, int L>
__device__ __forceinline__ void stage_planes_dx_scaled(float2 *sh, const H *Hc, int N, int Q, const float *ref,
                                                       float kgh, float kgl)
{
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
#pragma unroll
        for (int l = 0; l < L; ++l) sh[(size_t)l * N + i] = dx_record_scaled<H>(Hc, N, Q, ref[l], kgh, kgl, l, i);
    }
}

// Per-surface minimum and maximum of the node offsets h - ref_l (or of
// -kg64 (h - ref_l) for scaled planes), from the staged records (planes in
// shared memory or HBM): ext[l] = min, ext[L + l] = max.  All threads must call it, after the planes are complete
// and visible.
template <int L>
__device__ __forceinline__ void surface_extent(const float2 *planes, int N, float *ext)
{
    __shared__ float red[2 * MT_MAX_L][32];
    float lo[L], hi[L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
        lo[l] = INFINITY;
        hi[l] = -INFINITY;
    }
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
#pragma unroll
        for (int l = 0; l < L; ++l) {
            // the segment's two end nodes, hm -+ dx / 2 (their rounding is far
            // inside the saturation threshold's margin)
            const float2 r = planes[(size_t)l * N + i];
            const float half = 0.5f * fabsf(r.y);
            lo[l] = fminf(lo[l], r.x - half);
            hi[l] = fmaxf(hi[l], r.x + half);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int l = 0; l < L; ++l) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[l] = fminf(lo[l], __shfl_xor_sync(0xffffffffu, lo[l], o));
            hi[l] = fmaxf(hi[l], __shfl_xor_sync(0xffffffffu, hi[l], o));
        }
        if (lane == 0) {
            red[l][warp] = lo[l];
            red[MT_MAX_L + l][warp] = hi[l];
        }
    }
    __syncthreads();
    if (threadIdx.x < L) {
        float a = INFINITY, b = -INFINITY;
        for (int j = 0; j < nw; ++j) {
            a = fminf(a, red[threadIdx.x][j]);
            b = fmaxf(b, red[MT_MAX_L + threadIdx.x][j]);
        }
        ext[threadIdx.x] = a;
        ext[L + threadIdx.x] = b;
    }
}

template <typename S, typename T, int L>
__device__ __forceinline__ void load_node(const S *sh, int node, T (&v)[L])
{
    using NL = NodeLayout<S, L>;
    const char *src = reinterpret_cast<const char *>(sh) + (size_t)node * NL::bytes;
    alignas(16) S tmp[NL::LP];
    if constexpr (NL::bytes == 4) {
        *reinterpret_cast<uint32_t *>(tmp) = *reinterpret_cast<const uint32_t *>(src);
    } else if constexpr (NL::bytes == 8) {
        *reinterpret_cast<uint2 *>(tmp) = *reinterpret_cast<const uint2 *>(src);
    } else {
#pragma unroll
        for (int q = 0; q < NL::bytes / 16; ++q)
            reinterpret_cast<uint4 *>(tmp)[q] = reinterpret_cast<const uint4 *>(src)[q];
    }
#pragma unroll
    for (int l = 0; l < L; ++l) {
        if constexpr (sizeof(T) == 8) v[l] = tmp[l];
        else v[l] = to_f(tmp[l]);
    }
}

// ---------------------------------------------------------------- FP32 helpers
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}


// float-float (unevaluated sum hi + lo) arithmetic from error-free transforms.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b)
{
    float s = a + b;
    float v = s - a;
    float e = (a - (s - v)) + (b - v);
    return {s, e};
}
__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    FF s = ff_two_sum(a.hi, b.hi);
    float e = s.lo + a.lo + b.lo;
    return ff_two_sum(s.hi, e);
}
__device__ __forceinline__ FF ff_mul(FF a, FF b)
{
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return ff_two_sum(p, e);
}

// g(y) = e^y - 1 - y of a float-float y, to ~2^-44 relative: the centred
// Poisson term of a ray is -C g(y), and a far-off chain sums ~1e5 of those
// per log-likelihood, so a per-ray relative error of 1e-8 would already add
// ~1e-3.  For |y| <= 1, g = y^2 P(y) with P(y) = sum_{n>=2} y^(n-2) / n!
// (Taylor series of the exponential): the terms n = 2..5 in float-float
// Horner steps, the rest (relative size < |y|^4 / 360 of P) in FP32.  Larger
// |y| (a ray's expected count off its observed count by a factor e) are
// rare and take FP64.
__device__ __forceinline__ FF ff_const(double v) { return FF{(float)v, (float)(v - (double)(float)v)}; }

__device__ __forceinline__ FF g_ff(FF y)
{
    const float yh = y.hi + y.lo;
    if (!(fabsf(yh) <= 1.0f)) {
        const double yd = (double)y.hi + (double)y.lo;
        const double g = expm1(yd) - yd;
        return ff_const(g);
    }
    // tail sum_{n>=6} y^(n-6) / n! to n = 17 (1/18! < 2^-52)
    float q = (float)(1.0 / 355687428096000.0);  // 1/17!
    q = fmaf(q, yh, (float)(1.0 / 20922789888000.0));
    q = fmaf(q, yh, (float)(1.0 / 1307674368000.0));
    q = fmaf(q, yh, (float)(1.0 / 87178291200.0));
    q = fmaf(q, yh, (float)(1.0 / 6227020800.0));
    q = fmaf(q, yh, (float)(1.0 / 479001600.0));
    q = fmaf(q, yh, (float)(1.0 / 39916800.0));
    q = fmaf(q, yh, (float)(1.0 / 3628800.0));
    q = fmaf(q, yh, (float)(1.0 / 362880.0));
    q = fmaf(q, yh, (float)(1.0 / 40320.0));
    q = fmaf(q, yh, (float)(1.0 / 5040.0));
    q = fmaf(q, yh, (float)(1.0 / 720.0));
    FF p = ff_add(ff_mul(FF{q, 0.f}, y), ff_const(1.0 / 120.0));
    p = ff_add(ff_mul(p, y), ff_const(1.0 / 24.0));
    p = ff_add(ff_mul(p, y), ff_const(1.0 / 6.0));
    p = ff_add(ff_mul(p, y), FF{0.5f, 0.f});
    return ff_mul(ff_mul(y, y), p);
}

// ---------------------------------------------------------------- FP32 march
// Blackwell's paired FP32 instructions (FFMA2 / FADD2 / FMUL2) do two lanes'
// worth of FP32 work per issue slot.  Surfaces are processed in pairs; the
// cell coordinates are computed as duplicated pairs {g, g} so no broadcast
// moves are needed.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// Builds with MT_BOUNDS_CHECK verify every cell index the kernels form from
// the ray table against the grid's cells [0, Q-1) x [0, R-1): an index out
// of range latches bit 4 of the device status word and is replaced by cell
// 0, so nothing is read or written out of bounds.  Other builds compile the
// checks away (the ray table keeps every sample inside the grid).
__device__ __forceinline__ bool cell_ok(int ix, int iy, int nxc, int nyc)
{
    return (unsigned)ix < (unsigned)nxc && (unsigned)iy < (unsigned)nyc;
}

// Corner heights of one surface group at a node: a pair (NS = 2) or the odd
// last surface (NS = 1), from node-major records.
template <int L, int NS, typename S, bool GLOBAL>
__device__ __forceinline__ float2 load_group(const S *sh, int node, int l0)
{
    using NL = NodeLayout<S, L>;
    const S *rec = reinterpret_cast<const S *>(reinterpret_cast<const char *>(sh) + (size_t)node * NL::bytes);
    return make_float2(to_f(rec[l0]), NS == 2 ? to_f(rec[l0 + 1]) : 0.f);
}

// March one surface group over every sample of a ray from node-major
// records (BF16 mode) and add its integer
// indicator sums (units 2^-23) to t0 (surface l0) and t1 (l0 + 1).
template <int L, int NS, bool HARD, typename S>
__device__ __forceinline__ void march_group(const Prob &pb, const S *sh, float4 o, float4 st,
                                            int l0, float2 zh, float2 zlo,
                                            unsigned long long &t0, unsigned long long &t1)
{
    const float M = 12582912.0f;  // 1.5 * 2^23: adding it rounds to an integer
    const int Q = pb.Q;
    const float nkg = -pb.kg;
    const float2 one2 = f2(1.0f), nkg2 = f2(nkg), szh2 = f2(st.z), szl2 = f2(st.w);
    float2 h00 = f2(0.f), h01 = f2(0.f), h10 = f2(0.f), h11 = f2(0.f);
    int cur = -1;
    float kf = 0.0f;
    for (int k0 = 0; k0 < pb.G; k0 += 256) {
        const int kn = min(256, pb.G - k0);
        uint32_t a0 = 0u, a1 = 0u;
        for (int k = 0; k < kn; ++k, kf += 1.0f) {
            const float gx = fmaf(kf, st.x, o.x), gy = fmaf(kf, st.y, o.y);
            const float tx = gx + M, ty = gy + M;
            const float fxs = (gx - (tx - M)) + 0.5f, fys = (gy - (ty - M)) + 0.5f;  // in [0, 1]
            int node = (__float_as_int(ty) - 0x4B400000) * Q + (__float_as_int(tx) - 0x4B400000);
#ifdef MT_BOUNDS_CHECK
            if (!cell_ok(__float_as_int(tx) - 0x4B400000, __float_as_int(ty) - 0x4B400000, Q - 1, pb.R - 1)) {
                atomicOr(pb.flag, 4);
                node = 0;
            }
#endif
            if (node != cur) {
                cur = node;
                h00 = load_group<L, NS, S, false>(sh, node, l0);
                h01 = load_group<L, NS, S, false>(sh, node + 1, l0);
                h10 = load_group<L, NS, S, false>(sh, node + Q, l0);
                h11 = load_group<L, NS, S, false>(sh, node + Q + 1, l0);
            }
            if constexpr (NS == 2) {
                const float2 fx = f2(fxs), fy = f2(fys), kf2 = f2(kf);
                const float2 omfx = f2(1.0f - fxs), omfy = f2(1.0f - fys);
                const float2 a = fma2(fx, h01, mul2(omfx, h00));
                const float2 b = fma2(fx, h11, mul2(omfx, h10));
                const float2 sl = fma2(fy, b, mul2(omfy, a));
                const float2 zl = fma2(kf2, szl2, add2(fma2(kf2, szh2, zh), zlo));
                const float2 arg = fma2(nkg2, sl, zl);                  // -kg (s_l - z)
                float2 sg;
                if constexpr (HARD) {
                    sg.x = arg.x < 0.f ? 1.f : (arg.x > 0.f ? 0.f : 0.5f);
                    sg.y = arg.y < 0.f ? 1.f : (arg.y > 0.f ? 0.f : 0.5f);
                } else {
                    const float2 d = add2(make_float2(ex2_approx(arg.x), ex2_approx(arg.y)), one2);
                    sg = make_float2(rcp_approx(d.x), rcp_approx(d.y));
                }
                const float2 t = add2(sg, one2);
                a0 += __float_as_uint(t.x);
                a1 += __float_as_uint(t.y);
            } else {
                const float a = fmaf(fxs, h01.x, (1.0f - fxs) * h00.x);
                const float b = fmaf(fxs, h11.x, (1.0f - fxs) * h10.x);
                const float sl = fmaf(fys, b, (1.0f - fys) * a);
                const float zl = fmaf(kf, st.w, fmaf(kf, st.z, zh.x) + zlo.x);
                const float arg = fmaf(nkg, sl, zl);
                float sig;
                if constexpr (HARD) sig = arg < 0.f ? 1.f : (arg > 0.f ? 0.f : 0.5f);
                else sig = rcp_approx(1.0f + ex2_approx(arg));
                a0 += __float_as_uint(sig + 1.0f);
            }
        }
        t0 += (unsigned long long)(a0 - (uint32_t)kn * 0x3F800000u);
        if constexpr (NS == 2) t1 += (unsigned long long)(a1 - (uint32_t)kn * 0x3F800000u);
    }
}

// Per surface l the ray accumulates N_l = sum_k varsigma(s_l - z_k) exactly:
// each sigma in [0, 1] is added as the integer round(sigma * 2^23), read off
// the bits of the FP32 sum sigma + 1 (mantissa of a number in [1, 2]), into a
// wrapping uint32 that is flushed to a uint64 every 256 samples.  Heights in
// shared memory and the ray's z are both taken relative to a per-surface
// reference height ref_l, and z is carried as float-float (start and step
// each split hi + lo), so the sigmoid argument -kg (s_l - z) is formed from
// numbers the size of the surface relief and rounded only at its own scale.
// The ray table guarantees every sample's cell coordinate lies in
// [-1/2, n - 3/2), so the cell split needs no clamp.  Surfaces are marched in
// pairs with paired FP32 instructions, every sample.  Returns
// tot[l] = N_l * 2^23.
template <int L, bool HARD, typename S>
__device__ __forceinline__ void march_ray_f32(const Prob &pb, const S *sh, int ray,
                                              unsigned long long (&tot)[L])
{
    constexpr int NP = L / 2;
    constexpr bool ODD = (L & 1) != 0;
    const float4 o = pb.o4[ray], st = pb.s4[ray];
#pragma unroll
    for (int q = 0; q < NP + (ODD ? 1 : 0); ++q) {
        const int l0 = 2 * q;
        const int ns = (q < NP) ? 2 : 1;
        const float zh0 = pb.kz0[(size_t)l0 * pb.n_rays + ray];
        const float zl0 = pb.kz0[(size_t)(L + l0) * pb.n_rays + ray];
        const float zh1 = ns == 2 ? pb.kz0[(size_t)(l0 + 1) * pb.n_rays + ray] : 0.f;
        const float zl1 = ns == 2 ? pb.kz0[(size_t)(L + l0 + 1) * pb.n_rays + ray] : 0.f;
        unsigned long long t0 = 0ull, t1 = 0ull;
        if (ns == 2)
            march_group<L, 2, HARD, S>(pb, sh, o, st, l0, make_float2(zh0, zh1), make_float2(zl0, zl1),
                                       t0, t1);
        else
            march_group<L, 1, HARD, S>(pb, sh, o, st, l0, make_float2(zh0, 0.f), make_float2(zl0, 0.f),
                                       t0, t1);
        tot[l0] = t0;
        if (ns == 2) tot[l0 + 1] = t1;
    }
}

// ---------------------------------------------------------------- FP32 march, (h, dx) planes
// One surface along one ray, two consecutive samples per step: lane .x of
// every paired FP32 instruction carries sample k, lane .y sample k + 1.
//
// Arithmetic of one sample (the FP32 modes' accuracy rests on its order):
//   position  g = fmaf(k, sh, fmaf(k, sl, o)) per axis, relative to the ray's
//             start cell (the step split hi + lo), so no per-ray FP32 offset
//             enters and each sample's rounding is its own; the cell split
//             adds 1.5 * 2^23, rounding x to the nearest integer i (x is
//             taken from the cell's centre) and y down (y from the cell's
//             lower edge; __fadd2_rd).  The fraction is then formed again as
//             (k sh - i) + fmaf(k, sl, o), the product exact inside the
//             fused multiply-add, so it carries the rounding of a number
//             below one cell instead of that of g (up to 2^-18 cells after
//             64 cells of travel).
//   height    z - ref_l in metres is split into zhi = zh + k szh, exact
//             (zh, szh on a grid), and a remainder carried as kg64 times it
//             in log2 units, zlo.  Each loaded (h_mid, dx) record enters as
//             h_mid - zhi, exact wherever that distance is at most the
//             record's offset |h_mid| (zhi's grid is then the coarser) and
//             otherwise rounded at the ulp of the distance, so the x-lerps
//             (scalar FMAs on the records as loaded)
//             and the y-lerp round at the scale of the distance to the
//             surface, not of the surface's offset from ref_l (tens of
//             metres for chains far from the data); the result is
//             d = s_l - zhi.
//   argument  a = kg64 (z - s_l) in log2 units, evaluated as
//             fmaf(-kgh, d, fmaf(-kgl, d, zlo)): the small terms (the z
//             remainder and the low part of kg) enter through the addend of a
//             fused multiply-add whose product has full-width bits.  (Adding
//             a small smooth term to an FP32 value already on its own grid
//             would round coherently along the ray.)
//   indicator varsigma = 1 / (1 + 2^a) through psi = 1 / (1 + 2^|a|) <= 1/2:
//             varsigma = psi above the surface (a > 0), 1 - psi below it.  psi
//             is formed as 1 / ((2^|a| + 1) c) with c = +-2^-28 carrying a's
//             sign, rounded to the nearest integer q (units 2^-28), and the
//             sample adds q + 2^28 [a < 0], i.e. round(varsigma 2^28), exactly:
//             no 1 - psi is ever rounded in FP32, and tails of psi down to
//             2^-29 are kept.  The FP32 and compensated modes (ACC) form
//             2^|a| with exp2_acc and the reciprocal with rcp_newton, neither
//             biased beyond rounding; the approximate-logistic mode uses
//             ex2.approx and rcp.approx with their mean error corrected by a
//             factor (1 - kappa) calibrated per device (k_psi_calib).
// The integer adds c_bits >> 3 = 2^28 [a < 0] + kJunk per sample (the
// exponent bits of 2^-28 shifted down); kJunk is subtracted once per window.
// The corner records of each sample are cached and reloaded when that
// sample enters a new cell.
constexpr uint32_t kQuantBits = 0x31800000u;      // FP32 bits of 2^-28
constexpr uint32_t kJunk = kQuantBits >> 3;       // added per sample by the sign trick
constexpr unsigned long long kUnit = 1ull << 28;  // one indicator = 2^28 units

// 2^x for x >= 0 to ~1 ulp with no bias beyond rounding (the accurate
// logistic of the FP32 modes): x (clamped to 64, where the logistic is
// 2^-64, far below the 2^-28 unit) = i + f with i = round(x) and
// f in [-1/2, 1/2] exact; 2^f by a degree-6 polynomial fitted for the least
// maximum relative error on that interval (1.6e-8 in exact arithmetic with
// its coefficients in FP32; the FP32 Horner steps give at most 7.9e-8 and a
// mean error of 0.004 ulp); then
// i is added to the exponent: bits(t) << 23 = i << 23 modulo 2^32, because
// the bits of 1.5 * 2^23 shifted by 23 vanish.
__device__ __forceinline__ float2 exp2_acc(float2 x)
{
    x = make_float2(fminf(x.x, 64.0f), fminf(x.y, 64.0f));
    const float2 t = add2(x, f2(12582912.0f));                      // 1.5 * 2^23 + round(x)
    const float2 f = fma2(add2(t, f2(-12582912.0f)), f2(-1.0f), x);  // x - round(x), exact
    float2 p = f2(1.534581242594868e-04f);
    p = fma2(p, f, f2(1.3399930903688073e-03f));
    p = fma2(p, f, f2(9.618489071726799e-03f));
    p = fma2(p, f, f2(5.550328642129898e-02f));
    p = fma2(p, f, f2(2.4022646248340607e-01f));
    p = fma2(p, f, f2(6.931471824645996e-01f));
    p = fma2(p, f, f2(1.0f));
    return make_float2(__int_as_float(__float_as_int(p.x) + (__float_as_int(t.x) << 23)),
                       __int_as_float(__float_as_int(p.y) + (__float_as_int(t.y) << 23)));
}

// 1 / e with rcp.approx refined by one Newton step r + r (1 - e r).
__device__ __forceinline__ float2 rcp_newton(float2 e)
{
    const float2 r = make_float2(rcp_approx(e.x), rcp_approx(e.y));
    return fma2(r, fma2(make_float2(-e.x, -e.y), r, f2(1.0f)), r);
}

// Records of rows r and r + 1 for the two samples of a step, each pair
// loaded (predicated, no branch) only when its sample's cell address differs
// from the one cached in cA / cB.
__device__ __forceinline__ void reload_pair(uint32_t aA, uint32_t aB, uint32_t rowb, int &cA, int &cB,
                                            float2 &rA0, float2 &rA1, float2 &rB0, float2 &rB1)
{
    asm volatile("{\n\t.reg .pred pa, pb;\n\tsetp.ne.u32 pa, %8, %9;\n\tsetp.ne.u32 pb, %10, %11;\n\t"
                 "@pa ld.shared.v2.f32 {%0, %1}, [%8];\n\t"
                 "@pa ld.shared.v2.f32 {%2, %3}, [%12];\n\t"
                 "@pb ld.shared.v2.f32 {%4, %5}, [%10];\n\t"
                 "@pb ld.shared.v2.f32 {%6, %7}, [%13];\n\t}"
                 : "+f"(rA0.x), "+f"(rA0.y), "+f"(rA1.x), "+f"(rA1.y),
                   "+f"(rB0.x), "+f"(rB0.y), "+f"(rB1.x), "+f"(rB1.y)
                 : "r"(aA), "r"((uint32_t)cA), "r"(aB), "r"((uint32_t)cB), "r"(aA + rowb), "r"(aB + rowb));
    cA = (int)aA;
    cB = (int)aB;
}

template <bool HARD, bool GLOBAL, bool ACC>
__device__ __forceinline__ uint32_t dx_pair(const float2 *pl, int Q, int R, int *flag, float2 kf2, float2 ix2,
                                            float2 iy2, float2 sxh2, float2 syh2,
                                            float2 szh2, float2 szl2, float2 zh2, float2 zl2, float2 nkgh2,
                                            float2 nkgl2, uint32_t nkc, uint32_t k0, int cell0, int2 c0,
                                            int &curA, int &curB,
                                            float2 &rA0, float2 &rA1, float2 &rB0, float2 &rB1)
{
    const float2 M2 = f2(12582912.0f);  // 1.5 * 2^23: adding it rounds to an integer
    const float2 gx = fma2(kf2, sxh2, ix2);  // ix2 = o + k sl (see march_surface_dx)
    const float2 gy = fma2(kf2, syh2, iy2);
    const float2 tx = add2(gx, M2), ty = __fadd2_rd(gy, M2);  // x rounded to nearest, y down
    // The fractions (about the row segment's midpoint in x, from the lower
    // row in y) from the exact product k sh minus the cell offset, then the
    // block's low part: rounded at the scale of the fraction, not of the
    // distance from the start cell as g - round(g) would be.
    const float2 fx = add2(fma2(kf2, sxh2, fma2(tx, f2(-1.0f), M2)), ix2);
    const float2 fy = add2(fma2(kf2, syh2, fma2(ty, f2(-1.0f), M2)), iy2);
#ifdef MT_BOUNDS_CHECK
    const bool in_grid =
        cell_ok(c0.x + __float_as_int(tx.x) - 0x4B400000, c0.y + __float_as_int(ty.x) - 0x4B400000, Q - 1, R - 1) &&
        cell_ok(c0.x + __float_as_int(tx.y) - 0x4B400000, c0.y + __float_as_int(ty.y) - 0x4B400000, Q - 1, R - 1);
    if (!in_grid) atomicOr(flag, 4);
#endif
    if constexpr (GLOBAL) {
        int nA = cell0 + (__float_as_int(ty.x) - 0x4B400000) * Q + (__float_as_int(tx.x) - 0x4B400000);
        int nB = cell0 + (__float_as_int(ty.y) - 0x4B400000) * Q + (__float_as_int(tx.y) - 0x4B400000);
#ifdef MT_BOUNDS_CHECK
        if (!in_grid) nA = nB = 0;
#endif
        if (nA != curA || nB != curB) {
            curA = nA;
            curB = nB;
            rA0 = __ldg(pl + nA);
            rA1 = __ldg(pl + nA + Q);
            rB0 = __ldg(pl + nB);
            rB1 = __ldg(pl + nB + Q);
        }
    } else {
        // reload a sample's corner records when it entered a new cell:
        // predicated shared loads instead of a divergent branch.  The record's
        // byte address 8 (Q iy + ix) + base comes straight from the float bits
        // (ix = bits(tx) - 0x4B400000 + c0x, likewise iy; k0 folds the base,
        // the start cell and the bit offsets), modulo 2^32; the current cells
        // are tracked by address (-1 is never one).
        const uint32_t rowb = 8u * (uint32_t)Q;
        uint32_t aA0 = (uint32_t)__float_as_int(ty.x) * rowb + ((uint32_t)__float_as_int(tx.x) * 8u + k0);
        uint32_t aB0 = (uint32_t)__float_as_int(ty.y) * rowb + ((uint32_t)__float_as_int(tx.y) * 8u + k0);
#ifdef MT_BOUNDS_CHECK
        if (!in_grid) aA0 = aB0 = (uint32_t)__cvta_generic_to_shared(pl);
#endif
        reload_pair(aA0, aB0, rowb, curA, curB, rA0, rA1, rB0, rB1);
    }
    const float2 zhi = fma2(kf2, szh2, zh2);  // z - ref_l in metres on its grid, exact
    const float2 zlo = fma2(kf2, szl2, zl2);  // kg64 times the remainder (log2 units)
    // Heights minus zhi: h_mid - zhi is exact where it is at most |h_mid|
    // and rounds at its own ulp otherwise, so the x-lerps and the y-lerp
    // round at the scale of the distance to the surface, not of its offset
    // from ref_l.
    const float2 a = make_float2(fmaf(fx.x, rA0.y, rA0.x - zhi.x), fmaf(fx.y, rB0.y, rB0.x - zhi.y));  // row r0
    const float2 b = make_float2(fmaf(fx.x, rA1.y, rA1.x - zhi.x), fmaf(fx.y, rB1.y, rB1.x - zhi.y));  // row r0 + 1
    const float2 d = fma2(fy, fma2(a, f2(-1.0f), b), a);           // s_l - zhi
    const float2 arg = fma2(nkgh2, d, fma2(nkgl2, d, zlo));        // kg64 (z - s_l)
    if constexpr (HARD) {
        const uint32_t vx = arg.x < 0.f ? (uint32_t)kUnit : (arg.x > 0.f ? 0u : (uint32_t)(kUnit >> 1));
        const uint32_t vy = arg.y < 0.f ? (uint32_t)kUnit : (arg.y > 0.f ? 0u : (uint32_t)(kUnit >> 1));
        return vx + vy + 2u * kJunk;
    } else if constexpr (ACC) {
        const uint32_t cbx = (__float_as_uint(arg.x) & 0x80000000u) | kQuantBits;
        const uint32_t cby = (__float_as_uint(arg.y) & 0x80000000u) | kQuantBits;
        const float2 c = make_float2(__uint_as_float(cbx), __uint_as_float(cby));
        const float2 e = fma2(exp2_acc(make_float2(fabsf(arg.x), fabsf(arg.y))), c, c);  // (2^|a| + 1) c
        const float2 r = rcp_newton(e);
        const int qx = __float2int_rn(r.x), qy = __float2int_rn(r.y);
        return ((uint32_t)qx + (cbx >> 3)) + ((uint32_t)qy + (cby >> 3));
    } else {
        const uint32_t cbx = (__float_as_uint(arg.x) & 0x80000000u) | kQuantBits;
        const uint32_t cby = (__float_as_uint(arg.y) & 0x80000000u) | kQuantBits;
        const float2 c = make_float2(__uint_as_float(cbx), __uint_as_float(cby));
        // -kappa c with c's sign: (2^|a| (1 - kappa) + 1) c, the calibrated logistic
        const float2 nk = make_float2(__uint_as_float((__float_as_uint(arg.x) & 0x80000000u) ^ nkc),
                                      __uint_as_float((__float_as_uint(arg.y) & 0x80000000u) ^ nkc));
        const float2 E = make_float2(ex2_approx(fabsf(arg.x)), ex2_approx(fabsf(arg.y)));
        const float2 e = fma2(E, c, fma2(E, nk, c));
        const int qx = __float2int_rn(rcp_approx(e.x)), qy = __float2int_rn(rcp_approx(e.y));
        return ((uint32_t)qx + (cbx >> 3)) + ((uint32_t)qy + (cby >> 3));
    }
}

// Samples [lo, he) of one surface (lo even); adds the indicator sum in units
// of 2^-28 to t.  Per block of up to eight samples (< 2^32 with kJunk) the
// 32-bit sum moves to t.  An odd count (he = G) ends with one sample
// evaluated in both lanes and counted once.
template <bool HARD, bool GLOBAL, bool ACC>
__device__ __forceinline__ void march_surface_dx(const float2 *pl, int Q, int R, int *flag, float4 xa, float4 xb,
                                                 float2 szm, float nkgh, float nkgl, uint32_t nkc, float zh, float zl,
                                                 uint32_t k0, int cell0, int2 c0, int lo, int he,
                                                 unsigned long long &t)
{
    const float2 ox2 = f2(xa.x), oy2 = f2(xa.y), sxh2 = f2(xa.z), syh2 = f2(xa.w);
    const float2 sxl2 = f2(xb.x), syl2 = f2(xb.y), szh2 = f2(szm.x), szl2 = f2(szm.y);
    const float2 zh2 = f2(zh), zl2 = f2(zl), nkgh2 = f2(nkgh), nkgl2 = f2(nkgl);
    float2 rA0 = f2(0.f), rA1 = f2(0.f), rB0 = f2(0.f), rB1 = f2(0.f);
    int curA = -1, curB = -1;
    float2 kf2 = make_float2((float)lo, (float)lo + 1.0f);
#define MT_PAIR(IX, IY)                                                                                     \
    dx_pair<HARD, GLOBAL, ACC>(pl, Q, R, flag, kf2, IX, IY, sxh2, syh2, szh2, szl2, zh2, zl2, nkgh2, nkgl2, nkc, k0, \
                          cell0, c0, curA, curB, rA0, rA1, rB0, rB1)
    // The low part of the step, o + k sl, changes by far less than an ulp of
    // o per sample: it is taken once per block of eight samples [8m, 8m + 8),
    // at the block's centre for each lane (k = 8m + 3 for the even samples of
    // lane .x, 8m + 4 for the odd ones of lane .y), which leaves an error
    // within +-4 |sl| (< 4e-8 cells) that averages to zero over the block.
    // The centre depends on k only, not on where the window starts (lo is
    // even), so a sample's arithmetic is the same in every window that holds
    // it and the exact-saturation windows stay bit-identical to full ones.
    auto centre = [&](int k) {
        const float b = (float)(k & ~7);
        return make_float2(b + 3.0f, b + 4.0f);
    };
    int k = lo;
    uint32_t acc = 0u;
    float2 kc2 = centre(k), ix2 = fma2(kc2, sxl2, ox2), iy2 = fma2(kc2, syl2, oy2);
    for (; (k & 7) != 0 && k + 2 <= he; k += 2) {  // up to three steps to a block boundary
        acc += MT_PAIR(ix2, iy2);
        kf2 = add2(kf2, f2(2.0f));
    }
    t += acc;
    for (; k + 8 <= he; k += 8) {  // whole blocks
        kc2 = add2(kf2, make_float2(3.0f, 3.0f));
        ix2 = fma2(kc2, sxl2, ox2);
        iy2 = fma2(kc2, syl2, oy2);
        acc = MT_PAIR(ix2, iy2);
        kf2 = add2(kf2, f2(2.0f));
        acc += MT_PAIR(ix2, iy2);
        kf2 = add2(kf2, f2(2.0f));
        acc += MT_PAIR(ix2, iy2);
        kf2 = add2(kf2, f2(2.0f));
        acc += MT_PAIR(ix2, iy2);
        kf2 = add2(kf2, f2(2.0f));
        t += acc;
    }
    acc = 0u;
    kc2 = centre(k);
    ix2 = fma2(kc2, sxl2, ox2);
    iy2 = fma2(kc2, syl2, oy2);
    for (; k + 2 <= he; k += 2) {  // up to three steps in the last block
        acc += MT_PAIR(ix2, iy2);
        kf2 = add2(kf2, f2(2.0f));
    }
    t += acc;
    unsigned long long ns = (unsigned long long)(k - lo);
    if (k < he) {  // one sample left (he == G): both lanes evaluate it, it counts once
        kf2 = f2((float)k);
        const float c = (float)(k & ~7) + ((k & 1) ? 4.0f : 3.0f);
        t += (unsigned long long)(MT_PAIR(fma2(f2(c), sxl2, ox2), fma2(f2(c), syl2, oy2)) >> 1);
        ns += 1ull;
    }
#undef MT_PAIR
    t -= ns * (unsigned long long)kJunk;
}

// Samples whose sigmoid argument is at least kSatX (log2 units) from zero
// have integer contributions known without evaluating them: there
// psi = 1 / (1 + 2^|a|) <= 2^-29.25 (1 + 2^-21) even with ex2.approx's and
// rcp.approx's relative errors, so psi 2^28 < 1/2 rounds to 0 and the sample
// adds exactly 0 above the surface and 2^28 below it.  The margin 0.25 over
// 29 is four orders of magnitude above the FP32 rounding of the argument and
// of the window bounds (~2e-5 log2 units).
constexpr float kSatX = 29.25f;
// The same bound for the adjoint's and the BF16 march's sigma + 1 form
// (exact integer round(sigma 2^23) outside 24.25 log2 units).
constexpr float kSat = 24.25f;

// Sample window [lo, hi] in which surface l can be transitional along a ray:
// outside it |kg (z - s_l)| >= ksat for every height in [smin, smax] (offsets
// h - ref_l).  z_l(k) = z0 + k dz (scaled by kg); rdz ~ 1 / dz.  The sample
// bounds are widened by 2^-20 (|k| + 1), many times the relative rounding
// error of (bound - z0) * rdz, so the window never loses a sample.
__device__ __forceinline__ void transition_window(float z0, float dz, float rdz, float kg, float smin,
                                                  float smax, int G, int &lo, int &hi,
                                                  float ksat = kSat)
{
    const float a = kg * smin - ksat, b = kg * smax + ksat;  // z_l must lie in (a, b)
    if (!(fabsf(dz) >= 1e-20f)) {
        const bool in = z0 > a && z0 < b;
        lo = in ? 0 : G;
        hi = in ? G - 1 : -1;
        return;
    }
    if (dz < 0.f) {  // samples before the window would lie above the surface: no skipping
        lo = 0;      // (rays pointing down are rare; they evaluate every sample)
        hi = G - 1;
        return;
    }
    float ka = (a - z0) * rdz, kb = (b - z0) * rdz;
    ka -= fmaf(fabsf(ka), 0x1p-20f, 0x1p-20f);
    kb += fmaf(fabsf(kb), 0x1p-20f, 0x1p-20f);
    ka = fminf(fmaxf(floorf(ka), -1.0f), (float)G);
    kb = fminf(fmaxf(ceilf(kb), -1.0f), (float)G);
    lo = max((int)ka, 0);
    hi = min((int)kb, G - 1);
}

// Surface l of one ray in the FP32 modes: the exact integer sum
// N_l = sum_k round(varsigma(s_l - z_k) 2^28) (see dx_pair for the
// arithmetic), computed over the samples where surface l can be
// transitional (transition_window over the surface's offsets [smin, smax]);
// the other samples' contributions are exact and added analytically (2^28
// below the surface, 0 above).  A window of odd length is widened by one
// saturated sample where the ray has one and starts at an even sample (one
// more saturated sample below), so that samples go in pairs aligned with the
// blocks of march_surface_dx.  plane: surface l's records; kl: their
// shared-window base folded as in march_ray_dx (0 for HBM records).
// Returns N_l 2^28.
template <bool HARD, bool GLOBAL, bool ACC>
__device__ __forceinline__ unsigned long long march_ray_surface_dx(const Prob &pb, const float2 *plane, uint32_t kl,
                                                                   int ray, int l, float4 xa, float4 xb, int2 c0,
                                                                   int cell0, float dz, float rdz, float smin,
                                                                   float smax, unsigned long long *evaluated)
{
    const int G = pb.G;
    int lo = 0, hi = G - 1;
    if (!pb.full_windows) {
        const float zh = pb.kz1[(size_t)l * pb.n_rays + ray];
        const float zl = pb.kz1[(size_t)(pb.L + l) * pb.n_rays + ray];
        transition_window(zh + zl, dz, rdz, pb.kg, smin, smax, G, lo, hi, kSatX);
    }
    const float zhm = pb.kzm[(size_t)l * pb.n_rays + ray];
    const float zlm = pb.kzm[(size_t)(pb.L + l) * pb.n_rays + ray];
    lo = min(lo, G) & ~1;  // even start (one more, saturated, sample below)
    int he = max(hi + 1, lo);
    if (((he - lo) & 1) && he < G) ++he;  // even length where the ray allows
    if (evaluated) *evaluated += (unsigned long long)(he - lo);
    unsigned long long t = (unsigned long long)lo * kUnit;  // samples below the window
    march_surface_dx<HARD, GLOBAL, ACC>(plane, pb.Q, pb.R, pb.flag, xa, xb, pb.szm[ray], -pb.kg, -pb.kgl,
                                        __float_as_uint(-pb.psi_kc), zhm, zlm, kl, cell0, c0, lo, he, t);
    return t;
}

// The FP32 modes' march of one ray over all L surfaces (planes [l][node],
// ext = per-surface min / max offsets): emit(l, N_l 2^28) is called for
// l = 0 .. L-1 in order.
template <int L, bool HARD, bool GLOBAL, bool ACC, typename Emit>
__device__ __forceinline__ void march_ray_dx(const Prob &pb, const float2 *planes, int ray,
                                             const float *ext, unsigned long long *evaluated,
                                             Emit &&emit)
{
    const float4 xa = pb.xa4[ray], xb = pb.xb4[ray];
    const int2 c0 = pb.xc2[ray];
    const int cell0 = c0.y * pb.Q + c0.x;
    const float dz = xb.z + xb.w;
    const float rdz = rcp_approx(dz);
    uint32_t k0 = 0u;
    if constexpr (!GLOBAL)
        k0 = (uint32_t)__cvta_generic_to_shared(planes) + 8u * (uint32_t)cell0 -
             8u * 0x4B400000u * (uint32_t)(pb.Q + 1);
#pragma unroll kSurfUnroll
    for (int l = 0; l < L; ++l) {
        const uint32_t kl = GLOBAL ? 0u : k0 + 8u * (uint32_t)((size_t)l * pb.N);
        emit(l, march_ray_surface_dx<HARD, GLOBAL, ACC>(pb, planes + (size_t)l * pb.N, kl, ray, l, xa, xb, c0, cell0, dz,
                                                   rdz, ext[l], ext[L + l], evaluated));
    }
}

// ---------------------------------------------------------------- FP64 march
// Plain FP64 sum of rho(x) - rho_top along one ray (nodes: node-major, any
// address space).
template <int L, bool HARD>
__device__ __forceinline__ double march_ray_f64(const Prob &pb, const double *nodes, int ray)
{
    const double gx0 = pb.o_d[3 * ray], gy0 = pb.o_d[3 * ray + 1], z0 = pb.o_d[3 * ray + 2];
    const double sgx = pb.s_d[3 * ray], sgy = pb.s_d[3 * ray + 1], sz = pb.s_d[3 * ray + 2];
    const double gxmax = (double)(pb.Q - 1), gymax = (double)(pb.R - 1);
    const int Q = pb.Q;
    const double inv_gamma = HARD ? 1.0 : 1.0 / pb.gamma;
    double cA[L], cB[L], cC[L], cD[L];
#pragma unroll
    for (int l = 0; l < L; ++l) cA[l] = cB[l] = cC[l] = cD[l] = 0.0;
    int cur = -1;
    double sum = 0.0;
    for (int k = 0; k < pb.G; ++k) {
        const double kd = (double)k;
        double gx = fmin(fmax(fma(kd, sgx, gx0), 0.0), gxmax);
        double gy = fmin(fmax(fma(kd, sgy, gy0), 0.0), gymax);
        const double z = fma(kd, sz, z0);
        int c0 = min((int)gx, pb.Q - 2), r0 = min((int)gy, pb.R - 2);
        const double fx = gx - (double)c0, fy = gy - (double)r0;
        const int node = r0 * Q + c0;
        if (node != cur) {
            cur = node;
            double h00[L], h01[L], h10[L], h11[L];
            load_node<double, double, L>(nodes, node, h00);
            load_node<double, double, L>(nodes, node + 1, h01);
            load_node<double, double, L>(nodes, node + Q, h10);
            load_node<double, double, L>(nodes, node + Q + 1, h11);
#pragma unroll
            for (int l = 0; l < L; ++l) {
                cA[l] = h00[l];
                cB[l] = h01[l] - h00[l];
                cC[l] = h10[l] - h00[l];
                cD[l] = (h11[l] - h10[l]) - cB[l];
            }
        }
        double rho = 0.0;
#pragma unroll
        for (int l = 0; l < L; ++l) {
            const double s = fma(fy, fma(fx, cD[l], cC[l]), fma(fx, cB[l], cA[l]));
            const double u = s - z;
            double sig;
            if constexpr (HARD) sig = u > 0.0 ? 1.0 : (u < 0.0 ? 0.0 : 0.5);
            else sig = 1.0 / (1.0 + exp(-u * inv_gamma));
            rho = fma(pb.drho[l], sig, rho);
        }
        sum += rho;
    }
    return sum;
}

// Poisson constant of one pixel: C ln C - C - ln C! (0 for C = 0).
__device__ __forceinline__ double poisson_K(int C)
{
    if (C <= 0) return 0.0;
    const double c = (double)C;
    return c * log(c) - c - lgamma(c + 1.0);
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ FF warp_sum(FF v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        FF w = {__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
        v = ff_add(v, w);
    }
    return v;
}

// Fixed-order block sums; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double red_d[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) red_d[warp] = v;
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? red_d[lane] : 0.0;
        v = warp_sum(v);
    }
    return v;
}
__device__ __forceinline__ FF block_sum(FF v)
{
    __shared__ float2 red_f[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) red_f[warp] = make_float2(v.hi, v.lo);
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        const float2 w = lane < nw ? red_f[lane] : make_float2(0.f, 0.f);
        v = warp_sum(FF{w.x, w.y});
    }
    return v;
}

// ---------------------------------------------------------------- FP32 epilogue
// S + drho_l N_l with N_l = tl 2^-28 split into two exactly representable
// parts (float-float).
__device__ __forceinline__ FF add_surface(const Prob &pb, FF S, int l, unsigned long long tl)
{
    const FF n = ff_two_sum((float)(uint32_t)(tl >> 24) * 0x1p-4f, (float)(uint32_t)(tl & 0xFFFFFFu) * 0x1p-28f);
    return ff_add(S, ff_mul(FF{pb.drho_ff[l].x, pb.drho_ff[l].y}, n));
}

// One ray's term of the FP32 modes from S = G rho_top + sum_l drho_l N_l:
// O = dt S and y = a - O / Lambda in float-float; the term -C (e^y - 1 - y)
// (or -I0 e^{-O/Lambda} for C = 0) in FP32, its product by C kept exact as
// a float-float.  Writes d ll / d O_p (for the adjoint) and the ray's
// opacity and full term where asked.
__device__ __forceinline__ FF ray_term_dx(const Prob &pb, int c, int ray, int Cp, FF Sff, double *ray_O,
                                          double *ray_term)
{
    const FF Off = ff_mul(FF{pb.dt_ff[ray].x, pb.dt_ff[ray].y}, Sff);
    const FF OL = ff_mul(Off, FF{pb.invL_ff.x, pb.invL_ff.y});
    FF tf;
    float dO;  // d ll / d O_p = (lambda - C) / Lambda
    if (Cp > 0) {
        const FF yff = ff_add(FF{pb.a_ff[ray].x, pb.a_ff[ray].y}, FF{-OL.hi, -OL.lo});
        const float y = yff.hi + yff.lo, cf = (float)Cp;
        const FF g = g_ff(yff);
        tf = ff_mul(g, FF{-cf, 0.f});
        dO = cf * expm1f(y) * pb.invL_ff.x;  // lambda - C = C (e^y - 1)
    } else {
        const double lam = pb.I0 * exp(-((double)OL.hi + (double)OL.lo));
        tf = FF{(float)-lam, (float)(-lam - (double)(float)-lam)};
        dO = (float)lam * pb.invL_ff.x;
    }
    if (pb.dO) pb.dO[(size_t)c * pb.n_rays + ray] = dO;
    if (ray_O) ray_O[(size_t)c * pb.n_rays + ray] = (double)Off.hi + (double)Off.lo;
    if (ray_term) ray_term[(size_t)c * pb.n_rays + ray] = ((double)tf.hi + (double)tf.lo) + poisson_K(Cp);
    return tf;
}

// The CTA's float-float sum of ray terms into its chain partial: float2 in
// the compensated mode, FP64 otherwise (the chain's partials are then summed
// in FP64).
template <int MODE>
__device__ __forceinline__ void store_partial_ff(void *partial, FF accf)
{
    accf = block_sum(accf);
    if (threadIdx.x == 0) {
        const size_t at = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
        if constexpr (MODE == MODE_F32C)
            reinterpret_cast<float2 *>(partial)[at] = make_float2(accf.hi, accf.lo);
        else
            reinterpret_cast<double *>(partial)[at] = (double)accf.hi + (double)accf.lo;
    }
}

// ---------------------------------------------------------------- kernel
// The FP32 modes use per-surface (h, dx) planes and MT_DX_THREADS-thread
// CTAs (one per SM with the scenario's 128 KB of records); BF16 keeps
// 4-corner node records to halve shared memory; FP64 has its own march.
template <int MODE, int L> struct MarchCfg {
    static constexpr bool DX = is_dx_mode(MODE);
    static constexpr int THREADS = DX ? MT_DX_THREADS : 256;
};

// (h, dx) planes of every chain into HBM for grids too large for shared
// memory, [chain][l][node] (one block of threads per chain and node slice).
template <typename H, int L>
__global__ void __launch_bounds__(256) k_stage_dx_global(Prob pb, HRef h)
{
    const int c = blockIdx.y;
    float2 *dst = reinterpret_cast<float2 *>(pb.gnodes) + (size_t)c * L * pb.N;
    const H *Hc = chain_ptr<H>(h, c);
    const int per = (pb.N + gridDim.x - 1) / gridDim.x;
    const int n0 = blockIdx.x * per, n1 = min(pb.N, n0 + per);
    for (int i = n0 + threadIdx.x; i < n1; i += blockDim.x) {
#pragma unroll
        for (int l = 0; l < L; ++l) dst[(size_t)l * pb.N + i] = dx_record<H>(Hc, pb.N, pb.Q, pb.ref[l], l, i);
    }
}

// One CTA = one chain x rays_per_block ray slots.  Slot i marches ray
// perm[i]: the ray table orders rays by their vertical step so that the
// 32 rays of a warp have near-equal sample windows.
template <int MODE, int L, bool HARD, bool GLOBAL = false>
__global__ void __launch_bounds__(MarchCfg<MODE, L>::THREADS)
k_march(Prob pb, HRef h, int rays_per_block, void *partial, double *ray_O, double *ray_term)
{
    using Ty = Types<MODE>;
    using S = typename Ty::S;
    using Hh = typename Ty::H;
    constexpr bool DX = MarchCfg<MODE, L>::DX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int c = blockIdx.y;
    S *sh = reinterpret_cast<S *>(smem_raw);
    const float2 *planes = nullptr;
    if constexpr (DX) {
        if constexpr (GLOBAL) {
            // planes were written to HBM by k_stage_dx_global
            planes = reinterpret_cast<const float2 *>(pb.gnodes) + (size_t)c * L * pb.N;
        } else {
            stage_planes_dx<Hh, L>(reinterpret_cast<float2 *>(smem_raw), chain_ptr<Hh>(h, c), pb.N, pb.Q, pb.ref);
            planes = reinterpret_cast<const float2 *>(smem_raw);
        }
    } else {
        stage_nodes<S, Hh, L>(sh, chain_ptr<Hh>(h, c), pb.N, (MODE == MODE_F64) ? nullptr : pb.ref);
    }
    __shared__ float ext[2 * MT_MAX_L];
    if constexpr (DX) {
        __syncthreads();  // planes staged
        surface_extent<L>(planes, pb.N, ext);
    }
    __syncthreads();

    const int r_begin = blockIdx.x * rays_per_block;
    const int r_end = min(r_begin + rays_per_block, pb.n_rays);
    double acc = 0.0;
    FF accf = {0.f, 0.f};
    unsigned long long n_eval = 0ull;
    for (int slot = r_begin + threadIdx.x; slot < r_end; slot += blockDim.x) {
        const int ray = pb.perm ? pb.perm[slot] : slot;
        const int Cp = pb.cnt[ray];
        if constexpr (DX) {
            FF Sff = {pb.grho_ff.x, pb.grho_ff.y};
            march_ray_dx<L, HARD, GLOBAL, MODE != MODE_F32A>(pb, planes, ray, ext, pb.work ? &n_eval : nullptr,
                                          [&](int l, unsigned long long tl) { Sff = add_surface(pb, Sff, l, tl); });
            accf = ff_add(accf, ray_term_dx(pb, c, ray, Cp, Sff, ray_O, ray_term));
        } else {
            double O, term;
            if constexpr (MODE == MODE_F64) {
                const double S_ = march_ray_f64<L, HARD>(pb, sh, ray);
                O = pb.dt[ray] * ((double)pb.G * pb.rho_top + S_);
                if (Cp > 0) {
                    const double y = pb.a[ray] - O * pb.inv_Lambda;
                    term = (double)Cp * y - (double)Cp * expm1(y);
                } else {
                    term = -pb.I0 * exp(-O * pb.inv_Lambda);
                }
            } else {
                unsigned long long tot[L];
                march_ray_f32<L, HARD, S>(pb, sh, ray, tot);
                if (pb.work) n_eval += (unsigned long long)L * pb.G;
                double S_ = 0.0;
#pragma unroll
                for (int l = 0; l < L; ++l) S_ = fma(pb.drho[l], (double)tot[l] * 0x1p-23, S_);
                O = pb.dt[ray] * ((double)pb.G * pb.rho_top + S_);
                if (Cp > 0) {
                    const double y = pb.a[ray] - O * pb.inv_Lambda;
                    const FF g = g_ff(ff_const(y));
                    term = -(double)Cp * ((double)g.hi + (double)g.lo);
                } else {
                    term = -pb.I0 * exp(-O * pb.inv_Lambda);
                }
            }
            acc += term;
            if (ray_O) ray_O[(size_t)c * pb.n_rays + ray] = O;
            if (ray_term) ray_term[(size_t)c * pb.n_rays + ray] = term + poisson_K(Cp);
        }
    }
    if (pb.work && n_eval) atomicAdd(pb.work, n_eval);
    if constexpr (DX) {
        // the CTA's ray terms are summed in float-float (relative error ~2^-44,
        // and it leaves the FP32 pipes to the march)
        store_partial_ff<MODE>(partial, accf);
    } else {
        acc = block_sum(acc);
        if (threadIdx.x == 0) reinterpret_cast<double *>(partial)[(size_t)c * gridDim.x + blockIdx.x] = acc;
    }
}


// The FP32 modes' march for grids whose planes do not all fit in shared
// memory but one plane does: the CTA stages one surface's plane at a time
// and marches every ray of its block over that surface, keeping each ray's
// float-float sum G rho_top + sum_l drho_l N_l in shared memory between
// surfaces (same order of operations as k_march, so the results are
// identical), then forms the ray terms.  Shared memory: N (h, dx) records and
// rays_per_block float-float sums.
template <int MODE, int L, bool HARD>
__global__ void __launch_bounds__(MT_DX_THREADS)
k_march_phased(Prob pb, HRef h, int rays_per_block, void *partial, double *ray_O, double *ray_term)
{
    using Hh = typename Types<MODE>::H;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *plane = reinterpret_cast<float2 *>(smem_raw);
    float2 *sums = reinterpret_cast<float2 *>(smem_raw + (size_t)pb.N * sizeof(float2));
    const int c = blockIdx.y;
    const Hh *Hc = chain_ptr<Hh>(h, c);
    __shared__ float ext[2];
    const int r_begin = blockIdx.x * rays_per_block;
    const int r_end = min(r_begin + rays_per_block, pb.n_rays);
    const uint32_t sp = (uint32_t)__cvta_generic_to_shared(plane);
    unsigned long long n_eval = 0ull;
#pragma unroll 1
    for (int l = 0; l < L; ++l) {
        if (l) __syncthreads();  // every ray is done with the previous plane
        for (int i = threadIdx.x; i < pb.N; i += blockDim.x)
            plane[i] = dx_record<Hh>(Hc, pb.N, pb.Q, pb.ref[l], l, i);
        __syncthreads();
        surface_extent<1>(plane, pb.N, ext);
        __syncthreads();
        const float smin = ext[0], smax = ext[1];
        for (int slot = r_begin + (int)threadIdx.x, j = threadIdx.x; slot < r_end; slot += blockDim.x, j += blockDim.x) {
            const int ray = pb.perm ? pb.perm[slot] : slot;
            const float4 xa = pb.xa4[ray], xb = pb.xb4[ray];
            const int2 c0 = pb.xc2[ray];
            const int cell0 = c0.y * pb.Q + c0.x;
            const float dz = xb.z + xb.w;
            const uint32_t kl = sp + 8u * (uint32_t)cell0 - 8u * 0x4B400000u * (uint32_t)(pb.Q + 1);
            const unsigned long long t =
                march_ray_surface_dx<HARD, false, MODE != MODE_F32A>(pb, plane, kl, ray, l, xa, xb, c0, cell0, dz,
                                                                     rcp_approx(dz), smin, smax,
                                                                     pb.work ? &n_eval : nullptr);
            const float2 s0 = l ? sums[j] : pb.grho_ff;
            const FF S = add_surface(pb, FF{s0.x, s0.y}, l, t);
            sums[j] = make_float2(S.hi, S.lo);
        }
    }
    FF accf = {0.f, 0.f};
    for (int slot = r_begin + (int)threadIdx.x, j = threadIdx.x; slot < r_end; slot += blockDim.x, j += blockDim.x) {
        const int ray = pb.perm ? pb.perm[slot] : slot;
        const float2 S = sums[j];  // written by this thread
        accf = ff_add(accf, ray_term_dx(pb, c, ray, pb.cnt[ray], FF{S.x, S.y}, ray_O, ray_term));
    }
    if (pb.work && n_eval) atomicAdd(pb.work, n_eval);
    store_partial_ff<MODE>(partial, accf);
}

}  // namespace mt
