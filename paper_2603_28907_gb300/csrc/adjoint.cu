// adjoint.cu -- gradient of the log-posterior with respect to every node
// height (the differentiable forward model of Sec. 2.1.4), hand-written.
//
// For ray p with opacity O_p: d ll / d O_p = (lambda_p - C_p) / Lambda
// (Eq. def_likelihood with lambda = I0 exp(-O/Lambda)).  The opacity is
// dt * sum_k rho(x_k) with rho = rho_top + sum_l (rho_l - rho_{l+1})
// varsigma((s_l - z)/gamma), so a node height h_{l,n} receives
//   (lambda_p - C_p)/Lambda * dt * (rho_l - rho_{l+1}) * varsigma' * w_n(x_k)
// from every sample k, with varsigma' = varsigma (1 - varsigma) / gamma and
// w_n the bilinear weight of the node.  The log-prior adds -tau Q (h_l - mu_l).
//
// The forward kernel (an FP32-mode march of the same heights) writes each
// ray's d ll / d O_p; this kernel then marches every ray once more, one
// surface at a time, over the samples near the surface, and scatters.  A
// lane sums its contributions per cell in FP32 registers (in sample order)
// and adds each cell's sums to 64-bit fixed-point
// accumulators (units of 2^-24) with integer atomics, so the gradient does not
// depend on the order in which threads add and is reproducible bit for bit; a
// sum that rounds to zero at that resolution is not added.  The unit is at or
// below the FP32 rounding of any cell sum of magnitude >= 1 (and of the SFU
// approximations' ~1e-7 relative error in each term).  The scatter visits only the
// samples within log2|coef_l| + 4 log2 units of surface l (coef_l: the sample
// weight in fixed-point units; a warp uses its largest); every sample outside
// has varsigma' <= 2^-(that) and adds less than 2^-4 units; varsigma' falls
// off geometrically along the ray, so all of them together add less than
// 2^-4 / (1 - 2^-s) units per cell and side (s: the ray's vertical step per
// sample in log2 units), and never more than G 2^-4.
#include <math.h>

#include "march.cuh"

namespace mt {

constexpr float kFix = 16777216.0f;  // 2^24
constexpr double kInvFix = 1.0 / 16777216.0;

// Add round(v) (to nearest, ties to even) to a fixed-point accumulator, with
// FP32 and integer operations only (a 64-bit float -> integer conversion runs
// on the FP64 pipe, which is slow on this part).
__device__ __forceinline__ void add_fixed(unsigned long long *p, float v)
{
    const float a = fabsf(v);
    long long q;
    if (a < 4194304.0f) {  // |v| < 2^22: adding 1.5 * 2^23 rounds to an integer
        q = (long long)(__float_as_int(v + 12582912.0f) - 0x4B400000);
    } else {               // |v| = m 2^(e - 150) with m the 24-bit significand
        const uint32_t bits = __float_as_uint(a);
        const uint32_t e = min(bits >> 23, 190u), m = (bits & 0x7FFFFFu) | 0x800000u;
        const unsigned long long mag = e >= 150u ? (unsigned long long)m << (e - 150u)
                                                 : (unsigned long long)((m >> 1) + (m & (m >> 1) & 1u));
        q = v < 0.f ? -(long long)mag : (long long)mag;
    }
    if (q != 0) atomicAdd(p, (unsigned long long)q);
}

// Surface l's corner heights of the cell at `node` from node-major records.
template <int L>
__device__ __forceinline__ void cell_corners(const float *sh, int node, int Q, int l, float &h00,
                                             float &d0, float &h10, float &d1)
{
    constexpr int LP = NodeLayout<float, L>::LP;
    h00 = sh[node * LP + l];
    d0 = sh[(node + 1) * LP + l] - h00;
    h10 = sh[(node + Q) * LP + l];
    d1 = sh[(node + Q + 1) * LP + l] - h10;
}

// Per-surface minimum / maximum of node-major records (block reduction into
// ext[l], ext[L + l]); all threads call it after the records are staged.
template <int L>
__device__ __forceinline__ void node_extent(const float *sh, int N, float *ext)
{
    constexpr int LP = NodeLayout<float, L>::LP;
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
            const float v = sh[i * LP + l];
            lo[l] = fminf(lo[l], v);
            hi[l] = fmaxf(hi[l], v);
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

// The four corner sums of a cell into the fixed-point accumulators.
__device__ __forceinline__ void flush_cell(unsigned long long *al, int cell, int Q, float c00, float c01,
                                           float c10, float c11)
{
    add_fixed(al + cell, c00);
    add_fixed(al + cell + 1, c01);
    add_fixed(al + cell + Q, c10);
    add_fixed(al + cell + Q + 1, c11);
}

// Surface l over samples [lo, he): scatter coef * varsigma' * w_n
// into acc[l][node].  Sums are kept per cell in registers; when a sample
// leaves its cell the cell's sums move to a pending slot, and the pending
// slots of all the warp's lanes are added to the fixed-point accumulators
// together, only when some lane needs its slot again (so the atomics run
// with most lanes active instead of one lane at every cell change; integer
// adds commute, so the result does not depend on when they happen).
template <int L>
__device__ __forceinline__ void scatter_surface(const Prob &pb, const float *sh, int l, float4 o,
                                                float4 st, float zh, float zl, int lo, int he,
                                                float coef, unsigned long long *acc)
{
    const float M = 12582912.0f;
    const float nkg = -pb.kg;
    const int Q = pb.Q;
    unsigned long long *al = acc + (size_t)l * pb.N;
    float h00 = 0.f, d0 = 0.f, h10 = 0.f, d1 = 0.f;
    float c00 = 0.f, c01 = 0.f, c10 = 0.f, c11 = 0.f;
    float p00 = 0.f, p01 = 0.f, p10 = 0.f, p11 = 0.f;
    int cur = -1, pend = -1;  // current cell; cell of the pending sums (-1: none)
    float kf = (float)lo;
    for (int k = lo; k < he; ++k, kf += 1.0f) {
        const float gx = fmaf(kf, st.x, o.x), gy = fmaf(kf, st.y, o.y);
        const float tx = gx + M, ty = gy + M;
        const float fx = (gx - (tx - M)) + 0.5f, fy = (gy - (ty - M)) + 0.5f;
        int node = (__float_as_int(ty) - 0x4B400000) * Q + (__float_as_int(tx) - 0x4B400000);
#ifdef MT_BOUNDS_CHECK
        if (!cell_ok(__float_as_int(tx) - 0x4B400000, __float_as_int(ty) - 0x4B400000, Q - 1, pb.R - 1)) {
            atomicOr(pb.flag, 4);
            node = 0;
        }
#endif
        const bool chg = node != cur;
        if (__any_sync(__activemask(), chg && pend >= 0)) {
            if (pend >= 0) {
                flush_cell(al, pend, Q, p00, p01, p10, p11);
                pend = -1;
            }
        }
        if (chg) {
            pend = cur;
            p00 = c00;
            p01 = c01;
            p10 = c10;
            p11 = c11;
            c00 = c01 = c10 = c11 = 0.f;
            cur = node;
            cell_corners<L>(sh, node, Q, l, h00, d0, h10, d1);
        }
        const float a = fmaf(fx, d0, h00), b = fmaf(fx, d1, h10);
        const float sl = fmaf(fy, fmaf(a, -1.0f, b), a);
        const float zlv = fmaf(kf, st.w, fmaf(kf, st.z, zh) + zl);
        // varsigma (1 - varsigma) = e / (1 + e)^2 is symmetric in the sign of
        // the argument; with e = 2^-|arg| <= 1 nothing overflows
        const float e = ex2_approx(-fabsf(fmaf(nkg, sl, zlv)));
        const float sg = rcp_approx(1.0f + e);
        const float v = coef * (e * sg * sg);
        const float vy = v * fy, vny = v - vy;  // v fy, v (1 - fy)
        c00 = fmaf(-fx, vny, c00 + vny);        // v (1 - fx)(1 - fy)
        c01 = fmaf(fx, vny, c01);               // v fx (1 - fy)
        c10 = fmaf(-fx, vy, c10 + vy);          // v (1 - fx) fy
        c11 = fmaf(fx, vy, c11);                // v fx fy
    }
    if (pend >= 0) flush_cell(al, pend, Q, p00, p01, p10, p11);
    if (cur >= 0) flush_cell(al, cur, Q, c00, c01, c10, c11);
}

// ---------------------------------------------------------------- adjoint on the (h, dx) planes
// The scatter on the forward march's scaled (h, dx) planes (shared memory),
// one surface at a time: a CTA holds every surface's plane plus one plane of
// fixed-point accumulators, which it adds to the chain's accumulators in HBM
// after each surface.  The fixed-point unit is a power of two per chain,
// 2^E with 2^(E + 28) >= max_p |coef_p| (coef_p = dO_p dt_p max_l |drho_l| /
// gamma), so a sample's weight is at most 2^28 units and a cell's sums
// nearly always convert with one 32-bit rounding; the totals are rescaled
// exactly to the shared 2^-24 unit when they leave the CTA (a right shift,
// rounding to nearest, for chains whose unit is finer).
#ifndef MT_ADJ_THREADS
#define MT_ADJ_THREADS 1024
#endif
constexpr int kAdjDxThreads = MT_ADJ_THREADS;

// Add round(v) (units) to the shared-memory accumulator at shared-window
// address a.  |v| < 2^31 converts with one 32-bit rounding; larger v split
// into a multiple of 2^22 (rounded by adding 1.5 * 2^45; |v| is clamped to
// 2^43, far beyond any weight a finite state produces) and a remainder.
__device__ __forceinline__ void red_fixed(uint32_t a, float v)
{
    long long q;
    if (fabsf(v) < 2147483520.0f) {  // the largest FP32 value below 2^31
        q = (long long)__float2int_rn(v);
    } else {
        const float M45 = 52776558133248.0f;  // 1.5 * 2^45: ulp 2^22
        const float vc = fminf(fmaxf(v, -8796093022208.0f), 8796093022208.0f);
        const float t = vc + M45;
        const float lo = vc - (t - M45);  // exact, |lo| <= 2^21
        q = ((long long)(__float_as_int(t) - __float_as_int(M45)) << 22) +
            (long long)(__float_as_int(lo + 12582912.0f) - 0x4B400000);
    }
    if (q != 0) asm volatile("red.shared.add.u64 [%0], %1;" ::"r"(a), "l"(q) : "memory");
}

// A cell's sums U0, U1 (row r), V0, V1 (row r + 1) onto its four nodes; a:
// accumulator address of node (r, c), rowb: bytes per row.
__device__ __forceinline__ void flush_dx(uint32_t a, uint32_t rowb, float U0, float U1, float V0, float V1)
{
    red_fixed(a, fmaf(0.5f, U0, -U1));
    red_fixed(a + 8u, fmaf(0.5f, U0, U1));
    red_fixed(a + rowb, fmaf(0.5f, V0, -V1));
    red_fixed(a + rowb + 8u, fmaf(0.5f, V0, V1));
}

// A pending cell's sums (record address x; pu = {U0, U1}, pw = {V0, V1})
// leave the lane while the next cell along the ray (record address y, sums
// uu, ww) is still accumulating.  After a step in x or y the two cells share
// two nodes: those two corner sums are added to the next cell's sums (the
// U/V form takes them as they are: a node on the shared column adds +-q/2 to
// U1 or V1 and q to U0 or V0, a shared row moves whole), and only the other
// two nodes are added to the accumulators; after a diagonal step all four.
// This halves the accumulator atomics along a ray; every node's share still
// reaches the accumulators exactly once.
__device__ __forceinline__ void flush_carry(uint32_t to_acc, uint32_t rowb, int x, float2 pu, float2 pw, int y,
                                            float2 &uu, float2 &ww)
{
    const float q00 = fmaf(0.5f, pu.x, -pu.y), q01 = fmaf(0.5f, pu.x, pu.y);
    const float q10 = fmaf(0.5f, pw.x, -pw.y), q11 = fmaf(0.5f, pw.x, pw.y);
    const int d = y - x;
    const bool xp = d == 8, xm = d == -8, yp = d == (int)rowb, ym = d == -(int)rowb;
    const uint32_t a = (uint32_t)x + to_acc;
    // the two nodes the next cell does not share (the lower two after a step
    // up, the upper two after a step down, the left column after a step
    // right, the right one after a step left; the lower two otherwise)
    const uint32_t a0 = xm ? a + 8u : (ym ? a + rowb : a);
    const uint32_t a1 = (xp | xm) ? a0 + rowb : a0 + 8u;
    const float v0 = xm ? q01 : (ym ? q10 : q00);
    const float v1 = xp ? q10 : (xm ? q11 : (ym ? q11 : q01));
    red_fixed(a0, v0);
    red_fixed(a1, v1);
    // carried into the next cell (selects, no branch): a shared column adds q
    // to U0 / V0 and -+q/2 to U1 / V1; the upper row moves whole into the
    // lower one after a step up, the lower into the upper after a step down
    const bool ax = xp | xm;
    const float cu = xp ? q01 : q00, cw = xp ? q11 : q10, h = xp ? -0.5f : 0.5f;
    const float2 du = ax ? make_float2(cu, h * cu) : (yp ? pw : f2(0.f));
    const float2 dw = ax ? make_float2(cw, h * cw) : (ym ? pu : f2(0.f));
    uu = add2(uu, du);
    ww = add2(ww, dw);
    if (!(ax | yp | ym)) {  // a diagonal step: the upper two nodes as well
        red_fixed(a + rowb, q10);
        red_fixed(a + rowb + 8u, q11);
    }
}

// Surface l along one ray: samples within the window where a weight can
// reach one unit, two per step in paired FP32 lanes (lane .x sample k,
// lane .y sample k + 1; positions from the ray's start cell, the records
// scaled to argument units and lerped, z added in log2 units: the argument
// a = kg64 (z - s_l) to the rounding of the surface's offset, which the
// gradient's accuracy does not need to go below; the forward march forms it
// from exact differences instead).  Per sample the weight
// v = coef psi (1 - psi) with psi (1 - psi) = 2^-|a| / (1 + 2^-|a|)^2
// (d varsigma / d s_l = psi (1 - psi) / gamma) goes to the cell's nodes with
// the bilinear weights: with the records' x-fraction f in [-1/2, 1/2] the
// two nodes of a row get 1/2 - f and 1/2 + f, and the rows 1 - fy and fy.
// A lane keeps per cell the sums U0 = sum v (1 - fy), U1 = sum v (1 - fy) f,
// V0 = sum v fy, V1 = sum v fy f and moves them to a pending slot when a
// sample enters the next cell (samples in order along the ray visit each
// cell once); the warp's pending slots are added to the accumulators
// together, when some lane needs its slot again.  pbase: shared-window
// address of plane l; to_acc: accumulator address minus record address.
template <int L>
__device__ __forceinline__ void scatter_ray_dx(const Prob &pb, int ray, int l, float coef, const float *ext,
                                               uint32_t pbase, uint32_t to_acc)
{
    const float4 xa = pb.xa4[ray], xb = pb.xb4[ray];
    const int2 c0 = pb.xc2[ray];
    const int Q = pb.Q, G = pb.G;
    const float dz = xb.z + xb.w, rdz = rcp_approx(dz);
    const float zh = pb.kz1[(size_t)l * pb.n_rays + ray], zl = pb.kz1[(size_t)(L + l) * pb.n_rays + ray];
    // psi (1 - psi) <= 2^-|a|: beyond |a| = log2|coef| a sample adds less
    // than one unit (2^-28 of the chain's largest ray weight) to any node,
    // and all of them together, falling off geometrically along the ray, less
    // than 1 / (1 - 2^-s) units per node and side (s: the vertical step per
    // sample in log2 units); the warp takes its largest width so that its
    // lanes run loops of near-equal length
    float ka = fmaxf(log2f(fabsf(coef) + 1e-30f), 1.0f);
    ka = __int_as_float(__reduce_max_sync(__activemask(), __float_as_int(ka)));
    int lo, hi;
    transition_window(zh + zl, dz, rdz, 1.0f, -ext[L + l], -ext[l], G, lo, hi, ka);
    lo = min(lo, G);
    const int he = max(hi + 1, lo);

    const float2 M2 = f2(12582912.0f);
    const float2 ox2 = f2(xa.x), oy2 = f2(xa.y), sxh2 = f2(xa.z), syh2 = f2(xa.w);
    const float2 sxl2 = f2(xb.x), syl2 = f2(xb.y), szh2 = f2(xb.z), szl2 = f2(xb.w);
    const float2 zh2 = f2(zh), zl2 = f2(zl);
    const uint32_t rowb = 8u * (uint32_t)Q;
    // record address 8 (Q iy + ix) + pbase from the float bits of the cell
    // coordinates (as in the forward march)
    const uint32_t k0 = pbase + 8u * (uint32_t)(c0.y * Q + c0.x) - 8u * 0x4B400000u * (uint32_t)(Q + 1);
    float2 rA0 = f2(0.f), rA1 = f2(0.f), rB0 = f2(0.f), rB1 = f2(0.f);
    int curA = -1, curB = -1, cur = -1, pend = -1;
    float2 uu = f2(0.f), ww = f2(0.f), pu = f2(0.f), pw = f2(0.f);  // {U0, U1}, {V0, V1}; pending

    auto step = [&](float2 kf, float cB) {
        const float2 gx = fma2(kf, sxh2, fma2(kf, sxl2, ox2)), gy = fma2(kf, syh2, fma2(kf, syl2, oy2));
        const float2 tx = add2(gx, M2), ty = __fadd2_rd(gy, M2);  // x rounded to nearest, y down
        const float2 fx = fma2(add2(tx, f2(-12582912.0f)), f2(-1.0f), gx);
        const float2 fy = fma2(add2(ty, f2(-12582912.0f)), f2(-1.0f), gy);
        uint32_t aA0 = (uint32_t)__float_as_int(ty.x) * rowb + ((uint32_t)__float_as_int(tx.x) * 8u + k0);
        uint32_t aB0 = (uint32_t)__float_as_int(ty.y) * rowb + ((uint32_t)__float_as_int(tx.y) * 8u + k0);
#ifdef MT_BOUNDS_CHECK
        if (!(cell_ok(c0.x + __float_as_int(tx.x) - 0x4B400000, c0.y + __float_as_int(ty.x) - 0x4B400000, Q - 1,
                      pb.R - 1) &&
              cell_ok(c0.x + __float_as_int(tx.y) - 0x4B400000, c0.y + __float_as_int(ty.y) - 0x4B400000, Q - 1,
                      pb.R - 1))) {
            atomicOr(pb.flag, 4);
            aA0 = aB0 = pbase;
        }
#endif
        reload_pair(aA0, aB0, rowb, curA, curB, rA0, rA1, rB0, rB1);
        const float2 a = make_float2(fmaf(fx.x, rA0.y, rA0.x), fmaf(fx.y, rB0.y, rB0.x));  // row r
        const float2 b = make_float2(fmaf(fx.x, rA1.y, rA1.x), fmaf(fx.y, rB1.y, rB1.x));  // row r + 1
        const float2 sl = fma2(fy, fma2(a, f2(-1.0f), b), a);  // -kg64 (s_l - ref_l)
        const float2 arg = add2(add2(sl, fma2(kf, szh2, zh2)), fma2(kf, szl2, zl2));
        const float2 e = make_float2(ex2_approx(-fabsf(arg.x)), ex2_approx(-fabsf(arg.y)));
        const float2 d = add2(e, f2(1.0f));
        const float2 r = make_float2(rcp_approx(d.x), rcp_approx(d.y));
        const float2 v = mul2(mul2(make_float2(coef, cB), e), mul2(r, r));
        const float2 vy = mul2(v, fy);
        const float2 vny = fma2(vy, f2(-1.0f), v);  // v (1 - fy)
        // sample A, then B, in order along the ray
        const int ia = (int)aA0, ib = (int)aB0;
        const bool chA = ia != cur, chB = ib != ia;
        if (__any_sync(__activemask(), (chA || chB) && pend >= 0)) {
            if (pend >= 0) {
                flush_carry(to_acc, rowb, pend, pu, pw, cur, uu, ww);
                pend = -1;
            }
        }
        // the cell sums move on when a sample enters the next cell: one
        // region for the first (or only) move of the step, A's share added
        // before it when only B moved (A stayed) and after it otherwise, and
        // a rare second region when B moved on again
        if (chB && !chA) {
            uu = fma2(f2(vny.x), make_float2(1.0f, fx.x), uu);
            ww = fma2(f2(vy.x), make_float2(1.0f, fx.x), ww);
        }
        if (chA || chB) {
            if (cur >= 0) {
                pend = cur;
                pu = uu;
                pw = ww;
            }
            uu = ww = f2(0.f);
            cur = chA ? ia : ib;
        }
        if (chA || !chB) {
            uu = fma2(f2(vny.x), make_float2(1.0f, fx.x), uu);
            ww = fma2(f2(vy.x), make_float2(1.0f, fx.x), ww);
        }
        if (chA && chB) {  // B entered yet another cell (rare): the second move
            flush_carry(to_acc, rowb, pend, pu, pw, cur, uu, ww);
            pend = cur;
            pu = uu;
            pw = ww;
            uu = ww = f2(0.f);
            cur = ib;
        }
        uu = fma2(f2(vny.y), make_float2(1.0f, fx.y), uu);
        ww = fma2(f2(vy.y), make_float2(1.0f, fx.y), ww);
    };

    int k = lo;
    float2 kf2 = make_float2((float)lo, (float)lo + 1.0f);
    for (; k + 2 <= he; k += 2) {
        step(kf2, coef);
        kf2 = add2(kf2, f2(2.0f));
    }
    if (k < he) step(f2(kf2.x), 0.0f);  // last sample of an odd window: lane .y repeats it with weight 0
    if (pend >= 0) flush_carry(to_acc, rowb, pend, pu, pw, cur, uu, ww);
    if (cur >= 0) flush_dx((uint32_t)cur + to_acc, rowb, uu.x, uu.y, ww.x, ww.y);
}

// A CTA total in units 2^E as a multiple of 2^-24 (shift = E + 24): exact
// for shift >= 0, rounded to nearest otherwise.
__device__ __forceinline__ unsigned long long to_fix24(long long v, int shift)
{
    if (shift >= 0) return (unsigned long long)v << shift;
    if (shift <= -63) return 0ull;
    return (unsigned long long)((v + (1ll << (-shift - 1))) >> (-shift));
}

// Per chain: unit_e[c] = E with 2^(E + 27) < max_p |dO_p dt_p| max_l |drho_l|
// / gamma <= 2^(E + 28) (E = -24, the absolute unit, when that is 0 or not
// finite); E is kept in [-100, 100].
__global__ void __launch_bounds__(1024) k_adj_unit(Prob pb, int *unit_e)
{
    const int c = blockIdx.x;
    const float *dO = pb.dO + (size_t)c * pb.n_rays;
    float m = 0.f;
    for (int p = threadIdx.x; p < pb.n_rays; p += blockDim.x) m = fmaxf(m, fabsf(dO[p] * pb.dt_ff[p].x));
    __shared__ int red[32];
    int mi = __reduce_max_sync(0xffffffffu, __float_as_int(m));  // m >= 0: ordered as integers
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mi;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 1; j < (int)(blockDim.x >> 5); ++j) mi = max(mi, red[j]);
        float dr = 0.f;
        for (int l = 0; l < pb.L; ++l) dr = fmaxf(dr, fabsf(pb.drho_f[l]));
        const float mm = __int_as_float(mi) * dr * (float)(1.0 / pb.gamma);
        int e = 4;
        if (mm > 0.f && mm <= 3.0e38f) frexpf(mm, &e);
        unit_e[c] = min(max(e - 28, -100), 100);
    }
}

template <int L>
__global__ void __launch_bounds__(kAdjDxThreads)
k_adjoint_dx(Prob pb, HRef h, int rays_per_block, const int *unit_e, unsigned long long *gacc)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *planes = reinterpret_cast<float2 *>(smem_raw);
    const int c = blockIdx.y, N = pb.N;
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(smem_raw + (size_t)L * N * sizeof(float2));
    stage_planes_dx_scaled<float, L>(planes, chain_ptr<float>(h, c), N, pb.Q, pb.ref, pb.kg, pb.kgl);
    for (int i = threadIdx.x; i < N; i += blockDim.x) acc[i] = 0ull;
    __shared__ float ext[2 * MT_MAX_L];
    __syncthreads();
    surface_extent<L>(planes, N, ext);
    __syncthreads();
    const int E = unit_e[c];
    const float cg = ldexpf((float)(1.0 / pb.gamma), -E);  // 1 / (gamma 2^E)
    const uint32_t sp = (uint32_t)__cvta_generic_to_shared(planes);
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(acc);
    unsigned long long *gc = gacc + (size_t)c * L * N;
    const int r_begin = blockIdx.x * rays_per_block;
    const int r_end = min(r_begin + rays_per_block, pb.n_rays);
#pragma unroll 1
    for (int l = 0; l < L; ++l) {
        const uint32_t pbase = sp + 8u * (uint32_t)(l * N);
        const float cl = pb.drho_f[l] * cg;
        for (int slot = r_begin + threadIdx.x; slot < r_end; slot += blockDim.x) {
            const int ray = pb.perm ? pb.perm[slot] : slot;
            const float coef = cl * (pb.dO[(size_t)c * pb.n_rays + ray] * pb.dt_ff[ray].x);
            scatter_ray_dx<L>(pb, ray, l, coef, ext, pbase, sa - pbase);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const long long v = (long long)acc[i];
            acc[i] = 0ull;
            if (v) atomicAdd(gc + (size_t)l * N + i, to_fix24(v, E + 24));
        }
        __syncthreads();
    }
}

bool adjoint_dx_fits(const Prob &pb)
{
    return (size_t)(pb.L + 1) * pb.N * 8 + MT_SMEM_STATIC <= MT_MAX_SMEM;
}

template <int L>
static cudaError_t adj_dx_l(const Prob &pb, HRef h, int n_chains, int rpb, unsigned long long *gacc,
                            cudaStream_t st)
{
    const size_t bytes = (size_t)(L + 1) * pb.N * 8;
    static size_t set = 0;
    if (bytes > 48 * 1024 && bytes > set) {
        cudaError_t e = cudaFuncSetAttribute(k_adjoint_dx<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        set = bytes;
    }
    int *unit_e = reinterpret_cast<int *>(pb.dO + (size_t)n_chains * pb.n_rays);
    k_adj_unit<<<n_chains, 1024, 0, st>>>(pb, unit_e);
    dim3 grid((pb.n_rays + rpb - 1) / rpb, n_chains);
    k_adjoint_dx<L><<<grid, kAdjDxThreads, bytes, st>>>(pb, h, rpb, unit_e, gacc);
    return cudaGetLastError();
}

// One CTA = one chain x one block of ray slots (slot i -> ray perm[i]).  SMEM:
// accumulate in shared memory and flush once per CTA; otherwise add straight
// into global memory.
constexpr int kAdjThreads = 1024;  // one CTA per SM with the scenario's 192 KB of shared memory

template <int L, bool SMEM>
__global__ void __launch_bounds__(kAdjThreads)
k_adjoint(Prob pb, HRef h, int rays_per_block, unsigned long long *gacc)
{
    using NL = NodeLayout<float, L>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sh = reinterpret_cast<float *>(smem_raw);
    const int c = blockIdx.y;
    const int N = pb.N;
    const size_t rec = ((size_t)N * NL::bytes + 255) & ~(size_t)255;
    unsigned long long *acc_s = reinterpret_cast<unsigned long long *>(smem_raw + rec);
    unsigned long long *gc = gacc + (size_t)c * L * N;
    stage_nodes<float, float, L>(sh, chain_ptr<float>(h, c), N, pb.ref);
    if constexpr (SMEM)
        for (int i = threadIdx.x; i < L * N; i += blockDim.x) acc_s[i] = 0ull;
    __shared__ float ext[2 * MT_MAX_L];
    __syncthreads();
    node_extent<L>(sh, N, ext);
    __syncthreads();
    unsigned long long *acc = SMEM ? acc_s : gc;

    const int r_begin = blockIdx.x * rays_per_block;
    const int r_end = min(r_begin + rays_per_block, pb.n_rays);
    for (int slot = r_begin + threadIdx.x; slot < r_end; slot += blockDim.x) {
        const int ray = pb.perm ? pb.perm[slot] : slot;
        const float4 o = pb.o4[ray], st = pb.s4[ray];
        const float rdz = rcp_approx(st.z);
        const float dO = pb.dO[(size_t)c * pb.n_rays + ray];  // d ll / d O_p from the march
        const float base = dO * pb.dt_ff[ray].x * (float)(1.0 / pb.gamma) * kFix;
#pragma unroll 1
        for (int l = 0; l < L; ++l) {
            const float coef = base * pb.drho_f[l];
            // samples beyond log2|coef| + 4 log2 units from the surface add
            // less than 2^-4 fixed-point units each; the warp takes its
            // largest such width (its rays have near-equal windows) so that
            // its lanes run loops of equal length
            float ka = fmaxf(log2f(fabsf(coef) + 1e-30f) + 4.0f, 1.0f);
            ka = __int_as_float(__reduce_max_sync(__activemask(), __float_as_int(ka)));
            const float zh = pb.kz0[(size_t)l * pb.n_rays + ray];
            const float zl = pb.kz0[(size_t)(L + l) * pb.n_rays + ray];
            int lo, hi;
            transition_window(zh, st.z, rdz, pb.kg, ext[l], ext[L + l], pb.G, lo, hi, ka);
            lo = min(lo, pb.G);
            const int he = max(hi + 1, lo);
            scatter_surface<L>(pb, sh, l, o, st, zh, zl, lo, he, coef, acc);
        }
    }
    if constexpr (SMEM) {
        __syncthreads();
        for (int i = threadIdx.x; i < L * N; i += blockDim.x) {
            const unsigned long long v = acc_s[i];
            if (v) atomicAdd(gc + i, v);
        }
    }
}

size_t adjoint_smem_bytes(const Prob &pb, bool with_acc)
{
    const int raw = pb.L * 4;
    const int bytes = raw <= 4 ? 4 : raw <= 8 ? 8 : ((raw + 15) / 16) * 16;
    const size_t rec = ((size_t)pb.N * bytes + 255) & ~(size_t)255;
    return rec + (with_acc ? (size_t)pb.L * pb.N * 8 : 0);
}

template <int L>
static cudaError_t adj_l(const Prob &pb, HRef h, int n_chains, int rpb, unsigned long long *gacc,
                         cudaStream_t st)
{
    const size_t with = adjoint_smem_bytes(pb, true);
    const bool smem_acc = with + MT_SMEM_STATIC <= MT_MAX_SMEM;
    const size_t bytes = smem_acc ? with : adjoint_smem_bytes(pb, false);
    void (*fn)(Prob, HRef, int, unsigned long long *) = smem_acc ? k_adjoint<L, true> : k_adjoint<L, false>;
    static size_t set[2] = {0, 0};
    if (bytes > 48 * 1024 && bytes > set[smem_acc]) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        set[smem_acc] = bytes;
    }
    dim3 grid((pb.n_rays + rpb - 1) / rpb, n_chains);
    fn<<<grid, kAdjThreads, bytes, st>>>(pb, h, rpb, gacc);
    return cudaGetLastError();
}

// gacc: [n_chains][L][N] zeroed by the caller; pb.dO: [n_chains][n_rays] followed by
// n_chains ints of scratch (the per-chain fixed-point units).
cudaError_t launch_adjoint(const Prob &pb, HRef h, int n_chains, unsigned long long *gacc, cudaStream_t st)
{
    if (!pb.dO) return cudaErrorInvalidValue;
    const int rpb = march_rays_per_block(pb);
    if (adjoint_dx_fits(pb)) {
        switch (pb.L) {
            case 1: return adj_dx_l<1>(pb, h, n_chains, rpb, gacc, st);
            case 2: return adj_dx_l<2>(pb, h, n_chains, rpb, gacc, st);
            case 3: return adj_dx_l<3>(pb, h, n_chains, rpb, gacc, st);
            case 4: return adj_dx_l<4>(pb, h, n_chains, rpb, gacc, st);
            case 5: return adj_dx_l<5>(pb, h, n_chains, rpb, gacc, st);
            case 6: return adj_dx_l<6>(pb, h, n_chains, rpb, gacc, st);
            case 7: return adj_dx_l<7>(pb, h, n_chains, rpb, gacc, st);
            case 8: return adj_dx_l<8>(pb, h, n_chains, rpb, gacc, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (pb.L) {
        case 1: return adj_l<1>(pb, h, n_chains, rpb, gacc, st);
        case 2: return adj_l<2>(pb, h, n_chains, rpb, gacc, st);
        case 3: return adj_l<3>(pb, h, n_chains, rpb, gacc, st);
        case 4: return adj_l<4>(pb, h, n_chains, rpb, gacc, st);
        case 5: return adj_l<5>(pb, h, n_chains, rpb, gacc, st);
        case 6: return adj_l<6>(pb, h, n_chains, rpb, gacc, st);
        case 7: return adj_l<7>(pb, h, n_chains, rpb, gacc, st);
        case 8: return adj_l<8>(pb, h, n_chains, rpb, gacc, st);
        default: return cudaErrorInvalidValue;
    }
}

// grad[c][i] = gacc * 2^-24 - tau (Q (h - mu))_i, and logpost = ll + lp.
template <typename H>
__global__ void k_grad_finish(Prob pb, HRef h, const double *mu, const unsigned long long *gacc,
                              double *grad)
{
    const int c = blockIdx.y;
    const int n = pb.L * pb.N;
    const H *Hc = chain_ptr<H>(h, c);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int l = i / pb.N, rc = i - l * pb.N, r = rc / pb.Q, cc = rc - r * pb.Q;
        const int up = r + 1 == pb.R ? 0 : r + 1, dn = r == 0 ? pb.R - 1 : r - 1;
        const int rt = cc + 1 == pb.Q ? 0 : cc + 1, lf = cc == 0 ? pb.Q - 1 : cc - 1;
        const H *hl = Hc + (size_t)l * pb.N;
        const double *ml = mu + (size_t)l * pb.N;
        const double e = (double)hl[rc] - ml[rc];
        const double nb = ((double)hl[up * pb.Q + cc] - ml[up * pb.Q + cc]) +
                          ((double)hl[dn * pb.Q + cc] - ml[dn * pb.Q + cc]) +
                          ((double)hl[r * pb.Q + rt] - ml[r * pb.Q + rt]) +
                          ((double)hl[r * pb.Q + lf] - ml[r * pb.Q + lf]);
        const double gl = (double)(long long)gacc[(size_t)c * n + i] * kInvFix;
        grad[(size_t)c * n + i] = gl - pb.tau * (4.0 * e - pb.car_r * nb);
    }
}

cudaError_t launch_grad_finish(const Prob &pb, int mode, HRef h, const double *mu, int n_chains,
                               const unsigned long long *gacc, double *grad, cudaStream_t st)
{
    const int n = pb.L * pb.N;
    dim3 grid((n + 255) / 256 < 256 ? (n + 255) / 256 : 256, n_chains);
    if (mode == MODE_F64) k_grad_finish<double><<<grid, 256, 0, st>>>(pb, h, mu, gacc, grad);
    else k_grad_finish<float><<<grid, 256, 0, st>>>(pb, h, mu, gacc, grad);
    return cudaGetLastError();
}

// Gradient of proposals (heights selected by h) into G[1 - cur[c]] of [2][C][n].
template <typename H>
__global__ void k_grad_finish_sel(Prob pb, HRef h, const double *mu, const unsigned long long *gacc,
                                  double *G, const uint8_t *cur, int n_chains)
{
    const int c = blockIdx.y;
    const int n = pb.L * pb.N;
    double *dst = G + ((size_t)(1 - cur[c]) * n_chains + c) * n;
    const H *Hc = chain_ptr<H>(h, c);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int l = i / pb.N, rc = i - l * pb.N, r = rc / pb.Q, cc = rc - r * pb.Q;
        const int up = r + 1 == pb.R ? 0 : r + 1, dn = r == 0 ? pb.R - 1 : r - 1;
        const int rt = cc + 1 == pb.Q ? 0 : cc + 1, lf = cc == 0 ? pb.Q - 1 : cc - 1;
        const H *hl = Hc + (size_t)l * pb.N;
        const double *ml = mu + (size_t)l * pb.N;
        const double e = (double)hl[rc] - ml[rc];
        const double nb = ((double)hl[up * pb.Q + cc] - ml[up * pb.Q + cc]) +
                          ((double)hl[dn * pb.Q + cc] - ml[dn * pb.Q + cc]) +
                          ((double)hl[r * pb.Q + rt] - ml[r * pb.Q + rt]) +
                          ((double)hl[r * pb.Q + lf] - ml[r * pb.Q + lf]);
        const double gl = (double)(long long)gacc[(size_t)c * n + i] * kInvFix;
        dst[i] = gl - pb.tau * (4.0 * e - pb.car_r * nb);
    }
}

cudaError_t launch_grad_finish_sel(const Prob &pb, int mode, HRef h, const double *mu, int n_chains,
                                   const unsigned long long *gacc, double *G, const uint8_t *cur,
                                   cudaStream_t st)
{
    const int n = pb.L * pb.N;
    dim3 grid((n + 255) / 256 < 256 ? (n + 255) / 256 : 256, n_chains);
    if (mode == MODE_F64) k_grad_finish_sel<double><<<grid, 256, 0, st>>>(pb, h, mu, gacc, G, cur, n_chains);
    else k_grad_finish_sel<float><<<grid, 256, 0, st>>>(pb, h, mu, gacc, G, cur, n_chains);
    return cudaGetLastError();
}

// src [C][n] -> G[cur[c]][c] of [2][C][n].
__global__ void k_scatter_sel(int n_chains, long long n, const double *src, const uint8_t *cur, double *G)
{
    const int c = blockIdx.y;
    double *dst = G + ((size_t)cur[c] * n_chains + c) * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[(size_t)c * n + i];
}

cudaError_t launch_scatter_sel(int n_chains, long long n, const double *src, const uint8_t *cur,
                               double *G, cudaStream_t st)
{
    dim3 grid((unsigned)((n + 255) / 256 < 256 ? (n + 255) / 256 : 256), n_chains);
    k_scatter_sel<<<grid, 256, 0, st>>>(n_chains, n, src, cur, G);
    return cudaGetLastError();
}

__global__ void k_add(int n, const double *a, const double *b, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] + b[i];
}

cudaError_t launch_add(int n, const double *a, const double *b, double *out, cudaStream_t st)
{
    k_add<<<(n + 255) / 256, 256, 0, st>>>(n, a, b, out);
    return cudaGetLastError();
}

}  // namespace mt
