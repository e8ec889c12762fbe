// linear.cu -- the paper's linearised forward model (Sec. 2.1.2, Eqs.
// expected_counts_linearized / _approx) on the voxel density grid of
// Sec. 2.1.4 (Eq. def_LM_density_grid_smooth).
//
// Voxels: the (R-1) x (Q-1) cells of the surface grid times n_z levels of
// height dz = Lz / n_z, flat index v = (k ny + i) nx + j.  Density at the
// voxel centre: R_v = rho_top + sum_l (rho_l - rho_{l+1}) varsigma(h_l - z_k),
// h_l = mean of the cell's four corner heights, z_k = (k + 1/2) dz.
// L_pv = length of ray p inside voxel v (its in-box segment), a sparse
// matrix in CSR by ray, built once on the host in FP64.  With lambda0_p =
// I0 exp(-O_p(R0) / Lambda) at the reference density R0 = R(H_ref):
//   lambda_hat_p(R) = lambda0_p (1 - sum_v L_pv (R_v - R0_v) / Lambda).
// Per evaluation: k_lin_density writes dR = R - R0 for every voxel and
// chain, [v][chain] (chains fastest, padded to 32), as differences of the
// indicators; k_lin_ll gives each warp
// one ray at a time for 32 chains (lane = chain), sums L_pv dR_v over the
// ray's voxels and adds the Poisson term, C (ln(lambda_hat / C) - (lambda_hat
// - C) / C) = -C (x - log1p(x)), x = (lambda_hat - C) / C, or -lambda_hat
// for C = 0 (-inf where lambda_hat <= 0).
#include <math.h>

#include <algorithm>
#include <vector>

#include "march.cuh"

namespace mt {

// ---------------------------------------------------------------- host
static double slab_exit(const double o[3], const double d[3], const double box[3])
{
    double te = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double ta = INFINITY;
        if (d[a] > 0.0) ta = (box[a] - o[a]) / d[a];
        else if (d[a] < 0.0) ta = (0.0 - o[a]) / d[a];
        te = fmin(te, ta);
    }
    return te;
}

// Voxel path lengths of every ray (ray = s * P + p), appended in CSR order.
void lin_build_lengths(const Prob &pb, const std::vector<double> &sensors,
                       const std::vector<double> &dirs, int nz, std::vector<int> &row,
                       std::vector<int> &col, std::vector<double> &val)
{
    const int nx = pb.Q - 1, ny = pb.R - 1;
    const int n[3] = {nx, ny, nz};
    const double h[3] = {pb.box[0] / nx, pb.box[1] / ny, pb.box[2] / nz};
    row.assign(1, 0);
    col.clear();
    val.clear();
    std::vector<double> ts;
    std::vector<std::pair<int, double>> seg;
    for (int s = 0; s < pb.S; ++s)
        for (int p = 0; p < pb.P; ++p) {
            const double *o = &sensors[3 * s], *d = &dirs[3 * p];
            const double te = slab_exit(o, d, pb.box);
            ts.assign({0.0, te});
            for (int a = 0; a < 3; ++a)
                if (d[a] != 0.0)
                    for (int b = 0; b <= n[a]; ++b) {
                        const double t = (b * h[a] - o[a]) / d[a];
                        if (t > 0.0 && t < te) ts.push_back(t);
                    }
            std::sort(ts.begin(), ts.end());
            seg.clear();
            for (size_t q = 0; q + 1 < ts.size(); ++q) {
                const double t0 = ts[q], t1 = ts[q + 1];
                if (!(t1 > t0)) continue;
                const double tm = 0.5 * (t0 + t1);
                const int j = std::min((int)((o[0] + tm * d[0]) / h[0]), nx - 1);
                const int i = std::min((int)((o[1] + tm * d[1]) / h[1]), ny - 1);
                const int k = std::min((int)((o[2] + tm * d[2]) / h[2]), nz - 1);
                seg.push_back({(k * ny + std::max(i, 0)) * nx + std::max(j, 0), t1 - t0});
            }
            std::sort(seg.begin(), seg.end());
            for (size_t q = 0; q < seg.size(); ++q) {
                if (q > 0 && seg[q].first == seg[q - 1].first) {
                    val.back() += seg[q].second;  // the same voxel entered twice (a grazing edge)
                } else {
                    col.push_back(seg[q].first);
                    val.push_back(seg[q].second);
                }
            }
            row.push_back((int)col.size());
        }
}

// Voxel densities of heights H [L][R][Q] (FP64).
void lin_density_host(const Prob &pb, const double *H, int nz, std::vector<double> &R)
{
    const int nx = pb.Q - 1, ny = pb.R - 1, Q = pb.Q, N = pb.N;
    R.assign((size_t)nz * ny * nx, pb.rho_top);
    const double dz = pb.box[2] / nz;
    for (int i = 0; i < ny; ++i)
        for (int j = 0; j < nx; ++j)
            for (int l = 0; l < pb.L; ++l) {
                const double *h = H + (size_t)l * N;
                const double hc = 0.25 * (h[i * Q + j] + h[i * Q + j + 1] + h[(i + 1) * Q + j] + h[(i + 1) * Q + j + 1]);
                for (int k = 0; k < nz; ++k) {
                    const double u = hc - (k + 0.5) * dz;
                    const double s = pb.gamma == 0.0 ? (u > 0 ? 1.0 : (u < 0 ? 0.0 : 0.5))
                                                     : 1.0 / (1.0 + exp(-u / pb.gamma));
                    R[((size_t)k * ny + i) * nx + j] += pb.drho[l] * s;
                }
            }
}

// ---------------------------------------------------------------- device
template <typename T> __device__ __forceinline__ T eta(T u) { return u > (T)0 ? (T)1 : (u < (T)0 ? (T)0 : (T)0.5); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }

// Voxel densities R_v(H_c) - R0_v of n_chains heights, [v][chain] (chains
// fastest, padded to Cp); with R0 == nullptr the densities themselves (used
// once for the reference, so that R and R0 come from the same arithmetic and
// dR is exactly 0 at the reference).  Threads = 32 chains x 8 cells per
// block, cells along x.
template <typename T>
__global__ void __launch_bounds__(256) k_lin_density(Prob pb, HRef h, int n_chains, int Cp, int nz,
                                                     const T *R0, T *dR)
{
    const int lane = threadIdx.x & 31, cw = threadIdx.x >> 5;
    const int nx = pb.Q - 1, ny = pb.R - 1;
    const int colv = blockIdx.x * 8 + cw;  // cell index i * nx + j
    const int c = blockIdx.y * 32 + lane;
    if (colv >= nx * ny || c >= Cp) return;  // the reference launch has Cp = 1
    const int i = colv / nx, j = colv - i * nx;
    const size_t ncell = (size_t)nx * ny;
    if (c >= n_chains) {
        for (int k = 0; k < nz; ++k) dR[((size_t)k * ncell + colv) * Cp + c] = (T)0;
        return;
    }
    const T *Hc = chain_ptr<T>(h, c);
    T hc[MT_MAX_L], dr[MT_MAX_L];
#pragma unroll
    for (int l = 0; l < MT_MAX_L; ++l) {
        if (l < pb.L) {
            const T *hl = Hc + (size_t)l * pb.N;
            hc[l] = (T)0.25 * (((hl[i * pb.Q + j] + hl[i * pb.Q + j + 1]) + hl[(i + 1) * pb.Q + j]) + hl[(i + 1) * pb.Q + j + 1]);
            dr[l] = (T)pb.drho[l];
        }
    }
    const T dz = (T)(pb.box[2] / nz), inv_g = pb.gamma > 0.0 ? (T)(1.0 / pb.gamma) : (T)0;
    const T rtop = (T)pb.rho_top;
    const bool hard = pb.gamma == 0.0;
    for (int k = 0; k < nz; ++k) {
        // z_k and h - z_k each rounded on their own (no fused multiply-add):
        // a surface exactly at a voxel centre gives u = 0 and the hard
        // indicator its midpoint value, as in the host's reference densities
        const T z = mul_rn((T)k + (T)0.5, dz);
        T r = rtop;
#pragma unroll
        for (int l = 0; l < MT_MAX_L; ++l) {
            if (l < pb.L) {
                const T u = sub_rn(hc[l], z);
                T sg;
                if (hard) sg = eta<T>(u);
                else if constexpr (sizeof(T) == 4) sg = __frcp_rn(1.0f + expf(-u * inv_g));
                else sg = 1.0 / (1.0 + exp(-u * inv_g));
                r += dr[l] * sg;
            }
        }
        const size_t v = (size_t)k * ncell + colv;
        dR[v * Cp + c] = R0 ? r - R0[v] : r;
    }
}

// x - log1p(x) without cancellation for small |x| (its series x^2/2 - x^3/3
// + x^4/4 - ...).
template <typename T> __device__ __forceinline__ T x_minus_log1p(T x)
{
    // |x| < 1/8: the series to x^11 (FP32) or x^22 (FP64) leaves less than
    // 8^-9 (resp. 8^-20) of x^2/2
    constexpr int NT = sizeof(T) == 4 ? 11 : 22;
    if (fabs(x) < (T)0.125) {
        T t = x, s = (T)0;
#pragma unroll
        for (int n = 2; n <= NT; ++n) {
            t *= x;
            s += ((n & 1) ? -t : t) * ((T)1 / (T)n);
        }
        return s;
    }
    return x - log1p(x);
}

// One warp = one ray at a time for 32 chains (lane = chain); a CTA = its 32
// warps over the block's rays for one tile of 32 chains.  Blocks are small
// and the grid runs ray blocks fastest, so the CTAs in flight work on one
// chain tile and their gathers hit L2.  Per chain the CTA's terms are
// summed (float-float for FP32, FP64 for F64) and written as
// partial[c][block]; -inf if any of them had lambda_hat <= 0.
template <typename T>
__global__ void __launch_bounds__(1024) k_lin_ll(Prob pb, int n_chains, int Cp, int rays_per_block, int nvox,
                                                 const int *row, const int *col, const T *val,
                                                 const T *dR, const double *lam0, const double *amc,
                                                 double *partial, T *fO)
{
    __shared__ double red[32][33];
    __shared__ int bad[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int c = blockIdx.y * 32 + lane;
    if (threadIdx.x < 32) bad[threadIdx.x] = 0;
    __syncthreads();
    const int r_begin = blockIdx.x * rays_per_block;
    const int r_end = min(r_begin + rays_per_block, pb.n_rays);
    const T invL = (T)pb.inv_Lambda;
    double acc_d = 0.0;
    FF acc_f = {0.f, 0.f};
    int neg = 0;
    for (int p = r_begin + wid; p < r_end; p += nw) {
        T dO = (T)0;
        int e1 = row[p + 1];
        int e = row[p];
#ifdef MT_BOUNDS_CHECK
        for (int q = row[p]; q < e1; ++q)
            if ((unsigned)col[q] >= (unsigned)nvox) {
                atomicOr(pb.flag, 4);
                e1 = row[p];  // skip the ray's gathers
                break;
            }
#endif
        for (; e + 4 <= e1; e += 4) {  // four gathers in flight
            const T d0 = dR[(size_t)col[e] * Cp + c], d1 = dR[(size_t)col[e + 1] * Cp + c];
            const T d2 = dR[(size_t)col[e + 2] * Cp + c], d3 = dR[(size_t)col[e + 3] * Cp + c];
            dO += val[e] * d0;
            dO += val[e + 1] * d1;
            dO += val[e + 2] * d2;
            dO += val[e + 3] * d3;
        }
        for (; e < e1; ++e) dO += val[e] * dR[(size_t)col[e] * Cp + c];
        const int Cn = pb.cnt[p];
        const T l0 = (T)lam0[p];
        const T lh = l0 * ((T)1 - dO * invL);
        neg |= !(lh > (T)0);
        // d ll / d O_p = (C / lambda_hat - 1) (-lambda0 / Lambda), for gradients
        if (fO) fO[(size_t)p * Cp + c] = lh > (T)0 ? ((T)Cn / lh - (T)1) * (-l0 * invL) : (T)0;
        T term;
        if (Cn > 0) {
            const T x = ((T)amc[p] - l0 * dO * invL) / (T)Cn;  // (lambda_hat - C) / C
            term = -(T)Cn * x_minus_log1p<T>(x);
        } else {
            term = -lh;
        }
        if constexpr (sizeof(T) == 8) acc_d += (double)term;
        else acc_f = ff_add(acc_f, FF{(float)term, 0.f});
    }
    red[wid][lane] = sizeof(T) == 8 ? acc_d : (double)acc_f.hi + (double)acc_f.lo;
    if (neg) atomicOr(&bad[lane], 1);
    __syncthreads();
    if (wid == 0 && c < n_chains) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += red[w][lane];
        partial[(size_t)c * gridDim.x + blockIdx.x] = bad[lane] ? -INFINITY : s;
    }
}

// part[c][b] = sum of the f consecutive fine partials of block b, in order.
__global__ void k_lin_fold(int n_chains, int n_fine, int n_blk, int f, const double *fine, double *part)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_chains * n_blk) return;
    const int c = idx / n_blk, b = idx - c * n_blk;
    double s = 0.0;
    for (int q = b * f; q < min((b + 1) * f, n_fine); ++q) s += fine[(size_t)c * n_fine + q];
    part[(size_t)c * n_blk + b] = s;
}

__global__ void k_lin_amc(int n, const double *lam0, const int32_t *cnt, double *amc)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) amc[p] = lam0[p] - (double)cnt[p];
}

cudaError_t launch_lin_amc(int n, const double *lam0, const int32_t *cnt, double *amc, cudaStream_t st)
{
    k_lin_amc<<<(n + 255) / 256, 256, 0, st>>>(n, lam0, cnt, amc);
    return cudaGetLastError();
}

// rays per k_lin_ll block (divides the march's ray slots per CTA): two per warp, so that
// one 32-chain tile fills the GPU and the CTAs in flight share its dR in L2
constexpr int kLinRays = 64;

size_t lin_fine_partials(const Prob &pb, int n_chains)
{
    return (size_t)n_chains * ((pb.n_rays + kLinRays - 1) / kLinRays);
}

cudaError_t launch_lin_reference(const Prob &pb, int mode, HRef h, int nz, void *R0, cudaStream_t st)
{
    const int ncol = (pb.Q - 1) * (pb.R - 1);
    dim3 gd((ncol + 7) / 8, 1);
    if (mode == MODE_F64) k_lin_density<double><<<gd, 256, 0, st>>>(pb, h, 1, 1, nz, nullptr, (double *)R0);
    else k_lin_density<float><<<gd, 256, 0, st>>>(pb, h, 1, 1, nz, nullptr, (float *)R0);
    return cudaGetLastError();
}

cudaError_t launch_lin(const Prob &pb, int mode, HRef h, int n_chains, int nz, const int *row,
                       const int *col, const void *val, const void *R0, void *dR, const double *lam0,
                       const double *amc, double *fine, double *partial, cudaStream_t st, void *fO)
{
    const int Cp = (n_chains + 31) / 32 * 32;
    const int ncol = (pb.Q - 1) * (pb.R - 1);
    dim3 gd((ncol + 7) / 8, Cp / 32);
    const int n_fine = (pb.n_rays + kLinRays - 1) / kLinRays;
    dim3 gl(n_fine, Cp / 32);
    if (mode == MODE_F64) {
        k_lin_density<double><<<gd, 256, 0, st>>>(pb, h, n_chains, Cp, nz, (const double *)R0, (double *)dR);
        k_lin_ll<double><<<gl, 1024, 0, st>>>(pb, n_chains, Cp, kLinRays, nz * ncol, row, col, (const double *)val,
                                              (const double *)dR, lam0, amc, fine, (double *)fO);
    } else {
        k_lin_density<float><<<gd, 256, 0, st>>>(pb, h, n_chains, Cp, nz, (const float *)R0, (float *)dR);
        k_lin_ll<float><<<gl, 1024, 0, st>>>(pb, n_chains, Cp, kLinRays, nz * ncol, row, col, (const float *)val,
                                             (const float *)dR, lam0, amc, fine, (float *)fO);
    }
    const int rpb = march_rays_per_block(pb);
    const int n_blk = (pb.n_rays + rpb - 1) / rpb;
    const int f = (rpb + kLinRays - 1) / kLinRays;
    k_lin_fold<<<(n_chains * n_blk + 255) / 256, 256, 0, st>>>(n_chains, n_fine, n_blk, f, fine, partial);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- gradient
// Gradient of the linearised log-likelihood with respect to the node heights
// (gamma > 0), written as the adjoint's 64-bit fixed-point accumulators
// (units 2^-24) so that the prior's gradient and the copula's reverse pass
// follow unchanged:
//   d ll / d R_v = sum_p L_pv d ll / d O_p          (k_lin_rgrad, the path
//                                                     lengths by voxel, CSC)
//   d ll / d h_l(cell) = sum_k (d ll / d R_v) (rho_l - rho_{l+1})
//                        varsigma(u) (1 - varsigma(u)) / gamma,
//                        u = h_l(cell) - z_k          (k_lin_cellgrad)
//   d ll / d H_l(node) = sum over the node's cells of d ll / d h_l(cell) / 4
//                                                     (k_lin_nodegrad)
// Lanes are chains (tiles of 32, padded to Cp); every output has one writer.
template <typename T>
__global__ void __launch_bounds__(256) k_lin_rgrad(int nvox, int Cp, const int *cptr, const int *crow,
                                                   const T *cval, const T *fO, T *gR)
{
    const int lane = threadIdx.x & 31, v = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int c = blockIdx.y * 32 + lane;
    if (v >= nvox) return;
    T s = (T)0;
    for (int e = cptr[v]; e < cptr[v + 1]; ++e) s += cval[e] * fO[(size_t)crow[e] * Cp + c];
    gR[(size_t)v * Cp + c] = s;
}

template <typename T>
__global__ void __launch_bounds__(256) k_lin_cellgrad(Prob pb, HRef h, int n_chains, int Cp, int nz, const T *gR,
                                                      T *gcell)
{
    const int lane = threadIdx.x & 31;
    const int nx = pb.Q - 1, ny = pb.R - 1;
    const int colv = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int c = blockIdx.y * 32 + lane;
    if (colv >= nx * ny || c >= n_chains) return;
    const int i = colv / nx, j = colv - i * nx;
    const size_t ncell = (size_t)nx * ny;
    const T *Hc = chain_ptr<T>(h, c);
    const T dz = (T)(pb.box[2] / nz), inv_g = (T)(1.0 / pb.gamma);
    for (int l = 0; l < pb.L; ++l) {
        const T *hl = Hc + (size_t)l * pb.N;
        const T hc = (T)0.25 * (((hl[i * pb.Q + j] + hl[i * pb.Q + j + 1]) + hl[(i + 1) * pb.Q + j]) +
                                hl[(i + 1) * pb.Q + j + 1]);
        const T dr = (T)pb.drho[l];
        T s = (T)0;
        for (int k = 0; k < nz; ++k) {
            const T u = sub_rn(hc, mul_rn((T)k + (T)0.5, dz));
            T sg;
            if constexpr (sizeof(T) == 4) sg = __frcp_rn(1.0f + expf(-u * inv_g));
            else sg = 1.0 / (1.0 + exp(-u * inv_g));
            s += gR[((size_t)k * ncell + colv) * Cp + c] * (sg * ((T)1 - sg));
        }
        gcell[((size_t)l * ncell + colv) * Cp + c] = s * dr * inv_g;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_lin_nodegrad(Prob pb, int n_chains, int Cp, const T *gcell,
                                                      unsigned long long *gacc)
{
    const int lane = threadIdx.x & 31;
    const int node = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int c = blockIdx.y * 32 + lane, l = blockIdx.z;
    if (node >= pb.N || c >= n_chains) return;
    const int nx = pb.Q - 1, ny = pb.R - 1;
    const int r = node / pb.Q, q = node - r * pb.Q;
    const size_t ncell = (size_t)nx * ny;
    double s = 0.0;
    for (int di = -1; di <= 0; ++di)
        for (int dj = -1; dj <= 0; ++dj) {
            const int i = r + di, j = q + dj;
            if (i >= 0 && i < ny && j >= 0 && j < nx)
                s += (double)gcell[((size_t)l * ncell + (size_t)i * nx + j) * Cp + c];
        }
    gacc[((size_t)c * pb.L + l) * pb.N + node] = (unsigned long long)llrint(0.25 * s * 16777216.0);
}

cudaError_t launch_lin_grad(const Prob &pb, int mode, HRef h, int n_chains, int nz, const int *cptr,
                            const int *crow, const void *cval, const void *fO, void *gR, void *gcell,
                            unsigned long long *gacc, cudaStream_t st)
{
    const int Cp = (n_chains + 31) / 32 * 32;
    const int ncol = (pb.Q - 1) * (pb.R - 1), nvox = nz * ncol;
    dim3 gv((nvox + 7) / 8, Cp / 32), gc((ncol + 7) / 8, Cp / 32), gn((pb.N + 7) / 8, Cp / 32, pb.L);
    if (mode == MODE_F64) {
        k_lin_rgrad<double><<<gv, 256, 0, st>>>(nvox, Cp, cptr, crow, (const double *)cval, (const double *)fO,
                                                (double *)gR);
        k_lin_cellgrad<double><<<gc, 256, 0, st>>>(pb, h, n_chains, Cp, nz, (const double *)gR, (double *)gcell);
        k_lin_nodegrad<double><<<gn, 256, 0, st>>>(pb, n_chains, Cp, (const double *)gcell, gacc);
    } else {
        k_lin_rgrad<float><<<gv, 256, 0, st>>>(nvox, Cp, cptr, crow, (const float *)cval, (const float *)fO,
                                               (float *)gR);
        k_lin_cellgrad<float><<<gc, 256, 0, st>>>(pb, h, n_chains, Cp, nz, (const float *)gR, (float *)gcell);
        k_lin_nodegrad<float><<<gn, 256, 0, st>>>(pb, n_chains, Cp, (const float *)gcell, gacc);
    }
    return cudaGetLastError();
}

// The path lengths by voxel (CSC) from the CSR by ray.
void lin_transpose(int n_rays, int nvox, const std::vector<int> &row, const std::vector<int> &col,
                   const std::vector<double> &val, std::vector<int> &cptr, std::vector<int> &crow,
                   std::vector<double> &cval)
{
    cptr.assign((size_t)nvox + 1, 0);
    for (int v : col) cptr[(size_t)v + 1] += 1;
    for (int v = 0; v < nvox; ++v) cptr[(size_t)v + 1] += cptr[v];
    crow.assign(col.size(), 0);
    cval.assign(col.size(), 0.0);
    std::vector<int> fill(cptr.begin(), cptr.end() - 1);
    for (int p = 0; p < n_rays; ++p)
        for (int e = row[p]; e < row[(size_t)p + 1]; ++e) {
            const int k = fill[col[e]]++;
            crow[k] = p;
            cval[k] = val[e];
        }
}

}  // namespace mt
