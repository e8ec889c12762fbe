// copula.cu -- the paper's copula prior over layer heights (Sec. 2.2.1).
//
// Per chain the state is a latent array laid out like the heights
// [L][R][Q]: planes 0 .. L-2 hold standard-normal fields z_l, the first L-1
// entries of plane L-1 hold the spatial-dependence parameters r_l in (0, 1).
// The heights follow by
//   x_l = Q(r_l)^-1/2 z_l   (Q(r) = 4 I - r A on the periodic 4-neighbour grid,
//                            Eq. def_CAR_precision),
//   u_l = Phi(x_l / sqrt(Sigma_11(r_l)))            (Eq. CAR_cdf_transform),
//   H_l = H_{l-1} + u_l (T - H_{l-1}),  H_{-1} = 0  (Eq. indep_columns with the
//                                                   copula's uniforms),
// and the top surface is the known terrain T.  Q(r)^-1/2 is applied
// spectrally: the periodic grid's Q is diagonalised by the 2-D discrete
// Fourier transform with eigenvalues 4 - 2 r (cos(2 pi k1/R) + cos(2 pi k2/Q)),
// so x = IDFT(DFT(z) / sqrt(eigenvalue)) and Sigma_11 is the mean of the
// inverse eigenvalues.  (The paper draws x with a Cholesky factor of Q; any U
// with U U^T = Q^-1 gives x the same law.)  One CTA per chain: the four
// one-dimensional DFT passes (rows, columns, inverse columns, inverse rows)
// run as direct sums over shared-memory planes with tabulated twiddles.
#include <math.h>

#include "march.cuh"

namespace mt {

template <typename T> __device__ __forceinline__ T phi_cdf(T x);
template <> __device__ __forceinline__ float phi_cdf<float>(float x) { return normcdff(x); }
template <> __device__ __forceinline__ double phi_cdf<double>(double x) { return normcdf(x); }

// smem: re/im planes A, B (4 N values) + cos/sin tables for R and Q + 32 partials
template <typename T>
__global__ void __launch_bounds__(256) k_copula(Prob pb, HRef lat, const T *terrain, T *H)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int R = pb.R, Q = pb.Q, N = pb.N, L = pb.L;
    T *are = reinterpret_cast<T *>(smem_raw), *aim = are + N, *bre = aim + N, *bim = bre + N;
    T *cR = bim + N, *sR = cR + R, *cQ = sR + R, *sQ = cQ + Q;
    T *red = sQ + Q;
    const int c = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const T *z = chain_ptr<T>(lat, c);
    T *Hc = H + (size_t)c * L * N;
    for (int k = tid; k < R; k += nt) {
        double s, co;
        sincospi(2.0 * k / R, &s, &co);
        cR[k] = (T)co;
        sR[k] = (T)s;
    }
    for (int k = tid; k < Q; k += nt) {
        double s, co;
        sincospi(2.0 * k / Q, &s, &co);
        cQ[k] = (T)co;
        sQ[k] = (T)s;
    }
    __syncthreads();
    for (int l = 0; l < L - 1; ++l) {
        const T *zl = z + (size_t)l * N;
        // r outside (0, 1) has log-prior -inf (rejected); clamp so the
        // heights stay finite
        const T r = fmin(fmax(z[(size_t)(L - 1) * N + l], (T)0), (T)0.999999);
        // rows: A[i][k2] = sum_j z[i][j] e^{-2 pi i j k2 / Q}
        for (int idx = tid; idx < N; idx += nt) {
            const int i = idx / Q, k2 = idx - i * Q;
            T sr = 0, si = 0;
            int t = 0;
            for (int j = 0; j < Q; ++j) {
                const T v = zl[i * Q + j];
                sr += v * cQ[t];
                si -= v * sQ[t];
                t += k2;
                if (t >= Q) t -= Q;
            }
            are[idx] = sr;
            aim[idx] = si;
        }
        __syncthreads();
        // columns: B[k1][k2] = sum_i A[i][k2] e^{-2 pi i i k1 / R}, then / sqrt(eigenvalue);
        // each thread also sums 1 / eigenvalue for Sigma_11
        T inv_sum = 0;
        for (int idx = tid; idx < N; idx += nt) {
            const int k1 = idx / Q, k2 = idx - k1 * Q;
            T sr = 0, si = 0;
            int t = 0;
            for (int i = 0; i < R; ++i) {
                const T ar = are[i * Q + k2], ai = aim[i * Q + k2];
                sr += ar * cR[t] + ai * sR[t];
                si += ai * cR[t] - ar * sR[t];
                t += k1;
                if (t >= R) t -= R;
            }
            const T lam = (T)4 - (T)2 * r * (cR[k1] + cQ[k2]);
            const T g = (T)1 / sqrt(lam);
            inv_sum += (T)1 / lam;
            bre[idx] = sr * g;
            bim[idx] = si * g;
        }
        // Sigma_11 (block sum of inv_sum)
        for (int o = 16; o > 0; o >>= 1) inv_sum += __shfl_xor_sync(0xffffffffu, inv_sum, o);
        if ((tid & 31) == 0) red[tid >> 5] = inv_sum;
        __syncthreads();
        T s11 = 0;
        for (int w = 0; w < (nt + 31) / 32; ++w) s11 += red[w];
        s11 /= (T)N;
        // inverse columns: A[i][k2] = sum_k1 B[k1][k2] e^{+2 pi i i k1 / R}
        for (int idx = tid; idx < N; idx += nt) {
            const int i = idx / Q, k2 = idx - i * Q;
            T sr = 0, si = 0;
            int t = 0;
            for (int k1 = 0; k1 < R; ++k1) {
                const T br = bre[k1 * Q + k2], bi = bim[k1 * Q + k2];
                sr += br * cR[t] - bi * sR[t];
                si += bi * cR[t] + br * sR[t];
                t += i;
                if (t >= R) t -= R;
            }
            are[idx] = sr;
            aim[idx] = si;
        }
        __syncthreads();
        // inverse rows (real part) / N, copula uniform, stick-breaking
        const T scale = (T)1 / ((T)N * sqrt(s11));
        for (int idx = tid; idx < N; idx += nt) {
            const int i = idx / Q, j = idx - i * Q;
            T sr = 0;
            int t = 0;
            for (int k2 = 0; k2 < Q; ++k2) {
                sr += are[i * Q + k2] * cQ[t] - aim[i * Q + k2] * sQ[t];
                t += j;
                if (t >= Q) t -= Q;
            }
            const T u = phi_cdf<T>(sr * scale);
            const T below = l > 0 ? Hc[(size_t)(l - 1) * N + idx] : (T)0;
            Hc[(size_t)l * N + idx] = below + u * (terrain[idx] - below);
        }
        __syncthreads();
    }
    for (int idx = tid; idx < N; idx += nt) Hc[(size_t)(L - 1) * N + idx] = terrain[idx];
}

size_t copula_smem_bytes(const Prob &pb, int mode)
{
    const size_t es = mode == MODE_F64 ? 8 : 4;
    return es * (4 * (size_t)pb.N + 2 * (size_t)(pb.R + pb.Q) + 32);
}

cudaError_t launch_copula(const Prob &pb, int mode, HRef lat, const void *terrain, void *H, int n_chains,
                          cudaStream_t st)
{
    const size_t smem = copula_smem_bytes(pb, mode);
    cudaError_t e;
    if (mode == MODE_F64) {
        static size_t set = 0;
        if (smem > 48 * 1024 && smem > set) {
            e = cudaFuncSetAttribute(k_copula<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            set = smem;
        }
        k_copula<double><<<n_chains, 256, smem, st>>>(pb, lat, (const double *)terrain, (double *)H);
    } else {
        static size_t set = 0;
        if (smem > 48 * 1024 && smem > set) {
            e = cudaFuncSetAttribute(k_copula<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            set = smem;
        }
        k_copula<float><<<n_chains, 256, smem, st>>>(pb, lat, (const float *)terrain, (float *)H);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- reverse pass
// Gradient with respect to the latents of the log-posterior, given the
// log-likelihood gradient with respect to the heights (the adjoint's
// fixed-point accumulators, units 2^-24): the chain rule through the
// stick-breaking H_l = (1 - u_l) H_{l-1} + u_l T (surfaces in reverse order,
// carrying a = d/dH_l of everything above), u = Phi(s), s = x / sqrt(S(r)),
// x = F^-1 (F z / sqrt(lambda(r))) (symmetric: the z gradient is the filtered
// x gradient), plus r through lambda (d lambda^-1/2 / dr = c lambda^-3/2 with
// c_k = cos 2 pi k1/R + cos 2 pi k2/Q) and through S (dS/dr = mean 2 c /
// lambda^2), plus the latent log-prior's -z.  One CTA per chain; the heights
// H_{l-1} come from the forward transform's output.  Writes the gradient
// [L][R][Q] (r gradients in the first L-1 entries of plane L-1, the rest of
// that plane 0) to G[1 - cur[c]][c] (cur != nullptr) or G[c].
template <typename T>
__global__ void __launch_bounds__(256)
k_copula_vjp(Prob pb, HRef lat, HRef hts, const T *terrain, const unsigned long long *gacc, double *G,
             const uint8_t *cur, int n_chains)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int R = pb.R, Q = pb.Q, N = pb.N, L = pb.L;
    T *are = reinterpret_cast<T *>(smem_raw), *aim = are + N, *bre = aim + N, *bim = bre + N;
    T *zre = bim + N, *zim = zre + N, *acar = zim + N;
    T *cR = acar + N, *sR = cR + R, *cQ = sR + R, *sQ = cQ + Q;
    __shared__ double red[3][32];
    const int c = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = (nt + 31) >> 5;
    const T *z = chain_ptr<T>(lat, c);
    const T *Hc = chain_ptr<T>(hts, c);
    const unsigned long long *ga = gacc + (size_t)c * L * N;
    double *dst = G + (cur ? ((size_t)(1 - cur[c]) * n_chains + c) : (size_t)c) * (size_t)L * N;
    auto block3 = [&](double &v0, double &v1, double &v2) {  // block sums, valid in every thread
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v0 += __shfl_xor_sync(0xffffffffu, v0, o);
            v1 += __shfl_xor_sync(0xffffffffu, v1, o);
            v2 += __shfl_xor_sync(0xffffffffu, v2, o);
        }
        __syncthreads();
        if (lane == 0) {
            red[0][warp] = v0;
            red[1][warp] = v1;
            red[2][warp] = v2;
        }
        __syncthreads();
        v0 = v1 = v2 = 0.0;
        for (int w = 0; w < nw; ++w) {
            v0 += red[0][w];
            v1 += red[1][w];
            v2 += red[2][w];
        }
    };
    for (int k = tid; k < R; k += nt) {
        double s, co;
        sincospi(2.0 * k / R, &s, &co);
        cR[k] = (T)co;
        sR[k] = (T)s;
    }
    for (int k = tid; k < Q; k += nt) {
        double s, co;
        sincospi(2.0 * k / Q, &s, &co);
        cQ[k] = (T)co;
        sQ[k] = (T)s;
    }
    for (int i = tid; i < N; i += nt) {
        acar[i] = (T)0;
        dst[(size_t)(L - 1) * N + i] = 0.0;
    }
    __syncthreads();
    const T inv_fix = (T)(1.0 / 16777216.0);
    for (int l = L - 2; l >= 0; --l) {
        const T *zl = z + (size_t)l * N;
        const T r = fmin(fmax(z[(size_t)(L - 1) * N + l], (T)0), (T)0.999999);
        // x = Q(r)^-1/2 z_l as in the forward transform, keeping F z
        for (int idx = tid; idx < N; idx += nt) {
            const int i = idx / Q, k2 = idx - i * Q;
            T sr = 0, si = 0;
            int t = 0;
            for (int j = 0; j < Q; ++j) {
                const T v = zl[i * Q + j];
                sr += v * cQ[t];
                si -= v * sQ[t];
                t += k2;
                if (t >= Q) t -= Q;
            }
            are[idx] = sr;
            aim[idx] = si;
        }
        __syncthreads();
        double inv_sum = 0.0, d_s = 0.0, unused = 0.0;
        for (int idx = tid; idx < N; idx += nt) {
            const int k1 = idx / Q, k2 = idx - k1 * Q;
            T sr = 0, si = 0;
            int t = 0;
            for (int i = 0; i < R; ++i) {
                const T ar = are[i * Q + k2], ai = aim[i * Q + k2];
                sr += ar * cR[t] + ai * sR[t];
                si += ai * cR[t] - ar * sR[t];
                t += k1;
                if (t >= R) t -= R;
            }
            const T ck = cR[k1] + cQ[k2];
            const T lam = (T)4 - (T)2 * r * ck;
            const T g = (T)1 / sqrt(lam);
            inv_sum += (double)((T)1 / lam);
            d_s += 2.0 * (double)ck / ((double)lam * (double)lam);
            zre[idx] = sr;
            zim[idx] = si;
            bre[idx] = sr * g;
            bim[idx] = si * g;
        }
        block3(inv_sum, d_s, unused);
        const double S = inv_sum / N, dS = d_s / N;
        for (int idx = tid; idx < N; idx += nt) {
            const int i = idx / Q, k2 = idx - i * Q;
            T sr = 0, si = 0;
            int t = 0;
            for (int k1 = 0; k1 < R; ++k1) {
                const T br = bre[k1 * Q + k2], bi = bim[k1 * Q + k2];
                sr += br * cR[t] - bi * sR[t];
                si += bi * cR[t] + br * sR[t];
                t += i;
                if (t >= R) t -= R;
            }
            are[idx] = sr;
            aim[idx] = si;
        }
        __syncthreads();
        // s, u and the reverse steps through the stick-breaking and Phi; the x
        // gradient goes to bre (real plane)
        const T scale = (T)(1.0 / ((double)N * sqrt(S))), rs = (T)(1.0 / sqrt(S));
        double gss = 0.0;
        for (int idx = tid; idx < N; idx += nt) {
            const int i = idx / Q, j = idx - i * Q;
            T sr = 0;
            int t = 0;
            for (int k2 = 0; k2 < Q; ++k2) {
                sr += are[i * Q + k2] * cQ[t] - aim[i * Q + k2] * sQ[t];
                t += j;
                if (t >= Q) t -= Q;
            }
            const T sv = sr * scale;
            const T u = phi_cdf<T>(sv);
            const T below = l > 0 ? Hc[(size_t)(l - 1) * N + idx] : (T)0;
            const T gH = (T)(long long)ga[(size_t)l * N + idx] * inv_fix;
            const T a = acar[idx] + gH;
            const T gu = a * (terrain[idx] - below);
            acar[idx] = a * ((T)1 - u);
            const T gs = gu * (T)0.3989422804014327 * exp(-(T)0.5 * sv * sv);
            gss += (double)gs * (double)sv;
            bre[idx] = gs * rs;
        }
        block3(gss, unused, unused);  // also makes bre visible
        // z gradient = filtered x gradient; r gradient through the filter
        for (int idx = tid; idx < N; idx += nt) {
            const int i = idx / Q, k2 = idx - i * Q;
            T sr = 0, si = 0;
            int t = 0;
            for (int j = 0; j < Q; ++j) {
                const T v = bre[i * Q + j];
                sr += v * cQ[t];
                si -= v * sQ[t];
                t += k2;
                if (t >= Q) t -= Q;
            }
            are[idx] = sr;
            aim[idx] = si;
        }
        __syncthreads();
        double grx = 0.0;
        for (int idx = tid; idx < N; idx += nt) {
            const int k1 = idx / Q, k2 = idx - k1 * Q;
            T sr = 0, si = 0;
            int t = 0;
            for (int i = 0; i < R; ++i) {
                const T ar = are[i * Q + k2], ai = aim[i * Q + k2];
                sr += ar * cR[t] + ai * sR[t];
                si += ai * cR[t] - ar * sR[t];
                t += k1;
                if (t >= R) t -= R;
            }
            const T ck = cR[k1] + cQ[k2];
            const T lam = (T)4 - (T)2 * r * ck;
            const T g = (T)1 / sqrt(lam);
            grx += ((double)sr * (double)zre[idx] + (double)si * (double)zim[idx]) * (double)(ck * g / lam);
            bre[idx] = sr * g;
            bim[idx] = si * g;
        }
        block3(grx, unused, unused);  // also makes bre / bim visible
        for (int idx = tid; idx < N; idx += nt) {
            const int i = idx / Q, k2 = idx - i * Q;
            T sr = 0, si = 0;
            int t = 0;
            for (int k1 = 0; k1 < R; ++k1) {
                const T br = bre[k1 * Q + k2], bi = bim[k1 * Q + k2];
                sr += br * cR[t] - bi * sR[t];
                si += bi * cR[t] + br * sR[t];
                t += i;
                if (t >= R) t -= R;
            }
            are[idx] = sr;
            aim[idx] = si;
        }
        __syncthreads();
        const T inv_n = (T)(1.0 / N);
        for (int idx = tid; idx < N; idx += nt) {
            const int i = idx / Q, j = idx - i * Q;
            T sr = 0;
            int t = 0;
            for (int k2 = 0; k2 < Q; ++k2) {
                sr += are[i * Q + k2] * cQ[t] - aim[i * Q + k2] * sQ[t];
                t += j;
                if (t >= Q) t -= Q;
            }
            dst[(size_t)l * N + idx] = (double)(sr * inv_n) - (double)zl[idx];  // + latent prior
        }
        if (tid == 0) dst[(size_t)(L - 1) * N + l] = grx / N - 0.5 * gss / S * dS;
        __syncthreads();
    }
}

size_t copula_vjp_smem_bytes(const Prob &pb)
{
    return 4 * (7 * (size_t)pb.N + 2 * (size_t)(pb.R + pb.Q));
}

cudaError_t launch_copula_vjp(const Prob &pb, HRef lat, HRef hts, const void *terrain,
                              const unsigned long long *gacc, double *G, const uint8_t *cur, int n_chains,
                              cudaStream_t st)
{
    const size_t smem = copula_vjp_smem_bytes(pb);
    static size_t set = 0;
    if (smem > 48 * 1024 && smem > set) {
        cudaError_t e = cudaFuncSetAttribute(k_copula_vjp<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        set = smem;
    }
    k_copula_vjp<float><<<n_chains, 256, smem, st>>>(pb, lat, hts, (const float *)terrain, gacc, G, cur,
                                                     n_chains);
    return cudaGetLastError();
}

// Latent log-prior: -1/2 sum z^2 over planes 0 .. L-2 (FP64 sum), -inf unless
// every r_l lies in (0, 1).  One block per chain.
template <typename T>
__global__ void __launch_bounds__(256) k_prior_latent(Prob pb, HRef lat, double *lp_out)
{
    const int c = blockIdx.x;
    const T *z = chain_ptr<T>(lat, c);
    const int n = (pb.L - 1) * pb.N;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = (double)z[i];
        s = fma(v, v, s);
    }
    int bad = 0;
    if ((int)threadIdx.x < pb.L - 1) {
        const T r = z[(size_t)(pb.L - 1) * pb.N + threadIdx.x];
        if (!(r > (T)0 && r < (T)1)) bad = 1;
    }
    s = block_sum(s);
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) lp_out[c] = bad ? -INFINITY : -0.5 * s;
}

cudaError_t launch_prior_latent(const Prob &pb, int mode, HRef lat, int n_chains, double *lp_out,
                                cudaStream_t st)
{
    if (mode == MODE_F64) k_prior_latent<double><<<n_chains, 256, 0, st>>>(pb, lat, lp_out);
    else k_prior_latent<float><<<n_chains, 256, 0, st>>>(pb, lat, lp_out);
    return cudaGetLastError();
}

}  // namespace mt
