// diag.cu -- chain diagnostics on the device.
//
// * Nested R-hat (Sec. 3.2: chains grouped into super-chains that share a
//   start; definition of Margossian et al. 2024) of every height over stored
//   draws: per (parameter, super-chain) the super-chain mean and its
//   within-super-chain variance, then per parameter
//   sqrt(1 + B / W) with B the variance of the super-chain means and W the
//   mean within-super-chain variance.  FP64 throughout.
// * Tomographic standard deviation of the below-interface indicators
//   B^l_{ijk}(H) = eta(H_{l,i,j} - k dz), eta(0) = 1/2 (Eq.
//   def_below_interface_indicator; Sec. 4), across samples of H: per surface
//   node a histogram of m(H) = #{k : z_k < H} (and whether H hits a level
//   exactly) over the samples in shared memory, then suffix sums give every
//   level's mean of B and of B^2 exactly (integer counts).
#include <math.h>

#include "internal.h"

namespace mt {

// ---------------------------------------------------------------- nested R-hat
// Pass 1: one thread per (parameter p, super-chain k): sm[k][p] = super-chain
// mean, wk[k][p] = between-chain variance within the super-chain (M > 1)
// plus the mean within-chain variance (N > 1).  draws [N][C][P].
template <typename H>
__global__ void __launch_bounds__(256) k_rhat_super(const H *draws, int N, int C, int P, int K,
                                                    double *sm, double *wk)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (p >= P) return;
    const int M = C / K;
    const size_t sd = (size_t)C * P;  // stride between draws
    const H *x0 = draws + (size_t)k * M * P + p;
    double s = 0.0;
    for (int m = 0; m < M; ++m) {
        double cm = 0.0;
        for (int n = 0; n < N; ++n) cm += (double)x0[(size_t)m * P + n * sd];
        s += cm / N;
    }
    s /= M;
    double bk = 0.0, wn = 0.0;
    for (int m = 0; m < M; ++m) {
        double cm = 0.0;
        for (int n = 0; n < N; ++n) cm += (double)x0[(size_t)m * P + n * sd];
        cm /= N;
        bk += (cm - s) * (cm - s);
        if (N > 1) {
            double v = 0.0;
            for (int n = 0; n < N; ++n) {
                const double d = (double)x0[(size_t)m * P + n * sd] - cm;
                v += d * d;
            }
            wn += v / (N - 1);
        }
    }
    sm[(size_t)k * P + p] = s;
    wk[(size_t)k * P + p] = (M > 1 ? bk / (M - 1) : 0.0) + (N > 1 ? wn / M : 0.0);
}

// Pass 2: one thread per parameter: R-hat and the running maximum (R-hat >= 1,
// so the bit patterns of the doubles order like the values).
__global__ void __launch_bounds__(256) k_rhat_final(const double *sm, const double *wk, int P, int K,
                                                    double *rhat, unsigned long long *max_bits)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    double g = 0.0, w = 0.0;
    for (int k = 0; k < K; ++k) {
        g += sm[(size_t)k * P + p];
        w += wk[(size_t)k * P + p];
    }
    g /= K;
    w /= K;
    double b = 0.0;
    for (int k = 0; k < K; ++k) {
        const double d = sm[(size_t)k * P + p] - g;
        b += d * d;
    }
    b /= (K - 1);
    const double r = w > 0.0 ? sqrt(__dadd_rn(1.0, b / w)) : (b == 0.0 ? 1.0 : INFINITY);
    if (rhat) rhat[p] = r;
    atomicMax(max_bits, (unsigned long long)__double_as_longlong(r));
}

cudaError_t launch_nested_rhat(int mode, const void *draws, int N, int C, int P, int K, double *sm,
                               double *wk, double *rhat, unsigned long long *max_bits, cudaStream_t st)
{
    dim3 g1((P + 255) / 256, K);
    if (mode == MODE_F64) k_rhat_super<double><<<g1, 256, 0, st>>>((const double *)draws, N, C, P, K, sm, wk);
    else k_rhat_super<float><<<g1, 256, 0, st>>>((const float *)draws, N, C, P, K, sm, wk);
    k_rhat_final<<<(P + 255) / 256, 256, 0, st>>>(sm, wk, P, K, rhat, max_bits);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- interface std
// One block = one surface x a tile of TN nodes; threads (node j = t % TN,
// sample lane t / TN) walk the samples.  Shared memory: the n_z levels z_k
// (FP64) and the histogram hist[j][m][tie] (m = 0 .. n_z).
template <typename H>
__global__ void __launch_bounds__(256) k_interface_std(const H *samples, int S, int L, int N, int n_z,
                                                       const double *z, int TN, double *out)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *zs = reinterpret_cast<double *>(smem_raw);
    unsigned int *hist = reinterpret_cast<unsigned int *>(zs + n_z);
    const int l = blockIdx.y, n0 = blockIdx.x * TN;
    const int nb = 2 * (n_z + 1);
    for (int i = threadIdx.x; i < n_z; i += blockDim.x) zs[i] = z[i];
    for (int i = threadIdx.x; i < TN * nb; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    const int j = threadIdx.x % TN, lanes = blockDim.x / TN, lane = threadIdx.x / TN;
    const int node = n0 + j;
    if (node < N && lane < lanes) {
        for (int s = lane; s < S; s += lanes) {
            const double h = (double)samples[((size_t)s * L + l) * N + node];
            int lo = 0, hi = n_z;  // first level with z_k >= h
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (zs[mid] < h) lo = mid + 1;
                else hi = mid;
            }
            const int tie = (lo < n_z && zs[lo] == h) ? 1 : 0;
            atomicAdd(&hist[j * nb + 2 * lo + tie], 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x < TN && n0 + threadIdx.x < N) {
        const int jj = threadIdx.x;
        const unsigned int *hj = hist + jj * nb;
        unsigned long long above = (unsigned long long)hj[2 * n_z] + hj[2 * n_z + 1];  // m > k for k = n_z - 1
        for (int k = n_z - 1; k >= 0; --k) {
            const unsigned long long t = hj[2 * k + 1];
            const double mean = (double)(2 * above + t) / (2.0 * S);
            const double mean2 = (double)(4 * above + t) / (4.0 * S);
            // explicit roundings (no contraction into an FMA): the same
            // operations as the plain definition sqrt(mean(B^2) - mean(B)^2)
            const double var = __dsub_rn(mean2, __dmul_rn(mean, mean));
            out[((size_t)l * n_z + k) * N + n0 + jj] = sqrt(fmax(var, 0.0));
            above += (unsigned long long)hj[2 * k] + hj[2 * k + 1];
        }
    }
}

int interface_tile(int n_z)
{
    int tn = (96 * 1024 - 8 * n_z) / (8 * (n_z + 1));
    return tn < 1 ? 1 : (tn > 32 ? 32 : tn);
}

size_t interface_smem(int n_z) { return (size_t)8 * n_z + (size_t)interface_tile(n_z) * 8 * (n_z + 1); }

cudaError_t launch_interface_std(int mode, const void *samples, int S, int L, int N, int n_z,
                                 const double *z, double *out, cudaStream_t st)
{
    const int tn = interface_tile(n_z);
    const size_t smem = interface_smem(n_z);
    dim3 grid((N + tn - 1) / tn, L);
    cudaError_t e;
    if (mode == MODE_F64) {
        e = cudaFuncSetAttribute(k_interface_std<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_interface_std<double><<<grid, 256, smem, st>>>((const double *)samples, S, L, N, n_z, z, tn, out);
    } else {
        e = cudaFuncSetAttribute(k_interface_std<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_interface_std<float><<<grid, 256, smem, st>>>((const float *)samples, S, L, N, n_z, z, tn, out);
    }
    return cudaGetLastError();
}

}  // namespace mt
