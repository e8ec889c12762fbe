// noalloc.cu -- mt_logpost_noalloc: the log-posterior evaluation of
// mt_logpost for callers that cannot allocate device memory.
//
// The ray kernel writes one partial sum per (chain, CTA) that the reduction
// then adds in a fixed order.  mt_logpost keeps those partials in a buffer
// the context grows with cudaMalloc; here they live in a file-scope device
// array of fixed size instead, so the call itself allocates nothing.
#include <stdio.h>

#include <mutex>

#include "internal.h"

namespace {

constexpr size_t kScratchBytes = 1u << 20;  // 1 MiB: 131072 partial sums
constexpr int kMaxDevices = 64;

// Shared by every call on a device; keeps whatever the last call wrote.
__device__ __align__(256) unsigned char g_partials[kScratchBytes];

std::mutex g_lock;
void *g_partials_addr[kMaxDevices] = {};

// Device address of g_partials on the current device (set up on first use
// and kept for the process: the cache assumes the device's primary context
// lives as long as the process, i.e. nobody resets the device in between).
// In host code the name g_partials is only a stand-in for the symbol; a
// kernel must be given the address cudaGetSymbolAddress returns.
cudaError_t partials_address(int device, void **out)
{
    std::lock_guard<std::mutex> g(g_lock);
    if (!g_partials_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) return e;
        g_partials_addr[device] = p;
    }
    *out = g_partials_addr[device];
    return cudaSuccess;
}

// Device memory of `device` (or managed memory, which every device can
// reach); host memory and another GPU's memory are rejected, since the kernels
// would read them without a copy.
bool on_device(const void *p, int device)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == device);
}

}  // namespace

using namespace mt;

extern "C" MT_API mt_status mt_logpost_noalloc(mt_ctx *ctx, int n_chains, const void *heights,
                                               double *loglik_out, double *logprior_out)
{
    CtxView v;
    mt_status st = ctx_view(ctx, &v);
    if (st != MT_OK) return st;
    if (n_chains < 1 || n_chains > 65535)
        return ctx_fail(ctx, MT_EINVAL, "mt_logpost_noalloc: need 1 <= n_chains <= 65535");
    if (!heights || !loglik_out)
        return ctx_fail(ctx, MT_EINVAL, "mt_logpost_noalloc: heights and loglik_out are required");
    if (!on_device(heights, v.device) || !on_device(loglik_out, v.device) ||
        (logprior_out && !on_device(logprior_out, v.device)))
        return ctx_fail(ctx, MT_EINVAL,
                        "mt_logpost_noalloc: every array must be device memory of the context's "
                        "device (staging host memory would need an allocation)");
    if (!march_fits_smem(v.pb, v.mode) && !march_fits_phased(v.pb, v.mode))
        return ctx_fail(ctx, MT_EINVAL,
                        "mt_logpost_noalloc: not even one surface of the grid fits in shared memory "
                        "(that path needs an HBM buffer); use mt_logpost");
    v.pb.gnodes = nullptr;
    const int rpb = march_rays_per_block(v.pb);
    const size_t n_blk = (size_t)(v.pb.n_rays + rpb - 1) / rpb;
    const size_t need = (size_t)n_chains * n_blk * 8;
    if (need > kScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "mt_logpost_noalloc: %d chains need %zu bytes of partial sums, the fixed "
                 "limit is %zu bytes (at most %zu chains for this problem); use mt_logpost",
                 n_chains, need, kScratchBytes, kScratchBytes / (n_blk * 8));
        return ctx_fail(ctx, MT_EINVAL, msg);
    }
    if (v.device < 0 || v.device >= kMaxDevices)
        return ctx_fail(ctx, MT_EINVAL, "mt_logpost_noalloc: device ordinal out of range");
    void *partials = nullptr;
    cudaError_t e = partials_address(v.device, &partials);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ctx_fail(ctx, MT_ECUDA, cudaGetErrorString(e));
    }
    // Nothing in the array needs to start at zero: the ray kernel writes every
    // partial the reduction reads, earlier on the same stream.
    const long long np = (long long)v.pb.L * v.pb.N;
    HRef h{heights, np, nullptr, 0, 0};
    if (logprior_out) e = launch_prior(v.pb, v.mode, h, v.mu, n_chains, logprior_out, v.stream);
    if (e == cudaSuccess) e = launch_march(v.pb, v.mode, h, n_chains, partials, nullptr, nullptr, v.stream);
    if (e == cudaSuccess) e = launch_reduce_ll(v.pb, v.mode, n_chains, partials, loglik_out, v.stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ctx_fail(ctx, MT_ECUDA, cudaGetErrorString(e));
    }
    return MT_OK;
}
