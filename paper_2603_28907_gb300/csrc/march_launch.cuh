// march_launch.cuh -- instantiation and launch of k_march for one precision.
#pragma once

#include "march.cuh"

namespace mt {

template <int MODE, int L>
static cudaError_t launch_global(const Prob &pb, HRef h, int n_chains, int rpb, void *partial,
                                 double *ray_O, double *ray_term, cudaStream_t st)
{
    if constexpr (is_dx_mode(MODE)) {
        using Hh = typename Types<MODE>::H;
        dim3 sg((pb.N + 4095) / 4096, n_chains);
        k_stage_dx_global<Hh, L><<<sg, 256, 0, st>>>(pb, h);
        void (*fn)(Prob, HRef, int, void *, double *, double *) =
            pb.gamma == 0.0 ? k_march<MODE, L, true, true> : k_march<MODE, L, false, true>;
        dim3 grid((pb.n_rays + rpb - 1) / rpb, n_chains);
        fn<<<grid, MarchCfg<MODE, L>::THREADS, 0, st>>>(pb, h, rpb, partial, ray_O, ray_term);
        return cudaGetLastError();
    } else {
        return cudaErrorInvalidValue;
    }
}

template <int MODE, int L>
static cudaError_t launch_phased(const Prob &pb, HRef h, int n_chains, int rpb, void *partial, double *ray_O,
                                 double *ray_term, cudaStream_t st)
{
    if constexpr (is_dx_mode(MODE)) {
        const bool hard = pb.gamma == 0.0;
        void (*fn)(Prob, HRef, int, void *, double *, double *) =
            hard ? k_march_phased<MODE, L, true> : k_march_phased<MODE, L, false>;
        const size_t smem = march_phased_smem_bytes(pb);
        static size_t smem_set[2] = {0, 0};
        if (smem > 48 * 1024 && smem > smem_set[hard]) {
            cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            smem_set[hard] = smem;
        }
        dim3 grid((pb.n_rays + rpb - 1) / rpb, n_chains);
        fn<<<grid, MarchCfg<MODE, L>::THREADS, smem, st>>>(pb, h, rpb, partial, ray_O, ray_term);
        return cudaGetLastError();
    } else {
        return cudaErrorInvalidValue;
    }
}

template <int MODE, int L>
static cudaError_t launch_l(const Prob &pb, HRef h, int n_chains, int rpb, size_t smem,
                            void *partial, double *ray_O, double *ray_term, cudaStream_t st)
{
    if (pb.gnodes) return launch_global<MODE, L>(pb, h, n_chains, rpb, partial, ray_O, ray_term, st);
    if (smem + MT_SMEM_STATIC > MT_MAX_SMEM)  // one surface's plane at a time
        return launch_phased<MODE, L>(pb, h, n_chains, rpb, partial, ray_O, ray_term, st);
    const bool hard = pb.gamma == 0.0;
    void (*fn)(Prob, HRef, int, void *, double *, double *) =
        hard ? k_march<MODE, L, true> : k_march<MODE, L, false>;
    // Raise the dynamic shared-memory limit once per instantiation and size,
    // before any launch (so never inside a stream capture).
    static size_t smem_set[2] = {0, 0};
    if (smem > 48 * 1024 && smem > smem_set[hard]) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        smem_set[hard] = smem;
    }
    dim3 grid((pb.n_rays + rpb - 1) / rpb, n_chains);
    fn<<<grid, MarchCfg<MODE, L>::THREADS, smem, st>>>(pb, h, rpb, partial, ray_O, ray_term);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_march_mode(const Prob &pb, HRef h, int n_chains, int rpb, size_t smem,
                              void *partial, double *ray_O, double *ray_term, cudaStream_t st)
{
    switch (pb.L) {
        case 1: return launch_l<MODE, 1>(pb, h, n_chains, rpb, smem, partial, ray_O, ray_term, st);
        case 2: return launch_l<MODE, 2>(pb, h, n_chains, rpb, smem, partial, ray_O, ray_term, st);
        case 3: return launch_l<MODE, 3>(pb, h, n_chains, rpb, smem, partial, ray_O, ray_term, st);
        case 4: return launch_l<MODE, 4>(pb, h, n_chains, rpb, smem, partial, ray_O, ray_term, st);
        case 5: return launch_l<MODE, 5>(pb, h, n_chains, rpb, smem, partial, ray_O, ray_term, st);
        case 6: return launch_l<MODE, 6>(pb, h, n_chains, rpb, smem, partial, ray_O, ray_term, st);
        case 7: return launch_l<MODE, 7>(pb, h, n_chains, rpb, smem, partial, ray_O, ray_term, st);
        case 8: return launch_l<MODE, 8>(pb, h, n_chains, rpb, smem, partial, ray_O, ray_term, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace mt
