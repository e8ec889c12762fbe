// march_f32a.cu -- k_march instantiations for MODE_F32A (one translation unit
// per precision so they compile in parallel).
#include "march_launch.cuh"

namespace mt {
template cudaError_t launch_march_mode<MODE_F32A>(const Prob &, HRef, int, int, size_t, void *,
                                                  double *, double *, cudaStream_t);
}  // namespace mt
