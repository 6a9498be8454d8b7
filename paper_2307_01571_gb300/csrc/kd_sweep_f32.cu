// Instantiates the fused sweep kernels for float spinors, one launch variant per object
// file: the build compiles this file once per KD_SWEEP_VARIANT so that the variants
// compile in parallel.
#include "kd_sweep.cuh"

#ifndef KD_SWEEP_VARIANT
#define KD_SWEEP_VARIANT 0
#endif

namespace kd {
template <int V>
cudaError_t launch_sweep_f32_v(int axis, int shape, int logn, const SweepArgs& a, cudaStream_t s) {
    return launch_sweep<float, V>(axis, shape, logn, a, s);
}
template cudaError_t launch_sweep_f32_v<KD_SWEEP_VARIANT>(int, int, int, const SweepArgs&, cudaStream_t);

#if KD_SWEEP_VARIANT == 0
cudaError_t launch_sweep_f32(int variant, int axis, int shape, int logn, const SweepArgs& a,
                             cudaStream_t s) {
    static_assert(kNumSweepVariants == 4, "one case per compiled variant");
    switch (variant) {
        case 0: return launch_sweep_f32_v<0>(axis, shape, logn, a, s);
        case 1: return launch_sweep_f32_v<1>(axis, shape, logn, a, s);
        case 2: return launch_sweep_f32_v<2>(axis, shape, logn, a, s);
        case 3: return launch_sweep_f32_v<3>(axis, shape, logn, a, s);
        default: return cudaErrorInvalidValue;
    }
}
cudaError_t build_twiddles_f32(int logn, int loge, void* out, int* entries, cudaStream_t s) {
    return build_twiddles<float>(logn, loge, out, entries, s);
}
#endif
}  // namespace kd
