// Instantiates the fused sweep kernels for float spinors (one translation unit per
// precision so that the two compile in parallel).
#include "kd_sweep.cuh"

namespace kd {
cudaError_t launch_sweep_f32(int axis, int shape, int logn, const SweepArgs& a, cudaStream_t s) {
    return launch_sweep<float>(axis, shape, logn, a, s);
}
cudaError_t build_twiddles_f32(int logn, void* out, int* entries, cudaStream_t s) {
    return build_twiddles<float>(logn, out, entries, s);
}
}  // namespace kd
