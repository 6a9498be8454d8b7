// Instantiates the fused sweep kernels for double spinors (a translation unit of its own
// so that it compiles in parallel with the FP32 variants).
#include "kd_sweep.cuh"

namespace kd {
cudaError_t launch_sweep_f64(int axis, int shape, int logn, const SweepArgs& a, cudaStream_t s) {
    return launch_sweep<double, 0>(axis, shape, logn, a, s);
}
cudaError_t build_twiddles_f64(int logn, int loge, void* out, int* entries, cudaStream_t s) {
    return build_twiddles<double>(logn, loge, out, entries, s);
}
}  // namespace kd
