// Instantiates the fused sweep kernels for double spinors (one translation unit per
// precision so that the two compile in parallel).
#include "kd_sweep.cuh"

namespace kd {
cudaError_t launch_sweep_f64(int axis, int shape, int logn, const SweepArgs& a, cudaStream_t s) {
    return launch_sweep<double>(axis, shape, logn, a, s);
}
cudaError_t build_twiddles_f64(int logn, void* out, int* entries, cudaStream_t s) {
    return build_twiddles<double>(logn, out, entries, s);
}
}  // namespace kd
