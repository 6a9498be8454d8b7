// Instantiates the fused sweep kernels for the double-word form (KD_DW): every real of
// the spinor, the tables and the arithmetic is a pair of floats (kd_dw.cuh), one launch
// variant, the FP64 form's launch shapes.  The build compiles this file once per
// KD_DW_PART (axis x shape, 0..5) so that the heavy double-word kernels compile in
// parallel; part 0 also holds the dispatcher and the twiddle builder.
#include "kd_sweep.cuh"

#ifndef KD_DW_PART
#define KD_DW_PART 0
#endif

namespace kd {

template <int PART> cudaError_t launch_sweep_dw_part(int logn, const SweepArgs& a, cudaStream_t s);

template <> cudaError_t launch_sweep_dw_part<KD_DW_PART>(int logn, const SweepArgs& a, cudaStream_t s) {
    constexpr int AX = KD_DW_PART / 3 == 0 ? AXIS_X : AXIS_Y;
    constexpr int SH = KD_DW_PART % 3 == 0 ? SHAPE_F1F2 : (KD_DW_PART % 3 == 1 ? SHAPE_F1 : SHAPE_F2);
    return launch_logn<DW, AX, SH, 0>(logn, a, s);
}

#if KD_DW_PART == 0
template <> cudaError_t launch_sweep_dw_part<1>(int, const SweepArgs&, cudaStream_t);
template <> cudaError_t launch_sweep_dw_part<2>(int, const SweepArgs&, cudaStream_t);
template <> cudaError_t launch_sweep_dw_part<3>(int, const SweepArgs&, cudaStream_t);
template <> cudaError_t launch_sweep_dw_part<4>(int, const SweepArgs&, cudaStream_t);
template <> cudaError_t launch_sweep_dw_part<5>(int, const SweepArgs&, cudaStream_t);

cudaError_t launch_sweep_dw(int axis, int shape, int logn, const SweepArgs& a, cudaStream_t s) {
    const int sh = shape == SHAPE_F1F2 ? 0 : (shape == SHAPE_F1 ? 1 : (shape == SHAPE_F2 ? 2 : -1));
    if (sh < 0 || (axis != AXIS_X && axis != AXIS_Y)) return cudaErrorInvalidValue;
    switch ((axis == AXIS_X ? 0 : 3) + sh) {
        case 0: return launch_sweep_dw_part<0>(logn, a, s);
        case 1: return launch_sweep_dw_part<1>(logn, a, s);
        case 2: return launch_sweep_dw_part<2>(logn, a, s);
        case 3: return launch_sweep_dw_part<3>(logn, a, s);
        case 4: return launch_sweep_dw_part<4>(logn, a, s);
        default: return launch_sweep_dw_part<5>(logn, a, s);
    }
}
cudaError_t build_twiddles_dw(int logn, int loge, void* out, int* entries, cudaStream_t s) {
    return build_twiddles<DW>(logn, loge, out, entries, s);
}
#endif
}  // namespace kd
