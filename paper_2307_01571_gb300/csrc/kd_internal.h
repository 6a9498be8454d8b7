// kd_internal.h -- declarations shared by the host API (kd_api.cu) and the sweep kernels
// (kd_sweep_f32.cu, kd_sweep_f64.cu).  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace kd {

// Internal spinor layout: two pair planes [pair][ny][nx][2] complex.  In 2D with
// A = (A_x, A_y) and p = (p_x, p_y) both alpha.A and alpha.p + beta couple only
// psi1 <-> psi4 and psi2 <-> psi3, so the problem splits exactly into pair 0 = (psi1, psi4)
// and pair 1 = (psi2, psi3); internal slot s = 2 pair + index within the pair.  Pair 1's
// 2x2 generators are pair 0's with the y component negated.
__host__ __device__ constexpr int perm_to_dirac(int s) {  // internal slot -> Dirac component
    return s == 0 ? 0 : (s == 1 ? 3 : (s == 2 ? 1 : 2));
}

enum SweepAxis { AXIS_X = 0, AXIS_Y = 1 };
// FFT presence: FFT1 runs before the pointwise op, FFT2 after it.  On the x axis FFT1
// is inverse and FFT2 forward; on the y axis FFT1 is forward and FFT2 inverse.
enum SweepShape { SHAPE_F2 = 1, SHAPE_F1 = 2, SHAPE_F1F2 = 3 };
enum SweepOp { OP_NONE = 0, OP_POTENTIAL = 1, OP_KINETIC = 2 };

// Per-step scalars, FP64, written once per kd_step by a small kernel.
struct StepScalars {
    double t;      // time of the step boundary
    double s;      // a0 f(t) sin(omega t + phase0): common factor of the standing wave
    double ybase;  // y of row 0: y_min + box_vy t (co-moving box)
    float s_f;     // the same two, rounded once for the FP32 sweeps
    float ybase_f;
};

// Device clock: absolute step index of the state and the index at the start of the
// current kd_step call.  Kernels index StepScalars with (step - base) + n_local.
struct Clock {
    long long step;
    long long base;
};

struct SweepArgs {
    const void* in;
    void* out;
    const void* tw;       // stage-major twiddle table (build_twiddles_*): double2 (FP64)
                          // or float4 (c_hi, s_hi, c_lo, s_lo) (FP32)
    int nx, ny;
    int op;
    // potential (x sweep)
    const Clock* clock;
    const StepScalars* steps;
    int n_local;
    int kind, longitudinal;
    double kappa;         // tau m c^2 / hbar for this sweep (tau = dt or dt/2)
    double eps4;          // 4 epsilon (longitudinal amplitude factor)
    double y_min, dy;
    // FP32 copies of the scalars, rounded once on the host, so that the FP32 sweeps do
    // no FP64 arithmetic (the FP64 pipe is 1/64 of FP32 on GB300)
    float kappa_f, eps4_f, dy_f, mc_f, invP_f;
    double invP;          // 1 / (nx ny), exact
    const void* xtab;     // [2][nx][4] per-x field table, precision of the sweep:
                          // (Theta0, x/(x_R w^2), w0/w, 1/w^2) then (1/w, cos zeta, sin zeta, cos k x)
    // kinetic (y sweep)
    const void* ktab;     // [ny][nx] (C/P, c S/P) pairs
    const void* kxtab;    // [nx] pi_x
    const void* kytab;    // [ny] (pi_y, cos, sin of the frame phase, pad)
    double mc;            // m c
    // precision form (tensor-core sweeps of 1024-point axes, kd_tc.cu)
    const void* tc_b;     // 32-point DFT matrices (inverse hi, lo, forward hi, lo), FP16,
                          // times 2^10, in the kernel's shared-memory image (32 KiB)
    const void* tc_tw;    // [1024] float2 (cos, sin) of 2 pi m / 1024
    const float* tc_scale;  // [axis][2] power-of-two operand scales, set per kd_step
    const void* dwconst;  // double-word form: constant tables of exp and sin/cos (DWConst)
    int* status;          // error word of the simulation (KD_STATUS_* bits)
    int tc_fault;         // test hook (kd_inject_fault): the tensor-core sweep issues no
                          // matrix products, so that its bounded waits run out
};

// bits of the device status word
constexpr int KD_STATUS_NONFINITE = 1, KD_STATUS_DRIFT = 2, KD_STATUS_TC_TIMEOUT = 16;

// Launch variants of the FP32 sweeps, timed per grid by the autotuner (kd_autotune);
// variant 0 is the default.  A variant fixes the radix schedule (loge = log2 of the
// elements a thread owns: radix-8 or radix-4 Stockham stages), the threads per CTA (a
// target: at least one whole line), the minimum column-tile width of the y sweep, the
// spinor components per CTA (2: one 2x2 pair per CTA, the two pairs' CTAs side by side;
// 4: both pairs, sharing the field or table loads) and the resident warps per SM the
// register budget is built for.  Variants that differ only in threads or tile width do
// the same arithmetic per line (bitwise identical results); a different radix schedule,
// or components per CTA (the compiler may fuse the pointwise ops' multiply-adds
// differently), rounds differently.  share (x axis, nc 2): one CTA holds both pairs of its
// lines, the pairs' threads owning the same points; each thread evaluates the standing
// wave for half of its points and the two halves trade the potential factors through
// shared memory (the field costs as much as both pairs' arithmetic of the potential step).
// FP64 sweeps have the one variant 0.
struct SweepVariant {
    int loge, threads, minb, nc, resident_warps, share;
};
constexpr int kNumSweepVariants = 4;
__host__ __device__ constexpr SweepVariant sweep_variant(int axis, int v) {
    return axis == AXIS_X
        ? (v == 1 ? SweepVariant{3, 256, 1, 2, 24, 1}
         : v == 2 ? SweepVariant{2, 128, 1, 2, 32, 0}
         : v == 3 ? SweepVariant{3, 128, 1, 4, 16, 0}
                  : SweepVariant{3, 128, 1, 2, 28, 0})
        : (v == 1 ? SweepVariant{3, 512, 8, 4, 16, 0}
         : v == 2 ? SweepVariant{2, 256, 4, 4, 24, 0}
         : v == 3 ? SweepVariant{3, 256, 4, 2, 28, 0}
                  : SweepVariant{3, 256, 4, 4, 16, 0});
}
// spinor components per CTA: FP64 CTAs own both pairs (the costly FP64 field is evaluated
// once) except at N = 4096, where registers allow one pair
__host__ __device__ constexpr int sweep_nc(bool f64, int axis, int logn, int v) {
    return f64 ? (logn >= 12 ? 2 : 4) : sweep_variant(axis, v).nc;
}
// log2 of the elements per thread (the radix of the Stockham stages)
__host__ __device__ constexpr int sweep_loge(bool f64, int axis, int logn, int v) {
    const int lmax = f64 ? (sweep_nc(f64, axis, logn, v) == 2 ? 3 : 2) : sweep_variant(axis, v).loge;
    return logn < lmax ? logn : lmax;
}

// log2 of the elements per thread of the double-word form: radix-4 stages (four
// double-word complex values per component keep the register use within two CTAs per SM)
// up to 1024-point lines, radix-8 above (a line's threads stay within 256)
__host__ __device__ constexpr int sweep_loge_dw(int logn) { return logn < 2 ? logn : (logn <= 10 ? 2 : 3); }

// Launches one sweep; returns cudaSuccess or the launch error.  logn in [2, 12],
// variant in [0, kNumSweepVariants).
template <int V>
cudaError_t launch_sweep_f32_v(int axis, int shape, int logn, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_sweep_f32(int variant, int axis, int shape, int logn, const SweepArgs& a,
                             cudaStream_t s);
cudaError_t launch_sweep_f64(int axis, int shape, int logn, const SweepArgs& a, cudaStream_t s);
// Double-word form (KD_DW): the FP64 form's launch shapes with every real a float pair.
cudaError_t launch_sweep_dw(int axis, int shape, int logn, const SweepArgs& a, cudaStream_t s);
// Precision form: whether an axis of 2^logn points has the tensor-core sweep, and its
// launch (full sweeps only; persistent, at most two CTAs per SM).
bool tc_supported(int logn);
cudaError_t launch_tc_sweep(int axis, const SweepArgs& a, cudaStream_t s);
// Fills the stage-major twiddle table of an N = 2^logn sweep whose threads own 2^loge
// elements (at most 2N entries of 16 B) and returns the number of entries.
cudaError_t build_twiddles_f32(int logn, int loge, void* out, int* entries, cudaStream_t s);
cudaError_t build_twiddles_f64(int logn, int loge, void* out, int* entries, cudaStream_t s);
cudaError_t build_twiddles_dw(int logn, int loge, void* out, int* entries, cudaStream_t s);

}  // namespace kd
