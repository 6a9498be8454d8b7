// kd_api.cu -- host side of the C ABI declared in include/kd.h: validation, device
// buffers, FP64 phase tables, the graph-captured step loop, observables and
// checkpoints.  All arithmetic of the step runs in the sweep kernels (kd_sweep.cuh) and
// in the small kernels below; nothing here computes on the host except FP64 tables of
// at most max(nx, ny) entries.
//
// Paper: Ge, Ahrens & Shen, arXiv 2307.01571.  Sec. II.A (field), II.B (Hamiltonian,
// bispinors, energy), II.C (packet, Fourier convention), II.D (split-operator step),
// III (observables).
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/kd.h"
#include "kd_dw.cuh"
#include "kd_internal.h"
#include "kd_persist.h"

using namespace kd;

static_assert(KD_SWEEP_VARIANTS == kNumSweepVariants, "public and internal variant counts");

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define KD_CUDA(call)                                                                    \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? KD_ERR_NOMEM : KD_ERR_CUDA,    \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

constexpr double kPi = 3.14159265358979323846264338327950288;

bool pow2_in_range(int32_t n) { return n >= 4 && n <= 4096 && (n & (n - 1)) == 0; }
int ilog2(int32_t n) { int l = 0; while ((1 << l) < n) ++l; return l; }
int32_t signed_index(int32_t k, int32_t n) { return k < n / 2 ? k : k - n; }

struct ObsWin {  // window of signed momentum indices, integer, computed on the host
    int ilo[2], ihi[2], jlo[2], jhi[2];
    int it, jt;
};

struct GraphKey {
    int chunk, last, obs;
    bool operator<(const GraphKey& o) const {
        return std::tie(chunk, last, obs) < std::tie(o.chunk, o.last, o.obs);
    }
};

}  // namespace

namespace kd {
// Records a message for kd_last_error() from another translation unit.
int set_error(int code, const char* msg) { return fail(code, "%s", msg); }
// Clears the message of kd_last_error() after a successful call in another unit.
void clear_error() { g_err.clear(); }
}  // namespace kd

namespace {
// Test hook of kd_inject_alloc_failure: -1 = off; k >= 0 = the allocation after k more
// successful ones fails as if the device were out of memory (then the hook turns off).
std::atomic<int> g_alloc_fail_after{-1};

// Every device allocation of the library goes through here.
cudaError_t dev_alloc(void** p, size_t bytes) {
    int k = g_alloc_fail_after.load();
    while (k >= 0) {
        if (g_alloc_fail_after.compare_exchange_weak(k, k == 0 ? -1 : k - 1)) {
            if (k == 0) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMalloc(p, bytes);
}
}  // namespace

struct kd_sim {
    kd_units u;
    kd_grid g;
    kd_field f;
    int prec;
    size_t tsize;    // sizeof real
    cudaStream_t stream;
    cudaStream_t cap_stream;
    int device;
    int lx, ly;
    size_t P;
    void* psi = nullptr;
    void* work = nullptr;
    void* tw[2][2] = {};   // twiddle tables [axis][loge - 2] (radix-4 and radix-8 schedules)
    int var[2] = {0, 0};   // sweep launch variant per axis (kd_autotune)
    void* xtab = nullptr;
    void* kxtab = nullptr;
    void* kytab = nullptr;
    void* ktab = nullptr;
    double ktab_dt = 0.0;
    Clock* clock = nullptr;
    StepScalars* steps = nullptr;
    int64_t steps_cap = 0;
    double* rowsum = nullptr;
    double* md = nullptr;
    double* scalar = nullptr;   // [0] norm of a reduction, [1] reference norm
    kd_obs* obs_dev = nullptr;
    int64_t obs_dev_cap = 0;
    int* status = nullptr;
    // precision form: tensor-core sweeps of 1024-point axes (KD_FP32_TC)
    bool tc = false;
    void* tc_b = nullptr;
    void* tc_tw = nullptr;
    float* tc_scale = nullptr;
    int tc_fault = 0;          // kd_inject_fault: applies to the next kd_step call only
    int persist_hold = 0;      // kd_inject_fault(KD_FAULT_PERSIST_HOLD): next persistent batch step
    // double-word form (KD_DW): the state psi and the tables xtab, kxtab, kytab, ktab hold
    // float pairs; prec stays KD_FP64 for the observation path, which reads an FP64 copy
    // of the state (view) and runs the FP64 transforms on it
    bool dw = false;
    void* tw_dw[2] = {};       // double-word twiddles per axis
    void* dwconst = nullptr;   // DWConst (exp and sin/cos tables)
    void* view = nullptr;      // FP64 copy of the state for read-outs
    std::atomic<int> cancel{0};  // kd_cancel: the running or next kd_step stops early
    // kd_step keeps at most kRunAhead chunks in flight (host waits on the event of the
    // chunk kRunAhead back), so that a cancellation stops work that is not yet queued
    static constexpr int kRunAhead = 4;
    cudaEvent_t ahead[kRunAhead] = {};
    // host clock: t = t0 + step * dt_clock
    double t0 = 0.0, dt_clock = 0.0;
    int64_t step = 0;
    kd_obs_spec spec{};
    bool has_spec = false;
    double watch_tol = 0.0;
    // graphs of the step loop; cleared whenever a captured argument changes
    std::map<GraphKey, std::pair<cudaGraphExec_t, int64_t>> graphs;  // exec, kernel nodes
    uint64_t graph_gen = 0;   // incremented whenever captured arguments change
    int64_t launches = 0;
    int64_t graph_obs_every = -1, graph_obs_cap = -1;
    double graph_dt = 0.0, graph_t0 = 0.0;
    ObsWin graph_win{};
};

namespace {

size_t cbytes(const kd_sim* s) { return 2 * s->tsize; }                  // one complex
size_t spinor_bytes(const kd_sim* s) { return s->P * 4 * cbytes(s); }

double dxdy(const kd_sim* s) {
    return (s->g.x_max - s->g.x_min) / s->g.nx * (s->g.y_max - s->g.y_min) / s->g.ny;
}

void clear_graphs(kd_sim* s) {
    for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second.first);
    s->graphs.clear();
    ++s->graph_gen;
}

// ---------------------------------------------------------------- small kernels ---

// Kinetic table: (C - 1)/P and c S/P with C = cos(E dt/hbar) (C - 1 = -2 sin^2(E dt/2hbar)
// kept as a small number), S = sin(E dt/hbar)/E, E from the relativistic energy-momentum
// relation (Sec. II.B), pi = canonical + p_shift.  FP64 throughout; rounded once to the
// sweep precision.
template <typename T>
__global__ void k_ktab(T* out, int nx, int ny, double dpx, double dpy, double shx, double shy,
                       double c, double mc2, double hbar, double dt, const T* kxtab,
                       const T* kytab, double mc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx * ny) return;
    const int kx = i % nx, ky = i / nx;
    const double px = dpx * (kx < nx / 2 ? kx : kx - nx) + shx;
    const double py = dpy * (ky < ny / 2 ? ky : ky - ny) + shy;
    const double E = sqrt(mc2 * mc2 + c * c * (px * px + py * py));
    double sh, ch;
    sincos(0.5 * E * dt / hbar, &sh, &ch);
    const double P = (double)nx * (double)ny;
    const double a = -2.0 * sh * sh / P, b = c * (2.0 * sh * ch) / E / P;
    if (sizeof(T) == 8) {
        out[2 * i] = (T)a;
        out[2 * i + 1] = (T)b;
        return;
    }
    // FP32: of the pairs within 3 ulps of the rounded (a, b), take the one whose factor
    // 1/P + a - i b G, G = H0/c built from the same rounded m c, pi_x, pi_y that the sweep
    // uses, is closest to unitary: (1 + P a)^2 + (P b)^2 |G|^2 = 1, ties broken by the
    // closer rotation angle.  Plain rounding leaves a coherent per-step norm error of
    // order (E dt)^2 2^-24 at every k, which adds up over thousands of steps.
    const double gx = (double)kxtab[kx], gy = (double)kytab[4 * ky], gm = (double)(T)mc;
    const double G = sqrt(gm * gm + gx * gx + gy * gy);
    const float a0 = (float)a, b0 = (float)b;
    const double ang0 = atan2(P * b * E / c, 1.0 + P * a);
    float ba = a0, bb = b0;
    double best = 1e300;
    float ai = a0;
    for (int k = 0; k < 3; ++k) ai = nextafterf(ai, -INFINITY);
    for (int da = -3; da <= 3; ++da, ai = nextafterf(ai, INFINITY)) {
        float bi = b0;
        for (int k = 0; k < 3; ++k) bi = nextafterf(bi, -INFINITY);
        for (int db = -3; db <= 3; ++db, bi = nextafterf(bi, INFINITY)) {
            const double x = 1.0 + P * (double)ai, y = P * (double)bi * G;
            const double g = fabs(x * x + y * y - 1.0) + 1e-3 * fabs(atan2(y, x) - ang0);
            if (g < best) { best = g; ba = ai; bb = bi; }
        }
    }
    out[2 * i] = (T)ba;
    out[2 * i + 1] = (T)bb;
}

// Time-dependent scalars of the standing wave for the steps of one kd_step call:
// s(t) = a0 f(t) sin(omega t + phase0) and the co-moving box offset.
__global__ void k_step_scalars(StepScalars* out, int64_t n, double t0, int64_t step0, double dt,
                               double a0, double omega, double phase0, double env_T,
                               double box_vy, double y_min) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i > n) return;
    const double t = t0 + (double)(step0 + i) * dt;
    double f = 1.0;
    if (env_T > 0.0) {
        if (t < 0.0 || t > env_T) f = 0.0;
        else { const double sv = sin(kPi * t / env_T); f = sv * sv; }
    }
    StepScalars r;
    r.t = t;
    r.s = a0 * f * sin(omega * t + phase0);
    r.ybase = y_min + box_vy * t;
    r.s_f = (float)r.s;
    r.ybase_f = (float)r.ybase;
    out[i] = r;
}

__global__ void k_set_clock(Clock* c, long long step) { c->step = step; c->base = step; }
__global__ void k_advance_clock(Clock* c, int n) { c->step += n; }

// Real offset of internal slot s (0..3) of a point in the pair-plane layout
// [pair][P][2] complex: slot s = 2 pair + index within the pair.
__host__ __device__ inline size_t slot_off(size_t P, size_t point, int s) {
    return ((size_t)(s >> 1) * P + point) * 4 + 2 * (s & 1);
}

// Per-row sum of |psi|^2 over both pair planes (fixed-order tree: bitwise reproducible).
template <typename T>
__global__ void k_rowsum(const T* psi, int nx, int ny, double* rowsum) {
    __shared__ double red[256];
    const int row = blockIdx.x;
    const size_t P = (size_t)nx * ny;
    // squares summed in groups of 8 in the spinor's precision, groups in FP64: keeps the
    // FP32 sweeps' reduction off the slow FP64 pipe while the sum stays accurate to ~1e-9
    double acc = 0.0;
    T part = T(0);
    int cnt = 0;
    for (int i = threadIdx.x; i < nx * 8; i += blockDim.x) {
        const int pair = i / (nx * 4), k = i % (nx * 4);
        const T v = psi[(pair * P + (size_t)row * nx) * 4 + k];
        part += v * v;
        if (++cnt == 8) { acc += (double)part; part = T(0); cnt = 0; }
    }
    acc += (double)part;
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) rowsum[row] = red[0];
}

// Phi(x) = sum_y |psi|^2 dy, one thread per column, rows in order.
template <typename T>
__global__ void k_density_x(const T* psi, int nx, int ny, double dy, double* out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    double acc = 0.0;
    const size_t P = (size_t)nx * ny;
    for (int y = 0; y < ny; ++y) {
        double s = 0.0;
        for (int pair = 0; pair < 2; ++pair) {
            const T* p = psi + (pair * P + (size_t)y * nx + x) * 4;
            for (int i = 0; i < 4; ++i) s += (double)p[i] * (double)p[i];
        }
        acc += s;
    }
    out[x] = acc * dy;
}

// Sum of the row sums times dx dy into scalar[slot]; fixed order.
__global__ void k_norm(const double* rowsum, int ny, double cell, double* scalar, int slot) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < ny; i += blockDim.x) acc += rowsum[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) scalar[slot] = red[0] * cell;
}

// Power-of-two operand scales of the tensor-core sweeps from the state's 2-norm
// S = sqrt(sum |psi|^2) (position space, all components): every FP16 operand stays below
// 2^14 by the growth bounds of the unnormalised DFTs (an element of a 32-point partial DFT
// of a vector is at most sqrt(32) times the vector's 2-norm).  out = (x: s_a, s_b,
// y: s_a, s_b); operands before the pointwise factor carry s_a, after it s_a s_b.
__global__ void k_tc_scales(const double* rowsum, int nx, int ny, float* out) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < ny; i += blockDim.x) acc += rowsum[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    double S = sqrt(red[0]);
    if (!(S > 0.0) || !isfinite(S)) S = 1.0;
    auto p2 = [](double v) {   // largest power of two <= v, as a float
        int e = (int)floor(log2(v));
        e = e < -120 ? -120 : (e > 120 ? 120 : e);
        return ldexpf(1.0f, e);
    };
    const double P = (double)nx * ny;
    const double sa = 16384.0 / (sqrt(32.0 * nx) * S);
    out[0] = p2(sa);
    out[1] = p2(1.0 / sqrt((double)nx));
    out[2] = p2(sa);
    out[3] = p2(sqrt(P * nx));
}

template <typename T>
__global__ void k_scale_by_norm(T* psi, size_t n, const double* scalar) {
    const double nr = scalar[0];
    const T s = (T)(nr > 0.0 ? 1.0 / sqrt(nr) : 0.0);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        psi[i] *= s;
}

// Normalised positive-energy bispinor u^s(pi) of Eq. (Spinors_of_Dirac_equation) with
// unit chi (x-polarised chi = (1, +-1)/sqrt 2, or z-polarised); Dirac component order.
__device__ void bispinor(double c, double mc2, double pix, double piy, int spin, int basis,
                         double2 u[4]) {
    const double E = sqrt(mc2 * mc2 + c * c * (pix * pix + piy * piy));
    const double nrm = sqrt((E + mc2) / (2.0 * E));
    double2 chi[2];
    if (basis == 1) {
        chi[0] = make_double2(spin > 0 ? 1.0 : 0.0, 0.0);
        chi[1] = make_double2(spin > 0 ? 0.0 : 1.0, 0.0);
    } else {
        const double r = 0.70710678118654752440;
        chi[0] = make_double2(r, 0.0);
        chi[1] = make_double2(spin > 0 ? r : -r, 0.0);
    }
    // lower = c sigma.pi chi / (E + mc^2); sigma.pi = [[0, pix - i piy], [pix + i piy, 0]]
    const double f = c / (E + mc2);
    const double2 lo0 = make_double2(f * (pix * chi[1].x + piy * chi[1].y), f * (pix * chi[1].y - piy * chi[1].x));
    const double2 lo1 = make_double2(f * (pix * chi[0].x - piy * chi[0].y), f * (pix * chi[0].y + piy * chi[0].x));
    u[0] = make_double2(nrm * chi[0].x, nrm * chi[0].y);
    u[1] = make_double2(nrm * chi[1].x, nrm * chi[1].y);
    u[2] = make_double2(nrm * lo0.x, nrm * lo0.y);
    u[3] = make_double2(nrm * lo1.x, nrm * lo1.y);
}

// phi(p, 0) = u^s(pi) rho(pi), rho = exp(-|pi - p0|^2/(4 sigma^2) - i (r0 - origin).p/hbar)
// (Sec. II.C); written in the internal component order.
template <typename T>
__global__ void k_packet(T* psi, int nx, int ny, double dpx, double dpy, double shx, double shy,
                         double p0x, double p0y, double rx, double ry, double sig, int spin,
                         int basis, double c, double mc2, double hbar) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx * ny) return;
    const int kx = i % nx, ky = i / nx;
    const double px = dpx * (kx < nx / 2 ? kx : kx - nx), py = dpy * (ky < ny / 2 ? ky : ky - ny);
    const double pix = px + shx, piy = py + shy;
    const double ddx = pix - p0x, ddy = piy - p0y;
    const double mag = exp(-(ddx * ddx + ddy * ddy) / (4.0 * sig * sig));
    double sn, cs;
    sincos(-(rx * px + ry * py) / hbar, &sn, &cs);
    double2 u[4];
    bispinor(c, mc2, pix, piy, spin, basis, u);
    for (int s = 0; s < 4; ++s) {
        const double2 uu = u[perm_to_dirac(s)];
        const size_t o = slot_off((size_t)nx * ny, i, s);
        psi[o] = (T)(mag * (uu.x * cs - uu.y * sn));
        psi[o + 1] = (T)(mag * (uu.x * sn + uu.y * cs));
    }
}

// Per-cell momentum-space probabilities from phi = DFT psi (internal order):
// (|phi|^2, |c+|^2, |c-|^2) dx dy / P, c^s = u^s(pi)^dagger phi.
template <typename T>
__global__ void k_momentum_density(const T* phi, int nx, int ny, double dpx, double dpy,
                                   double shx, double shy, double c, double mc2, int basis,
                                   double cellw, double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx * ny) return;
    const int kx = i % nx, ky = i / nx;
    const double pix = dpx * (kx < nx / 2 ? kx : kx - nx) + shx;
    const double piy = dpy * (ky < ny / 2 ? ky : ky - ny) + shy;
    double2 f[4];
    for (int s = 0; s < 4; ++s) {
        const size_t o = slot_off((size_t)nx * ny, i, s);
        f[perm_to_dirac(s)] = make_double2((double)phi[o], (double)phi[o + 1]);
    }
    double p2 = 0.0;
    for (int d = 0; d < 4; ++d) p2 += f[d].x * f[d].x + f[d].y * f[d].y;
    double cpm[2];
    for (int si = 0; si < 2; ++si) {
        double2 u[4];
        bispinor(c, mc2, pix, piy, si == 0 ? 1 : -1, basis, u);
        double re = 0.0, im = 0.0;
        for (int d = 0; d < 4; ++d) {  // conj(u) * f
            re += u[d].x * f[d].x + u[d].y * f[d].y;
            im += u[d].x * f[d].y - u[d].y * f[d].x;
        }
        cpm[si] = re * re + im * im;
    }
    out[(size_t)i * 3 + 0] = p2 * cellw;
    out[(size_t)i * 3 + 1] = cpm[0] * cellw;
    out[(size_t)i * 3 + 2] = cpm[1] * cellw;
}

// Momentum-space cell values (|phi|^2, |c+|^2, |c-|^2) dx dy / P of the two observation
// windows (row-major within each window) and the target cell, from phi = DFT psi in the
// internal layout; FP64, one thread per cell.  out[cell][3].
template <typename T>
__global__ void k_obs_cells(const T* phi, int nx, int ny, double dpx, double dpy, double shx,
                            double shy, double c, double mc2, int basis, double cellw, ObsWin w,
                            double* out) {
    const int n0 = (w.ihi[0] - w.ilo[0] + 1) * (w.jhi[0] - w.jlo[0] + 1);
    const int n1 = (w.ihi[1] - w.ilo[1] + 1) * (w.jhi[1] - w.jlo[1] + 1);
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e > n0 + n1) return;
    int i, j;
    if (e < n0) {
        const int wx = w.ihi[0] - w.ilo[0] + 1;
        i = w.ilo[0] + e % wx; j = w.jlo[0] + e / wx;
    } else if (e < n0 + n1) {
        const int wx = w.ihi[1] - w.ilo[1] + 1;
        i = w.ilo[1] + (e - n0) % wx; j = w.jlo[1] + (e - n0) / wx;
    } else {
        i = w.it; j = w.jt;
    }
    const int kx = (i + nx) % nx, ky = (j + ny) % ny;
    const size_t pt = (size_t)ky * nx + kx;
    const double pix = dpx * (kx < nx / 2 ? kx : kx - nx) + shx;
    const double piy = dpy * (ky < ny / 2 ? ky : ky - ny) + shy;
    double2 f[4];
    for (int s = 0; s < 4; ++s) {
        const size_t o = slot_off((size_t)nx * ny, pt, s);
        f[perm_to_dirac(s)] = make_double2((double)phi[o], (double)phi[o + 1]);
    }
    double p2 = 0.0;
    for (int d = 0; d < 4; ++d) p2 += f[d].x * f[d].x + f[d].y * f[d].y;
    double cpm[2];
    for (int si = 0; si < 2; ++si) {
        double2 u[4];
        bispinor(c, mc2, pix, piy, si == 0 ? 1 : -1, basis, u);
        double re = 0.0, im = 0.0;
        for (int d = 0; d < 4; ++d) {
            re += u[d].x * f[d].x + u[d].y * f[d].y;
            im += u[d].x * f[d].y - u[d].y * f[d].x;
        }
        cpm[si] = re * re + im * im;
    }
    out[(size_t)e * 3 + 0] = p2 * cellw;
    out[(size_t)e * 3 + 1] = cpm[0] * cellw;
    out[(size_t)e * 3 + 2] = cpm[1] * cellw;
}

// One observation record from the row sums and the window cells (k_obs_cells): window
// sums in a fixed order (bitwise reproducible), status bits for the
// watchdog (1: non-finite norm, 2: drift beyond tol relative to scalar[1]).
__global__ void k_obs_reduce(const double* rowsum, const double* cells, int nx, int ny, double cell,
                             ObsWin w, const StepScalars* steps, const Clock* clock, int n_local,
                             double t_fixed, int64_t obs_every, int64_t cap, kd_obs* out,
                             const double* scalar, double tol, int* status) {
    __shared__ double red[256];
    const int tid = threadIdx.x;
    auto tree = [&](double v) -> double {
        red[tid] = v;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (tid < s) red[tid] += red[tid + s];
            __syncthreads();
        }
        const double r = red[0];
        __syncthreads();
        return r;
    };
    auto treemax = [&](double v) -> double {
        red[tid] = v;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (tid < s) red[tid] = fmax(red[tid], red[tid + s]);
            __syncthreads();
        }
        const double r = red[0];
        __syncthreads();
        return r;
    };
    double acc = 0.0;
    for (int i = tid; i < ny; i += blockDim.x) acc += rowsum[i];
    const double norm = tree(acc) * cell;
    double sums[2][3], mx[3] = {0, 0, 0};
    const int n0 = (w.ihi[0] - w.ilo[0] + 1) * (w.jhi[0] - w.jlo[0] + 1);
    const int n1 = (w.ihi[1] - w.ilo[1] + 1) * (w.jhi[1] - w.jlo[1] + 1);
    for (int wi = 0; wi < 2; ++wi) {
        const int nc = wi == 0 ? n0 : n1;
        const double* base = cells + (wi == 0 ? 0 : (size_t)n0 * 3);
        double a[3] = {0, 0, 0}, m[3] = {0, 0, 0};
        for (int q = tid; q < nc; q += blockDim.x) {
            const double* o = base + (size_t)q * 3;
            for (int k = 0; k < 3; ++k) { a[k] += o[k]; m[k] = fmax(m[k], o[k]); }
        }
        for (int k = 0; k < 3; ++k) sums[wi][k] = tree(a[k]);
        if (wi == 1)
            for (int k = 0; k < 3; ++k) mx[k] = treemax(m[k]);
    }
    if (tid == 0) {
        int64_t slot = 0;
        double t = t_fixed;
        if (clock) {
            const long long sidx = (clock->step - clock->base) + n_local;
            slot = sidx / obs_every - 1;
            t = steps[sidx].t;
        }
        const double* o = cells + (size_t)(n0 + n1) * 3;
        kd_obs r;
        r.t = t;
        r.norm = norm;
        r.pop_in = sums[0][0]; r.cp_in = sums[0][1]; r.cm_in = sums[0][2];
        r.pop_diff = sums[1][0]; r.cp_diff = sums[1][1]; r.cm_diff = sums[1][2];
        r.max_diff = mx[0]; r.cp_max_diff = mx[1]; r.cm_max_diff = mx[2];
        r.p_target = o[0]; r.cp_target = o[1]; r.cm_target = o[2];
        if (slot >= 0 && slot < cap) out[slot] = r;
        int st = 0;
        if (!isfinite(norm)) st |= 1;
        if (tol > 0.0 && fabs(norm - scalar[1]) > tol * scalar[1]) st |= 2;
        if (st && status) atomicOr(status, st);
    }
}

// Double-word form: n doubles -> n float pairs (h, l) in the same 8-byte slots (in place
// allowed), and back.
__global__ void k_dw_from_f64(void* buf, size_t n) {
    double* d = (double*)buf;
    float2* f = (float2*)buf;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const DW w = dw_from_double(d[i]);
        f[i] = make_float2(w.h, w.l);
    }
}
__global__ void k_dw_to_f64(const void* in, void* out, size_t n) {
    const float2* f = (const float2*)in;
    double* d = (double*)out;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float2 w = f[i];
        d[i] = dw_to_double(DW{w.x, w.y});
    }
}

// Layout conversion between the ABI's [P][4] Dirac order and the internal pair planes.
template <typename T>
__global__ void k_permute(const T* in, T* out, size_t npts, int to_internal) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < npts;
         i += (size_t)gridDim.x * blockDim.x) {
        for (int s = 0; s < 4; ++s) {
            const size_t o = slot_off(npts, i, s);
            const size_t d = i * 8 + 2 * perm_to_dirac(s);
            if (to_internal) { out[o] = in[d]; out[o + 1] = in[d + 1]; }
            else { out[d] = in[o]; out[d + 1] = in[o + 1]; }
        }
    }
}

// ---------------------------------------------------------------- host helpers ----

int grid_blocks(size_t n, int threads) { return (int)((n + threads - 1) / threads); }

int dw_from_f64_launch(kd_sim* s, void* buf, size_t n) {
    const int b = grid_blocks(n, 256) < 4096 ? grid_blocks(n, 256) : 4096;
    k_dw_from_f64<<<b, 256, 0, s->stream>>>(buf, n);
    KD_CUDA(cudaGetLastError());
    ++s->launches;
    return KD_OK;
}

// The state as FP64 (the internal pair-plane layout): psi itself, or for the double-word
// form an FP64 copy in s->view.
int state_view(kd_sim* s, const void** out) {
    if (!s->dw) { *out = s->psi; return KD_OK; }
    const size_t n = s->P * 8;
    const int b = grid_blocks(n, 256) < 4096 ? grid_blocks(n, 256) : 4096;
    k_dw_to_f64<<<b, 256, 0, s->stream>>>(s->psi, s->view, n);
    KD_CUDA(cudaGetLastError());
    ++s->launches;
    *out = s->view;
    return KD_OK;
}

// Double-word form: the per-x field table as float4 [2][nx][2] (each FP64 4-vector as two
// pairs of double-words), pi_x as float2, the twiddle tables of the double-word launch
// shapes, and the exp / sin-cos constant tables, from the FP64 values.
template <typename T> int upload_dw_tables(kd_sim* s, const std::vector<T>& xt, const std::vector<T>& kx) {
    const int nx = s->g.nx;
    std::vector<float4> xd(4 * (size_t)nx);
    for (size_t i = 0; i < 2 * (size_t)nx; ++i) {
        const DW a = dw_from_double((double)xt[4 * i]), b = dw_from_double((double)xt[4 * i + 1]);
        const DW c = dw_from_double((double)xt[4 * i + 2]), d = dw_from_double((double)xt[4 * i + 3]);
        xd[2 * i] = make_float4(a.h, a.l, b.h, b.l);
        xd[2 * i + 1] = make_float4(c.h, c.l, d.h, d.l);
    }
    KD_CUDA(cudaMemcpy(s->xtab, xd.data(), xd.size() * sizeof(float4), cudaMemcpyHostToDevice));
    std::vector<float2> kd2(nx);
    for (int i = 0; i < nx; ++i) {
        const DW a = dw_from_double((double)kx[i]);
        kd2[i] = make_float2(a.h, a.l);
    }
    KD_CUDA(cudaMemcpy(s->kxtab, kd2.data(), kd2.size() * sizeof(float2), cudaMemcpyHostToDevice));
    for (int ax = 0; ax < 2; ++ax) {
        const int logn = ax == 0 ? s->lx : s->ly;
        int entries = 0;
        KD_CUDA(build_twiddles_dw(logn, sweep_loge_dw(logn), s->tw_dw[ax], &entries, s->stream));
        if (entries > 2 * (1 << logn)) return fail(KD_ERR_CUDA, "twiddle table overflow");
    }
    DWConst K;
    for (int j = -13; j <= 13; ++j) {
        const DW sn = dw_from_double(sin(j / 16.0)), cs = dw_from_double(cos(j / 16.0));
        K.sc[j + 13] = make_float4(sn.h, sn.l, cs.h, cs.l);
    }
    for (int j = 0; j < 32; ++j) {
        const DW e = dw_from_double(exp2(-j / 32.0));
        K.e2[j] = make_float2(e.h, e.l);
    }
    KD_CUDA(cudaMemcpy(s->dwconst, &K, sizeof K, cudaMemcpyHostToDevice));
    KD_CUDA(cudaStreamSynchronize(s->stream));
    return KD_OK;
}

template <typename T> int upload_tables_t(kd_sim* s) {
    const int nx = s->g.nx;
    // stage-major twiddle tables, built on the device in FP64 (<= 2N entries of 16 B)
    // for both radix schedules a launch variant may use
    for (int ax = 0; ax < 2; ++ax)
        for (int le = 2; le <= 3; ++le) {
            int entries = 0;
            const int logn = ax == 0 ? s->lx : s->ly;
            void* dst = s->tw[ax][le - 2];
            KD_CUDA(sizeof(T) == 4 ? build_twiddles_f32(logn, le, dst, &entries, s->stream)
                                   : build_twiddles_f64(logn, le, dst, &entries, s->stream));
            if (entries > 2 * (1 << logn)) return fail(KD_ERR_CUDA, "twiddle table overflow");
        }
    // per-x field table (Eqs. Equation_of_Gaussian_beam, Phase_of_Gaussian_beam and w(x)),
    // two 4-vectors per column stored as [2][nx]: (Theta0 = (-k x + zeta) mod 2 pi,
    // x/(x_R w^2), w0/w, 1/w^2) and (1/w, cos zeta, sin zeta, cos k x), zeta = atan(x/x_R)
    std::vector<T> xt(8 * (size_t)nx, (T)0);
    const double dx = (s->g.x_max - s->g.x_min) / nx;
    const double k = s->f.k_L;
    for (int i = 0; i < nx; ++i) {
        const double x = s->g.x_min + i * dx;
        T* e0 = xt.data() + 4 * (size_t)i;          // first vector of column i
        T* e1 = xt.data() + 4 * ((size_t)nx + i);   // second vector of column i
        e1[3] = (T)cos(k * x);
        if (s->f.kind == KD_FIELD_GAUSS) {
            const double w0 = 1.0 / (k * s->f.epsilon);
            const double xR = k * w0 * w0 / 2.0;
            const double w = w0 * sqrt(1.0 + x * x / (xR * xR));
            const double zeta = atan(x / xR);
            e0[0] = (T)remainder(-k * x + zeta, 2.0 * kPi);
            e0[1] = (T)(x / (xR * w * w));
            e0[2] = (T)(w0 / w);
            e0[3] = (T)(1.0 / (w * w));
            e1[0] = (T)(1.0 / w);
            e1[1] = (T)cos(zeta);
            e1[2] = (T)sin(zeta);
        }
    }
    // kinetic x momentum per column
    std::vector<T> kx(nx);
    const double dpx = s->u.hbar * 2.0 * kPi / (s->g.x_max - s->g.x_min);
    for (int i = 0; i < nx; ++i) kx[i] = (T)(dpx * signed_index(i, nx) + s->f.p_shift_x);
    if (s->dw) return upload_dw_tables(s, xt, kx);
    KD_CUDA(cudaMemcpy(s->xtab, xt.data(), xt.size() * sizeof(T), cudaMemcpyHostToDevice));
    KD_CUDA(cudaMemcpy(s->kxtab, kx.data(), kx.size() * sizeof(T), cudaMemcpyHostToDevice));
    return KD_OK;
}

// ------------------------------------------------- precision form tables ---------
// 32-point DFT matrices for the tensor-core sweeps, in the kernels' shared-memory image:
// four 64 x 64 FP16 matrices (inverse hi, inverse lo, forward hi, forward lo), each in the
// dense no-swizzle K-major canonical layout (element (n, k) at byte
// (n / 8) 1024 + (k / 8) 128 + (n % 8) 16 + (k % 8) 2).  B[2k][2j] = c, B[2k][2j+1] = -s,
// B[2k+1][2j] = s, B[2k+1][2j+1] = c with c + i s = w_32^(jk) = exp(+-2 pi i jk / 32), all
// times 2^10 so that the lo parts are normal FP16 numbers.  For each of the 32 angles the
// lo parts of (c, s) are chosen among +-3 FP16 steps so that (c_hi + c_lo)^2 + (s_hi + s_lo)^2
// is closest to 2^20: the represented matrix is then unitary far below its rounding
// (an FP16 hi/lo matrix rounded to nearest loses ~1e-8 of the norm per product).
constexpr size_t kTcBImageBytes = 4 * 8192;

double h2d(__half h) { return (double)__half2float(h); }
__half step_half(__half h, int d) {
    __half_raw r = h;
    r.x = (unsigned short)(r.x + d);
    return __half(r);
}

void unit_pair_half(double c, double s, __half* ch, __half* cl, __half* sh, __half* sl) {
    *ch = __double2half(c);
    *sh = __double2half(s);
    const __half c0 = __double2half(c - h2d(*ch)), s0 = __double2half(s - h2d(*sh));
    *cl = c0;
    *sl = s0;
    const double target = 1024.0 * 1024.0;
    double best = 1e300;
    for (int dc = -3; dc <= 3; ++dc)
        for (int ds = -3; ds <= 3; ++ds) {
            // stepping the bits of a zero lo part would leave the finite numbers: keep it
            if ((h2d(c0) == 0.0 && dc) || (h2d(s0) == 0.0 && ds)) continue;
            const __half cc = step_half(c0, dc), ss = step_half(s0, ds);
            const double vc = h2d(*ch) + h2d(cc), vs = h2d(*sh) + h2d(ss);
            const double g = fabs(vc * vc + vs * vs - target) + 1e-6 * (fabs(vc - c) + fabs(vs - s));
            if (!isfinite(vc) || !isfinite(vs)) continue;
            if (g < best) { best = g; *cl = cc; *sl = ss; }
        }
}

int upload_tc_tables(kd_sim* s) {
    std::vector<__half> img(kTcBImageBytes / 2);
    for (int dir = 0; dir < 2; ++dir) {            // 0: inverse (+), 1: forward (-)
        const double sg = dir == 0 ? 1.0 : -1.0;
        __half ch[32], cl[32], sh[32], sl[32];
        for (int m = 0; m < 32; ++m) {
            const double th = 2.0 * kPi * m / 32.0;
            unit_pair_half(1024.0 * cos(th), sg * 1024.0 * sin(th), &ch[m], &cl[m], &sh[m], &sl[m]);
        }
        for (int part = 0; part < 2; ++part) {     // hi, lo
            __half* mat = img.data() + (size_t)(2 * dir + part) * 4096;
            for (int k = 0; k < 32; ++k)
                for (int j = 0; j < 32; ++j) {
                    const int m = (j * k) & 31;
                    const __half c = part ? cl[m] : ch[m], sn = part ? sl[m] : sh[m];
                    const __half msn = __hneg(sn);
                    const __half v[4] = {c, msn, sn, c};   // (2k, 2j), (2k, 2j+1), (2k+1, 2j), (2k+1, 2j+1)
                    for (int q = 0; q < 4; ++q) {
                        const int n = 2 * k + (q >> 1), kk = 2 * j + (q & 1);
                        mat[((n >> 3) * 1024 + (kk >> 3) * 128 + (n & 7) * 16 + (kk & 7) * 2) / 2] = v[q];
                    }
                }
        }
    }
    KD_CUDA(cudaMemcpy(s->tc_b, img.data(), kTcBImageBytes, cudaMemcpyHostToDevice));
    // twiddles w_1024^m in FP32, the pair within +-3 ulps with |w| closest to 1
    std::vector<float2> tw(1024);
    for (int m = 0; m < 1024; ++m) {
        const double th = 2.0 * kPi * m / 1024.0;
        const double c = cos(th), sn = sin(th);
        float bc = (float)c, bs = (float)sn;
        double best = 1e300;
        float ci = (float)c;
        for (int k = 0; k < 3; ++k) ci = nextafterf(ci, -INFINITY);
        for (int dc = -3; dc <= 3; ++dc, ci = nextafterf(ci, INFINITY)) {
            float si = (float)sn;
            for (int k = 0; k < 3; ++k) si = nextafterf(si, -INFINITY);
            for (int ds = -3; ds <= 3; ++ds, si = nextafterf(si, INFINITY)) {
                const double g = fabs((double)ci * ci + (double)si * si - 1.0) +
                                 1e-3 * (fabs(ci - c) + fabs(si - sn));
                if (g < best) { best = g; bc = ci; bs = si; }
            }
        }
        tw[m] = make_float2(bc, bs);
    }
    KD_CUDA(cudaMemcpy(s->tc_tw, tw.data(), 1024 * sizeof(float2), cudaMemcpyHostToDevice));
    const float one[4] = {1.0f, 1.0f, 1.0f, 1.0f};
    KD_CUDA(cudaMemcpy(s->tc_scale, one, sizeof one, cudaMemcpyHostToDevice));
    return KD_OK;
}

// Tables that depend on dt: the kinetic table (device, FP64) and the per-row
// (pi_y, cos, sin of the frame phase box_vy p_y dt / hbar).
// Rounded (cos(ph) - 1, sin(ph)) with |1 + f| = 1 as closely as the precision allows:
// for FP32 the pair within 3 ulps of the rounded values with the smallest modulus error.
template <typename T> void unit_phase(double ph, T* fx, T* fy) {
    const double sh = sin(0.5 * ph);
    const double x = -2.0 * sh * sh, y = sin(ph);
    *fx = (T)x;
    *fy = (T)y;
    if (sizeof(T) != 4) return;
    double best = 1e300;
    float xi = (float)x;
    for (int k = 0; k < 3; ++k) xi = nextafterf(xi, -INFINITY);
    for (int dx = -3; dx <= 3; ++dx, xi = nextafterf(xi, INFINITY)) {
        float yi = (float)y;
        for (int k = 0; k < 3; ++k) yi = nextafterf(yi, -INFINITY);
        for (int dy = -3; dy <= 3; ++dy, yi = nextafterf(yi, INFINITY)) {
            const double g = fabs(2.0 * xi + (double)xi * xi + (double)yi * yi) +
                             1e-3 * fabs(atan2((double)yi, 1.0 + xi) - ph);
            if (g < best) { best = g; *fx = (T)xi; *fy = (T)yi; }
        }
    }
}

// Tables that depend on dt: the per-row (pi_y, cos(phi) - 1, sin(phi)) of the frame phase
// phi = box_vy p_y dt / hbar and the kinetic table (device, FP64).
template <typename T> int build_dt_tables_t(kd_sim* s, double dt) {
    const int nx = s->g.nx, ny = s->g.ny;
    const double dpx = s->u.hbar * 2.0 * kPi / (s->g.x_max - s->g.x_min);
    const double dpy = s->u.hbar * 2.0 * kPi / (s->g.y_max - s->g.y_min);
    const double mc2 = s->u.m * s->u.c * s->u.c;
    std::vector<T> ky(4 * (size_t)ny);
    for (int j = 0; j < ny; ++j) {
        const double py = dpy * signed_index(j, ny);
        ky[4 * j] = (T)(py + s->f.p_shift_y);
        unit_phase<T>(s->f.box_vy * py * dt / s->u.hbar, &ky[4 * j + 1], &ky[4 * j + 2]);
        ky[4 * j + 3] = (T)0;
    }
    std::vector<float4> kyd;
    if (s->dw) {   // per row (pi_y | cos phi - 1) and (sin phi | 0) as double-words
        kyd.resize(2 * (size_t)ny);
        for (int j = 0; j < ny; ++j) {
            const DW a = dw_from_double((double)ky[4 * j]), b = dw_from_double((double)ky[4 * j + 1]);
            const DW c = dw_from_double((double)ky[4 * j + 2]);
            kyd[2 * j] = make_float4(a.h, a.l, b.h, b.l);
            kyd[2 * j + 1] = make_float4(c.h, c.l, 0.0f, 0.0f);
        }
        KD_CUDA(cudaMemcpyAsync(s->kytab, kyd.data(), kyd.size() * sizeof(float4), cudaMemcpyHostToDevice,
                                s->stream));
    } else {
        KD_CUDA(cudaMemcpyAsync(s->kytab, ky.data(), ky.size() * sizeof(T), cudaMemcpyHostToDevice,
                                s->stream));
    }
    k_ktab<T><<<grid_blocks(s->P, 256), 256, 0, s->stream>>>(
        (T*)s->ktab, nx, ny, dpx, dpy, s->f.p_shift_x, s->f.p_shift_y, s->u.c, mc2, s->u.hbar, dt,
        (const T*)s->kxtab, (const T*)s->kytab, s->u.m * s->u.c);
    KD_CUDA(cudaGetLastError());
    ++s->launches;
    if (s->dw) {   // (C - 1)/P and c S/P as double-words, in place
        int rc = dw_from_f64_launch(s, s->ktab, 2 * s->P);
        if (rc) return rc;
    }
    KD_CUDA(cudaStreamSynchronize(s->stream));
    s->ktab_dt = dt;
    return KD_OK;
}

int build_dt_tables(kd_sim* s, double dt) {
    return s->prec == KD_FP64 ? build_dt_tables_t<double>(s, dt) : build_dt_tables_t<float>(s, dt);
}

// One fused sweep of the state (the simulation's own form), or, with view = true, an FP64
// transform of the FP64 view of the state (read-outs of the double-word form).
SweepArgs make_args(const kd_sim* s, int axis, int op, const void* in, void* out, int n_local,
                    double tau, bool view) {
    SweepArgs a{};
    a.in = in;
    a.out = out;
    a.nx = s->g.nx;
    a.ny = s->g.ny;
    a.op = op;
    const int logn = axis == AXIS_X ? s->lx : s->ly;
    const int var = s->prec == KD_FP64 ? 0 : s->var[axis];
    const bool dwk = s->dw && !view;   // the double-word kernels
    a.tw = dwk ? s->tw_dw[axis] : s->tw[axis][sweep_loge(s->prec == KD_FP64, axis, logn, var) - 2];
    a.dwconst = s->dwconst;
    a.clock = s->clock;
    a.steps = s->steps;
    a.n_local = n_local;
    a.kind = s->f.kind;
    a.longitudinal = s->f.longitudinal;
    a.kappa = tau * s->u.m * s->u.c * s->u.c / s->u.hbar;
    a.eps4 = 4.0 * s->f.epsilon;
    a.y_min = s->g.y_min;
    a.dy = (s->g.y_max - s->g.y_min) / s->g.ny;
    a.xtab = s->xtab;
    a.ktab = s->ktab;
    a.kxtab = s->kxtab;
    a.kytab = s->kytab;
    a.mc = s->u.m * s->u.c;
    a.kappa_f = (float)a.kappa;
    a.eps4_f = (float)a.eps4;
    a.dy_f = (float)a.dy;
    a.mc_f = (float)a.mc;
    a.invP = 1.0 / ((double)s->g.nx * (double)s->g.ny);
    a.invP_f = (float)a.invP;
    a.tc_b = s->tc_b;
    a.tc_tw = s->tc_tw;
    a.tc_scale = s->tc_scale;
    a.status = s->status;
    a.tc_fault = s->tc_fault;
    return a;
}

cudaError_t sweep(kd_sim* s, int axis, int shape, int op, const void* in, void* out, int n_local,
                  double tau, bool view = false) {
    const SweepArgs a = make_args(s, axis, op, in, out, n_local, tau, view);
    const int logn = axis == AXIS_X ? s->lx : s->ly;
    const int var = s->prec == KD_FP64 ? 0 : s->var[axis];
    const bool dwk = s->dw && !view;
    ++s->launches;
    if (s->tc && shape == SHAPE_F1F2 && tc_supported(logn)) return launch_tc_sweep(axis, a, s->stream);
    if (dwk) return launch_sweep_dw(axis, shape, logn, a, s->stream);
    return s->prec == KD_FP64 ? launch_sweep_f64(axis, shape, logn, a, s->stream)
                              : launch_sweep_f32(var, axis, shape, logn, a, s->stream);
}

// ------------------------------------------------------------------ autotuner ------
// Process-wide record of tuned launch variants per device, grid and field kind, so that
// simulations of the same shape (the members of a batch, repeated runs) are timed once.
struct TuneKey {
    int device, nx, ny, kind, longitudinal, tc;
    bool operator<(const TuneKey& o) const {
        return std::tie(device, nx, ny, kind, longitudinal, tc) <
               std::tie(o.device, o.nx, o.ny, o.kind, o.longitudinal, o.tc);
    }
};
struct TuneResult {
    int var[2];
    float ms[2][KD_SWEEP_VARIANTS];
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneResult> g_tune;

// KD_ERR_ARG when the simulation's stream is being captured (for calls that launch and
// synchronise outside the step loop)
int reject_capture(kd_sim* s, const char* what) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s->stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        return KD_OK;
    }
    if (cs != cudaStreamCaptureStatusNone)
        return fail(KD_ERR_ARG, "%s: the simulation's stream is being captured", what);
    return KD_OK;
}

// First launch of every sweep shape of the current variants outside any stream capture
// (sets the kernels' shared-memory attributes); reads psi, writes only the work buffer.
int warm_variants(kd_sim* s) {
    const int shapes[3] = {SHAPE_F1, SHAPE_F2, SHAPE_F1F2};
    for (int ax = 0; ax < 2; ++ax)
        for (int sh : shapes) {
            cudaError_t el = sweep(s, ax, sh, OP_NONE, s->psi, s->work, 0, 0.0);
            if (el != cudaSuccess) return fail(KD_ERR_CUDA, "sweep launch: %s", cudaGetErrorString(el));
        }
    KD_CUDA(cudaStreamSynchronize(s->stream));
    return KD_OK;
}

// Mean time per launch (ms) of `reps` back-to-back full sweeps of one axis with the
// step's pointwise op, psi -> work (the state is not modified).  The launches are
// captured into a graph and replayed twice after one warm replay, so that host launch
// overhead does not enter.
int time_sweep(kd_sim* s, int axis, int reps, double dt, float* ms) {
    cudaStream_t user = s->stream;
    s->stream = s->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        s->stream = user;
        return fail(KD_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
    }
    cudaError_t el = cudaSuccess;
    for (int i = 0; i < reps && el == cudaSuccess; ++i)
        el = axis == AXIS_X ? sweep(s, AXIS_X, SHAPE_F1F2, OP_POTENTIAL, s->psi, s->work, 0, dt)
                            : sweep(s, AXIS_Y, SHAPE_F1F2, OP_KINETIC, s->psi, s->work, 0, 0.0);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s->stream, &graph);
    s->stream = user;
    if (el != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(KD_ERR_CUDA, "tuning capture: %s", cudaGetErrorString(el != cudaSuccess ? el : e));
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(KD_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int rc = KD_OK;
    if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess ||
        cudaGraphLaunch(exec, s->stream) != cudaSuccess ||
        cudaEventRecord(ev[0], s->stream) != cudaSuccess ||
        cudaGraphLaunch(exec, s->stream) != cudaSuccess ||
        cudaGraphLaunch(exec, s->stream) != cudaSuccess ||
        cudaEventRecord(ev[1], s->stream) != cudaSuccess ||
        cudaEventSynchronize(ev[1]) != cudaSuccess ||
        cudaEventElapsedTime(ms, ev[0], ev[1]) != cudaSuccess)
        rc = fail(KD_ERR_CUDA, "tuning run failed: %s", cudaGetErrorString(cudaGetLastError()));
    else
        *ms /= (float)(2 * reps);
    s->launches += 2 * (int64_t)reps;   // replays beyond the one counted at capture
    for (cudaEvent_t v : ev)
        if (v) cudaEventDestroy(v);
    cudaGraphExecDestroy(exec);
    return rc;
}

#define KD_LAUNCH(expr)                                                                  \
    do {                                                                                 \
        cudaError_t e_ = (expr);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(KD_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_));          \
    } while (0)

int rowsum_launch(kd_sim* s, const void* psi) {   // psi: FP64 for KD_FP64 and KD_DW (view)
    if (s->prec == KD_FP64) k_rowsum<double><<<s->g.ny, 256, 0, s->stream>>>((const double*)psi, s->g.nx, s->g.ny, s->rowsum);
    else k_rowsum<float><<<s->g.ny, 256, 0, s->stream>>>((const float*)psi, s->g.nx, s->g.ny, s->rowsum);
    KD_CUDA(cudaGetLastError());
    ++s->launches;
    return KD_OK;
}

int ensure_md(kd_sim* s) {
    if (!s->md) KD_CUDA(dev_alloc((void**)&s->md, s->P * 3 * sizeof(double)));
    return KD_OK;
}

// psi (position space) -> work = DFT psi (internal order) -> md
int momentum_density_launch(kd_sim* s, int basis, double* out) {
    const double dpx = s->u.hbar * 2.0 * kPi / (s->g.x_max - s->g.x_min);
    const double dpy = s->u.hbar * 2.0 * kPi / (s->g.y_max - s->g.y_min);
    const double mc2 = s->u.m * s->u.c * s->u.c;
    const void* st = nullptr;
    int rc = state_view(s, &st);
    if (rc) return rc;
    KD_LAUNCH(sweep(s, AXIS_X, SHAPE_F2, OP_NONE, st, s->work, 0, 0.0, true));
    KD_LAUNCH(sweep(s, AXIS_Y, SHAPE_F1, OP_NONE, s->work, s->work, 0, 0.0, true));
    const double cellw = dxdy(s) / (double)s->P;
    if (s->prec == KD_FP64)
        k_momentum_density<double><<<grid_blocks(s->P, 256), 256, 0, s->stream>>>(
            (const double*)s->work, s->g.nx, s->g.ny, dpx, dpy, s->f.p_shift_x, s->f.p_shift_y,
            s->u.c, mc2, basis, cellw, out);
    else
        k_momentum_density<float><<<grid_blocks(s->P, 256), 256, 0, s->stream>>>(
            (const float*)s->work, s->g.nx, s->g.ny, dpx, dpy, s->f.p_shift_x, s->f.p_shift_y,
            s->u.c, mc2, basis, cellw, out);
    KD_CUDA(cudaGetLastError());
    ++s->launches;
    return KD_OK;
}

// Window of signed indices around the grid point nearest to a kinetic momentum:
// centre round((pi - p_shift)/dp), half width floor(h/dp), clamped to the grid.
int window_axis(double pic, double shift, double dp, double h, int n, int* lo, int* hi, int* c) {
    const double v = floor((pic - shift) / dp + 0.5);
    if (!(v >= -(double)(n / 2) && v <= (double)(n / 2 - 1))) return -1;
    const int cc = (int)v;
    const int w = (int)floor(h / dp + 1e-9);
    if (w < 0) return -1;
    *c = cc;
    *lo = cc - w < -(n / 2) ? -(n / 2) : cc - w;
    *hi = cc + w > n / 2 - 1 ? n / 2 - 1 : cc + w;
    return 0;
}

int make_window(const kd_sim* s, const kd_obs_spec* sp, ObsWin* w) {
    if (!(sp->half_width >= 0.0)) return fail(KD_ERR_ARG, "obs spec half_width must be >= 0");
    if (sp->basis != 0 && sp->basis != 1) return fail(KD_ERR_ARG, "obs spec basis must be 0 or 1");
    const double dpx = s->u.hbar * 2.0 * kPi / (s->g.x_max - s->g.x_min);
    const double dpy = s->u.hbar * 2.0 * kPi / (s->g.y_max - s->g.y_min);
    const double cx[3] = {sp->p_in_x, sp->p_diff_x, sp->target_x};
    const double cy[3] = {sp->p_in_y, sp->p_diff_y, sp->target_y};
    for (int k = 0; k < 3; ++k) {
        int lo, hi, c, lo2, hi2, c2;
        if (window_axis(cx[k], s->f.p_shift_x, dpx, sp->half_width, s->g.nx, &lo, &hi, &c) ||
            window_axis(cy[k], s->f.p_shift_y, dpy, sp->half_width, s->g.ny, &lo2, &hi2, &c2))
            return fail(KD_ERR_ARG, "obs spec momentum %d lies outside the momentum grid", k);
        if (k < 2) { w->ilo[k] = lo; w->ihi[k] = hi; w->jlo[k] = lo2; w->jhi[k] = hi2; }
        else { w->it = c; w->jt = c2; }
    }
    return KD_OK;
}

// Observation of the position-space state psi: row sums, forward 2D FFT into work, the
// window cells' momentum-space values (into the md scratch), window reduction into
// out[slot].
int observe_launch(kd_sim* s, const ObsWin& w, int basis, bool in_step, int n_local, double t_fixed,
                   int64_t obs_every, int64_t cap, kd_obs* out) {
    int rc = ensure_md(s);
    if (rc) return rc;
    const void* st = nullptr;
    rc = state_view(s, &st);
    if (rc) return rc;
    rc = rowsum_launch(s, st);
    if (rc) return rc;
    KD_LAUNCH(sweep(s, AXIS_X, SHAPE_F2, OP_NONE, st, s->work, 0, 0.0, true));
    KD_LAUNCH(sweep(s, AXIS_Y, SHAPE_F1, OP_NONE, s->work, s->work, 0, 0.0, true));
    {
        const double dpx = s->u.hbar * 2.0 * kPi / (s->g.x_max - s->g.x_min);
        const double dpy = s->u.hbar * 2.0 * kPi / (s->g.y_max - s->g.y_min);
        const double mc2 = s->u.m * s->u.c * s->u.c;
        const double cellw = dxdy(s) / (double)s->P;
        const int ncell = (w.ihi[0] - w.ilo[0] + 1) * (w.jhi[0] - w.jlo[0] + 1) +
                          (w.ihi[1] - w.ilo[1] + 1) * (w.jhi[1] - w.jlo[1] + 1) + 1;
        if (s->prec == KD_FP64)
            k_obs_cells<double><<<grid_blocks(ncell, 128), 128, 0, s->stream>>>(
                (const double*)s->work, s->g.nx, s->g.ny, dpx, dpy, s->f.p_shift_x, s->f.p_shift_y,
                s->u.c, mc2, basis, cellw, w, s->md);
        else
            k_obs_cells<float><<<grid_blocks(ncell, 128), 128, 0, s->stream>>>(
                (const float*)s->work, s->g.nx, s->g.ny, dpx, dpy, s->f.p_shift_x, s->f.p_shift_y,
                s->u.c, mc2, basis, cellw, w, s->md);
        KD_CUDA(cudaGetLastError());
        ++s->launches;
    }
    k_obs_reduce<<<1, 256, 0, s->stream>>>(s->rowsum, s->md, s->g.nx, s->g.ny, dxdy(s), w, s->steps,
                                           in_step ? s->clock : nullptr, n_local, t_fixed,
                                           obs_every, cap, out, s->scalar, s->watch_tol, s->status);
    KD_CUDA(cudaGetLastError());
    ++s->launches;
    return KD_OK;
}

int ensure_steps(kd_sim* s, int64_t n) {
    if (n + 1 <= s->steps_cap) return KD_OK;
    clear_graphs(s);
    if (s->steps) cudaFree(s->steps);
    s->steps = nullptr;
    s->steps_cap = 0;   // no buffer until the allocation below succeeds
    int64_t cap = 1024;
    while (cap < n + 1) cap *= 2;
    KD_CUDA(dev_alloc((void**)&s->steps, cap * sizeof(StepScalars)));
    s->steps_cap = cap;
    return KD_OK;
}

int ensure_obs(kd_sim* s, int64_t n) {
    if (n <= s->obs_dev_cap) return KD_OK;
    clear_graphs(s);
    if (s->obs_dev) cudaFree(s->obs_dev);
    s->obs_dev = nullptr;
    s->obs_dev_cap = 0;   // no buffer until the allocation below succeeds
    int64_t cap = 16;
    while (cap < n) cap *= 2;
    KD_CUDA(dev_alloc((void**)&s->obs_dev, cap * sizeof(kd_obs)));
    s->obs_dev_cap = cap;
    return KD_OK;
}

// Enqueues one chunk of `chunk` steps starting from the "open" state (x sweep of the
// opening half already applied): chunk-1 merged steps, then the chunk's last step,
// which closes (last chunk, or an observation point) or merges.
int enqueue_chunk(kd_sim* s, double dt, int chunk, bool last, bool obs, const ObsWin& w,
                  int64_t obs_every, int64_t cap) {
    for (int i = 1; i <= chunk; ++i) {
        KD_LAUNCH(sweep(s, AXIS_Y, SHAPE_F1F2, OP_KINETIC, s->psi, s->psi, 0, 0.0));
        if (i < chunk) {
            KD_LAUNCH(sweep(s, AXIS_X, SHAPE_F1F2, OP_POTENTIAL, s->psi, s->psi, i, dt));
        } else if (last || obs) {
            KD_LAUNCH(sweep(s, AXIS_X, SHAPE_F1, OP_POTENTIAL, s->psi, s->psi, i, 0.5 * dt));
            if (obs) {
                int rc = observe_launch(s, w, s->spec.basis, true, i, 0.0, obs_every, cap, s->obs_dev);
                if (rc) return rc;
            }
            if (!last) KD_LAUNCH(sweep(s, AXIS_X, SHAPE_F2, OP_POTENTIAL, s->psi, s->psi, i, 0.5 * dt));
        } else {
            KD_LAUNCH(sweep(s, AXIS_X, SHAPE_F1F2, OP_POTENTIAL, s->psi, s->psi, i, dt));
        }
    }
    k_advance_clock<<<1, 1, 0, s->stream>>>(s->clock, chunk);
    KD_CUDA(cudaGetLastError());
    ++s->launches;
    return KD_OK;
}

int run_chunk(kd_sim* s, double dt, int chunk, bool last, bool obs, const ObsWin& w,
              int64_t obs_every, int64_t cap) {
    GraphKey key{chunk, last ? 1 : 0, obs ? 1 : 0};
    auto it = s->graphs.find(key);
    if (it == s->graphs.end()) {
        // capture on the private stream, launch on the simulation's stream
        cudaStream_t user = s->stream;
        s->stream = s->cap_stream;
        cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            s->stream = user;
            return fail(KD_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
        }
        const int64_t before = s->launches;
        int rc = enqueue_chunk(s, dt, chunk, last, obs, w, obs_every, cap);
        const int64_t nodes = s->launches - before;
        s->launches = before;
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(s->stream, &graph);
        s->stream = user;
        if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
        if (e != cudaSuccess) return fail(KD_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(KD_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        it = s->graphs.emplace(key, std::make_pair(exec, nodes)).first;
    }
    KD_CUDA(cudaGraphLaunch(it->second.first, s->stream));
    s->launches += it->second.second;
    return KD_OK;
}

uint64_t fnv(uint64_t h, const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ull; }
    return h;
}

uint64_t param_hash(const kd_sim* s) {
    uint64_t h = 1469598103934665603ull;
    h = fnv(h, &s->u, sizeof s->u);
    h = fnv(h, &s->g, sizeof s->g);
    h = fnv(h, &s->f, sizeof s->f);
    h = fnv(h, &s->prec, sizeof s->prec);
    if (s->dw) h = fnv(h, &s->dw, sizeof s->dw);
    return h;
}

struct StateHeader {
    uint32_t magic, version;
    int32_t nx, ny, prec, pad;
    uint64_t hash;
    double t0, dt_clock;
    int64_t step;
    uint64_t payload;
};

int check_sim(kd_sim* s) {
    if (!s) return fail(KD_ERR_ARG, "null simulation");
    cudaError_t e = cudaSetDevice(s->device);
    if (e != cudaSuccess) return fail(KD_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return KD_OK;
}

int copy_in(kd_sim* s, const void* psi, int32_t where) {
    const size_t bytes = spinor_bytes(s);
    const void* src = psi;
    if (where == KD_HOST) {
        KD_CUDA(cudaMemcpyAsync(s->work, psi, bytes, cudaMemcpyHostToDevice, s->stream));
        src = s->work;
    }
    const int blocks = grid_blocks(s->P, 256) < 4096 ? grid_blocks(s->P, 256) : 4096;
    if (s->prec == KD_FP64) k_permute<double><<<blocks, 256, 0, s->stream>>>((const double*)src, (double*)s->psi, s->P, 1);
    else k_permute<float><<<blocks, 256, 0, s->stream>>>((const float*)src, (float*)s->psi, s->P, 1);
    KD_CUDA(cudaGetLastError());
    ++s->launches;
    if (s->dw) {
        int rc = dw_from_f64_launch(s, s->psi, s->P * 8);
        if (rc) return rc;
    }
    if (where == KD_HOST) KD_CUDA(cudaStreamSynchronize(s->stream));
    return KD_OK;
}

int copy_out(kd_sim* s, void* psi, int32_t where) {
    const size_t bytes = spinor_bytes(s);
    void* dst = where == KD_HOST ? s->work : psi;
    const int blocks = grid_blocks(s->P, 256) < 4096 ? grid_blocks(s->P, 256) : 4096;
    const void* st = nullptr;
    int rc = state_view(s, &st);
    if (rc) return rc;
    if (s->prec == KD_FP64) k_permute<double><<<blocks, 256, 0, s->stream>>>((const double*)st, (double*)dst, s->P, 0);
    else k_permute<float><<<blocks, 256, 0, s->stream>>>((const float*)st, (float*)dst, s->P, 0);
    KD_CUDA(cudaGetLastError());
    ++s->launches;
    if (where == KD_HOST) {
        KD_CUDA(cudaMemcpyAsync(psi, s->work, bytes, cudaMemcpyDeviceToHost, s->stream));
        KD_CUDA(cudaStreamSynchronize(s->stream));
    }
    return KD_OK;
}

}  // namespace

// =================================================================== public ABI ===

extern "C" {

const char* kd_last_error(void) { return g_err.c_str(); }

int kd_version(void) { return 100; }

int kd_create(const kd_units* units, const kd_grid* grid, const kd_field* field, int32_t precision,
              void* cuda_stream, kd_sim** out) {
    g_err.clear();
    if (!units || !grid || !field || !out) return fail(KD_ERR_ARG, "null argument");
    *out = nullptr;
    if (precision != KD_FP64 && precision != KD_FP32 && precision != KD_FP32_TC && precision != KD_DW)
        return fail(KD_ERR_ARG, "precision must be KD_FP64, KD_FP32, KD_FP32_TC or KD_DW");
    if (!pow2_in_range(grid->nx) || !pow2_in_range(grid->ny))
        return fail(KD_ERR_UNSUPPORTED_SIZE, "nx=%d ny=%d: need powers of two in [4, 4096]", grid->nx, grid->ny);
    if (!(grid->x_max > grid->x_min) || !(grid->y_max > grid->y_min) || !isfinite(grid->x_min) ||
        !isfinite(grid->x_max) || !isfinite(grid->y_min) || !isfinite(grid->y_max))
        return fail(KD_ERR_ARG, "box limits must be finite with max > min");
    if (!(units->m > 0) || !(units->c > 0) || !(units->hbar > 0) || !isfinite(units->m) ||
        !isfinite(units->c) || !isfinite(units->hbar))
        return fail(KD_ERR_ARG, "units m, c, hbar must be positive and finite");
    if (field->kind < KD_FIELD_NONE || field->kind > KD_FIELD_GAUSS) return fail(KD_ERR_ARG, "unknown field kind %d", field->kind);
    const double fv[] = {field->a0, field->k_L, field->epsilon, field->env_T, field->phase0,
                         field->p_shift_x, field->p_shift_y, field->box_vy};
    for (double v : fv)
        if (!isfinite(v)) return fail(KD_ERR_ARG, "field parameters must be finite");
    if (field->kind != KD_FIELD_NONE && !(field->k_L > 0)) return fail(KD_ERR_ARG, "k_L must be > 0");
    if (field->kind == KD_FIELD_GAUSS && !(field->epsilon > 0)) return fail(KD_ERR_ARG, "epsilon must be > 0 for the Gaussian beam");
    if (field->env_T < 0) return fail(KD_ERR_ARG, "env_T must be >= 0");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(KD_ERR_CUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
    int ndev = 0;
    e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev <= 0) return fail(KD_ERR_CUDA, "no usable CUDA device: %s", cudaGetErrorString(e));

    kd_sim* s = new kd_sim();
    s->u = *units;
    s->g = *grid;
    s->f = *field;
    s->tc = precision == KD_FP32_TC;       // FP32 storage and tables, tensor-core sweeps
    s->dw = precision == KD_DW;            // float-pair storage and tables, FP64 read-outs
    s->prec = s->tc ? KD_FP32 : (s->dw ? KD_FP64 : precision);
    s->tsize = s->prec == KD_FP64 ? 8 : 4;
    s->stream = (cudaStream_t)cuda_stream;
    s->device = dev;
    s->lx = ilog2(grid->nx);
    s->ly = ilog2(grid->ny);
    s->P = (size_t)grid->nx * grid->ny;
    auto bail = [&](int rc) { kd_destroy(s); return rc; };
#define KD_ALLOC(ptr, bytes)                                                             \
    do {                                                                                 \
        cudaError_t ea_ = dev_alloc((void**)&(ptr), (bytes));                            \
        if (ea_ != cudaSuccess)                                                          \
            return bail(fail(KD_ERR_NOMEM, "cudaMalloc(%zu): %s", (size_t)(bytes), cudaGetErrorString(ea_))); \
    } while (0)
    if (cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(KD_ERR_CUDA, "stream create failed"));
    for (cudaEvent_t& ev : s->ahead)
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
            return bail(fail(KD_ERR_CUDA, "event create failed"));
    KD_ALLOC(s->psi, spinor_bytes(s));
    KD_ALLOC(s->work, spinor_bytes(s));
    for (int le = 0; le < 2; ++le) {
        KD_ALLOC(s->tw[AXIS_X][le], 2 * (size_t)grid->nx * 16);
        KD_ALLOC(s->tw[AXIS_Y][le], 2 * (size_t)grid->ny * 16);
    }
    KD_ALLOC(s->xtab, 8 * (size_t)grid->nx * s->tsize);
    KD_ALLOC(s->kxtab, (size_t)grid->nx * s->tsize);
    KD_ALLOC(s->kytab, 4 * (size_t)grid->ny * s->tsize);
    KD_ALLOC(s->ktab, s->P * cbytes(s));
    KD_ALLOC(s->clock, sizeof(Clock));
    KD_ALLOC(s->rowsum, (size_t)grid->ny * sizeof(double));
    KD_ALLOC(s->scalar, 4 * sizeof(double));
    KD_ALLOC(s->status, sizeof(int));
    if (s->dw) {
        KD_ALLOC(s->tw_dw[AXIS_X], 2 * (size_t)grid->nx * 16);
        KD_ALLOC(s->tw_dw[AXIS_Y], 2 * (size_t)grid->ny * 16);
        KD_ALLOC(s->dwconst, sizeof(DWConst));
        KD_ALLOC(s->view, spinor_bytes(s));
    }
    if (s->tc) {
        KD_ALLOC(s->tc_b, kTcBImageBytes);
        KD_ALLOC(s->tc_tw, 1024 * sizeof(float2));
        KD_ALLOC(s->tc_scale, 4 * sizeof(float));
    }
#undef KD_ALLOC
    if (cudaMemset(s->psi, 0, spinor_bytes(s)) != cudaSuccess ||
        cudaMemset(s->clock, 0, sizeof(Clock)) != cudaSuccess ||
        cudaMemset(s->scalar, 0, 4 * sizeof(double)) != cudaSuccess ||
        cudaMemset(s->status, 0, sizeof(int)) != cudaSuccess)
        return bail(fail(KD_ERR_CUDA, "memset failed"));
    int rc = s->prec == KD_FP64 ? upload_tables_t<double>(s) : upload_tables_t<float>(s);
    if (rc) return bail(rc);
    if (s->tc) {
        rc = upload_tc_tables(s);
        if (rc) return bail(rc);
    }
    rc = warm_variants(s);
    if (rc) return bail(rc);
    *out = s;
    return KD_OK;
}

void kd_destroy(kd_sim* s) {
    if (!s) return;
    cudaSetDevice(s->device);
    cudaStreamSynchronize(s->stream);
    clear_graphs(s);
    void* bufs[] = {s->psi, s->work, s->tw[0][0], s->tw[0][1], s->tw[1][0], s->tw[1][1], s->xtab,
                    s->kxtab, s->kytab, s->ktab, s->clock, s->steps, s->rowsum, s->md, s->scalar,
                    s->obs_dev, s->status, s->tc_b, s->tc_tw, s->tc_scale, s->tw_dw[0], s->tw_dw[1],
                    s->dwconst, s->view};
    for (void* b : bufs)
        if (b) cudaFree(b);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    for (cudaEvent_t ev : s->ahead)
        if (ev) cudaEventDestroy(ev);
    delete s;
}

int kd_set_spinor(kd_sim* s, const void* psi, int32_t where) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (!psi || (where != KD_HOST && where != KD_DEVICE)) return fail(KD_ERR_ARG, "bad spinor pointer or where");
    return copy_in(s, psi, where);
}

int kd_get_spinor(kd_sim* s, void* psi, int32_t where) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (!psi || (where != KD_HOST && where != KD_DEVICE)) return fail(KD_ERR_ARG, "bad spinor pointer or where");
    return copy_out(s, psi, where);
}

int kd_set_time(kd_sim* s, double t) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (!isfinite(t)) return fail(KD_ERR_ARG, "time must be finite");
    s->t0 = t;
    s->step = 0;
    clear_graphs(s);
    return KD_OK;
}

int kd_get_time(kd_sim* s, double* t, int64_t* steps_done) {
    if (!s) return fail(KD_ERR_ARG, "null simulation");
    if (t) *t = s->t0 + (double)s->step * s->dt_clock;
    if (steps_done) *steps_done = s->step;
    return KD_OK;
}

int kd_set_obs_spec(kd_sim* s, const kd_obs_spec* spec) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (!spec) return fail(KD_ERR_ARG, "null spec");
    ObsWin w;
    rc = make_window(s, spec, &w);
    if (rc) return rc;
    s->spec = *spec;
    s->has_spec = true;
    clear_graphs(s);
    return KD_OK;
}

int kd_set_watchdog(kd_sim* s, double tol) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (!(tol == tol)) return fail(KD_ERR_ARG, "tol is NaN");
    s->watch_tol = tol;
    clear_graphs(s);
    return KD_OK;
}

int kd_init_packet(kd_sim* s, const kd_packet* pk) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (!pk) return fail(KD_ERR_ARG, "null packet");
    if (!(pk->sigma_p > 0) || !isfinite(pk->sigma_p) || !isfinite(pk->p0x) || !isfinite(pk->p0y) ||
        !isfinite(pk->r0x) || !isfinite(pk->r0y))
        return fail(KD_ERR_ARG, "packet parameters must be finite with sigma_p > 0");
    if ((pk->spin != 1 && pk->spin != -1) || (pk->basis != 0 && pk->basis != 1))
        return fail(KD_ERR_ARG, "spin must be +-1 and basis 0 or 1");
    const double dpx = s->u.hbar * 2.0 * kPi / (s->g.x_max - s->g.x_min);
    const double dpy = s->u.hbar * 2.0 * kPi / (s->g.y_max - s->g.y_min);
    const double mc2 = s->u.m * s->u.c * s->u.c;
    const double rx = pk->r0x - s->g.x_min, ry = pk->r0y - s->g.y_min;
    if (s->prec == KD_FP64)
        k_packet<double><<<grid_blocks(s->P, 256), 256, 0, s->stream>>>(
            (double*)s->psi, s->g.nx, s->g.ny, dpx, dpy, s->f.p_shift_x, s->f.p_shift_y, pk->p0x,
            pk->p0y, rx, ry, pk->sigma_p, pk->spin, pk->basis, s->u.c, mc2, s->u.hbar);
    else
        k_packet<float><<<grid_blocks(s->P, 256), 256, 0, s->stream>>>(
            (float*)s->psi, s->g.nx, s->g.ny, dpx, dpy, s->f.p_shift_x, s->f.p_shift_y, pk->p0x,
            pk->p0y, rx, ry, pk->sigma_p, pk->spin, pk->basis, s->u.c, mc2, s->u.hbar);
    KD_CUDA(cudaGetLastError());
    ++s->launches;
    // the packet is built in FP64 in place (also for the double-word form, converted below)
    KD_LAUNCH(sweep(s, AXIS_Y, SHAPE_F2, OP_NONE, s->psi, s->psi, 0, 0.0, true));
    KD_LAUNCH(sweep(s, AXIS_X, SHAPE_F1, OP_NONE, s->psi, s->psi, 0, 0.0, true));
    rc = rowsum_launch(s, s->psi);
    if (rc) return rc;
    k_norm<<<1, 256, 0, s->stream>>>(s->rowsum, s->g.ny, dxdy(s), s->scalar, 0);
    KD_CUDA(cudaGetLastError());
    ++s->launches;
    const size_t nreal = s->P * 8;
    if (s->prec == KD_FP64) k_scale_by_norm<double><<<1024, 256, 0, s->stream>>>((double*)s->psi, nreal, s->scalar);
    else k_scale_by_norm<float><<<1024, 256, 0, s->stream>>>((float*)s->psi, nreal, s->scalar);
    KD_CUDA(cudaGetLastError());
    ++s->launches;
    if (s->dw) {
        rc = dw_from_f64_launch(s, s->psi, nreal);
        if (rc) return rc;
    }
    KD_CUDA(cudaStreamSynchronize(s->stream));
    s->t0 = 0.0;
    s->step = 0;
    const double hk = s->u.hbar * s->f.k_L;
    kd_obs_spec sp{};
    sp.p_in_x = pk->p0x; sp.p_in_y = pk->p0y;
    sp.p_diff_x = pk->p0x + 2.0 * hk; sp.p_diff_y = pk->p0y;
    sp.target_x = sp.p_diff_x; sp.target_y = sp.p_diff_y;
    sp.half_width = 0.5 * hk;
    sp.basis = pk->basis;
    ObsWin w;
    if (make_window(s, &sp, &w) == KD_OK) { s->spec = sp; s->has_spec = true; }
    else { s->has_spec = false; g_err.clear(); }
    clear_graphs(s);
    return KD_OK;
}

}  // extern "C"

namespace {

// One kd_step call's parameters after validation.
struct StepPlan {
    double dt;
    int64_t nsteps, obs_every, nobs, cap;
    ObsWin w;
};

// Validates the arguments, rebases the clock, (re)builds the dt tables and buffers, and
// drops cached graphs whose captured arguments changed.  No device work is enqueued
// except the table build.
int prepare_step(kd_sim* s, double dt, int64_t nsteps, int64_t obs_every, kd_obs* obs_out,
                 int64_t obs_cap, StepPlan* plan) {
    if (!(dt > 0) || !isfinite(dt)) return fail(KD_ERR_ARG, "dt must be positive and finite");
    if (nsteps < 0 || obs_every < 0 || obs_cap < 0) return fail(KD_ERR_ARG, "negative count");
    if (nsteps > (int64_t)1 << 40) return fail(KD_ERR_ARG, "nsteps too large");
    if (obs_every > 0 && obs_cap > 0 && !obs_out) return fail(KD_ERR_ARG, "obs_out is null");
    if (obs_every > 0 && !s->has_spec) return fail(KD_ERR_ARG, "no observation spec: call kd_init_packet or kd_set_obs_spec");
    plan->w = ObsWin{};
    int rc;
    if (obs_every > 0) {
        rc = make_window(s, &s->spec, &plan->w);
        if (rc) return rc;
    }
    // rebase the clock when dt changes: t = t0 + step * dt
    if (dt != s->dt_clock) {
        s->t0 = s->t0 + (double)s->step * s->dt_clock;
        s->step = 0;
        s->dt_clock = dt;
    }
    if (dt != s->ktab_dt) {
        rc = build_dt_tables(s, dt);
        if (rc) return rc;
        clear_graphs(s);
    }
    const int64_t nobs = obs_every > 0 ? nsteps / obs_every : 0;
    const int64_t cap = nobs < obs_cap ? nobs : obs_cap;
    rc = ensure_steps(s, nsteps);
    if (rc) return rc;
    if (nobs > 0) {
        rc = ensure_obs(s, cap > 0 ? cap : 1);
        if (!rc) rc = ensure_md(s);
        if (rc) return rc;
    }
    if (obs_every != s->graph_obs_every || cap != s->graph_obs_cap || dt != s->graph_dt ||
        s->t0 != s->graph_t0 || memcmp(&plan->w, &s->graph_win, sizeof plan->w) != 0) {
        clear_graphs(s);
        s->graph_obs_every = obs_every;
        s->graph_obs_cap = cap;
        s->graph_dt = dt;
        s->graph_t0 = s->t0;
        s->graph_win = plan->w;
    }
    plan->dt = dt;
    plan->nsteps = nsteps;
    plan->obs_every = obs_every;
    plan->nobs = nobs;
    plan->cap = cap;
    return KD_OK;
}

// Per-call device work before the step loop: per-step scalars, clock, watchdog
// reference, and the opening half step of the first step (t_0).
int enqueue_prologue(kd_sim* s, const StepPlan& p) {
    const double omega = s->u.c * s->f.k_L;
    k_step_scalars<<<grid_blocks((size_t)p.nsteps + 1, 256), 256, 0, s->stream>>>(
        s->steps, p.nsteps, s->t0, s->step, p.dt, s->f.a0, omega, s->f.phase0, s->f.env_T,
        s->f.box_vy, s->g.y_min);
    KD_CUDA(cudaGetLastError());
    ++s->launches;
    k_set_clock<<<1, 1, 0, s->stream>>>(s->clock, 0);
    KD_CUDA(cudaGetLastError());
    ++s->launches;
    if (s->tc) {
        int rc = rowsum_launch(s, s->psi);
        if (rc) return rc;
        k_tc_scales<<<1, 256, 0, s->stream>>>(s->rowsum, s->g.nx, s->g.ny, s->tc_scale);
        KD_CUDA(cudaGetLastError());
        ++s->launches;
    }
    if (p.nobs > 0 || s->tc) {
        KD_CUDA(cudaMemsetAsync(s->status, 0, sizeof(int), s->stream));
        if (p.nobs > 0 && s->watch_tol > 0) {
            const void* st = nullptr;
            int rc = state_view(s, &st);
            if (!rc) rc = rowsum_launch(s, st);
            if (rc) return rc;
            k_norm<<<1, 256, 0, s->stream>>>(s->rowsum, s->g.ny, dxdy(s), s->scalar, 1);
            KD_CUDA(cudaGetLastError());
            ++s->launches;
        }
    }
    KD_LAUNCH(sweep(s, AXIS_X, SHAPE_F2, OP_POTENTIAL, s->psi, s->psi, 0, 0.5 * p.dt));
    return KD_OK;
}

// The chunks of a call: chunk i covers steps [i c, (i + 1) c) with c = obs_every (or 64
// without observations); fn(chunk, last, obs) enqueues or launches one chunk.  When
// *cancel is set (kd_cancel) before a chunk is enqueued, that chunk is enqueued as the
// call's last one (it closes the state at its end boundary) and the loop stops; *done
// receives the steps enqueued.
template <typename F> int for_each_chunk(const StepPlan& p, F fn, std::atomic<int>* cancel = nullptr,
                                         int64_t* done_out = nullptr) {
    const int64_t chunk_n = p.obs_every > 0 ? p.obs_every : 64;
    int64_t done = 0;
    if (done_out) *done_out = 0;
    while (done < p.nsteps) {
        const bool stop = cancel && cancel->exchange(0) != 0;
        const int64_t left = p.nsteps - done;
        int64_t chunk = left < chunk_n ? left : chunk_n;
        if (stop && chunk > 64 && p.obs_every == 0) chunk = 64;
        const bool last = stop || done + chunk == p.nsteps;
        const bool obs = p.obs_every > 0 && chunk == p.obs_every;
        int rc = KD_OK;
        if (chunk <= 4096) {
            rc = fn((int)chunk, last, obs);
        } else {  // very long chunks without observations run in pieces of 64
            int64_t rem = chunk;
            while (rem > 0 && rc == KD_OK) {
                const int c2 = (int)(rem < 64 ? rem : 64);
                rc = fn(c2, last && rem == c2, false);
                rem -= c2;
            }
        }
        if (rc) return rc;
        done += chunk;
        if (done_out) *done_out = done;
        if (stop) return KD_ERR_CANCELLED;
    }
    return KD_OK;
}

// After the loop: copy the observation records (synchronises the stream) and turn the
// watchdog status into a return code.
int finish_step(kd_sim* s, const StepPlan& p, kd_obs* obs_out, int64_t* n_obs) {
    s->step += p.nsteps;   // the steps enqueued (fewer than asked after a cancellation)
    if (p.nobs > 0 || s->tc) {
        if (p.nobs > 0 && p.cap > 0)
            KD_CUDA(cudaMemcpyAsync(obs_out, s->obs_dev, p.cap * sizeof(kd_obs), cudaMemcpyDeviceToHost, s->stream));
        int st = 0;
        KD_CUDA(cudaMemcpyAsync(&st, s->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
        KD_CUDA(cudaStreamSynchronize(s->stream));
        if (n_obs) *n_obs = p.nobs;
        if (st & KD_STATUS_TC_TIMEOUT)
            return fail(KD_ERR_TIMEOUT, "tensor-core sweep: a wait for the matrix products gave up");
        if (st & KD_STATUS_NONFINITE) return fail(KD_ERR_NONFINITE, "non-finite norm observed");
        if (st & KD_STATUS_DRIFT) return fail(KD_ERR_NORM_DRIFT, "norm drift beyond %g", s->watch_tol);
    }
    return KD_OK;
}

}  // namespace

extern "C" {

int kd_step(kd_sim* s, double dt, int64_t nsteps, int64_t obs_every, kd_obs* obs_out,
            int64_t obs_cap, int64_t* n_obs) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (n_obs) *n_obs = 0;
    StepPlan p;
    rc = prepare_step(s, dt, nsteps, obs_every, obs_out, obs_cap, &p);
    if (rc || nsteps == 0) return rc;
    rc = enqueue_prologue(s, p);
    if (rc) return rc;
    int64_t done = 0, ci = 0;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool throttle = cudaStreamIsCapturing(s->stream, &cs) == cudaSuccess &&
                          cs == cudaStreamCaptureStatusNone;
    rc = for_each_chunk(p, [&](int chunk, bool last, bool obs) {
        cudaEvent_t& ev = s->ahead[ci % kd_sim::kRunAhead];
        if (throttle && ci >= kd_sim::kRunAhead) KD_CUDA(cudaEventSynchronize(ev));
        int r = run_chunk(s, p.dt, chunk, last, obs, p.w, p.obs_every, p.cap);
        if (r) return r;
        if (throttle) KD_CUDA(cudaEventRecord(ev, s->stream));
        ++ci;
        return KD_OK;
    }, &s->cancel, &done);
    const bool cancelled = rc == KD_ERR_CANCELLED;
    if (rc && !cancelled) return rc;
    if (cancelled) {   // the state is closed at step `done`: account for what ran
        p.nsteps = done;
        p.nobs = p.obs_every > 0 ? done / p.obs_every : 0;
        if (p.cap > p.nobs) p.cap = p.nobs;
    }
    rc = finish_step(s, p, obs_out, n_obs);
    if (cancelled && rc == KD_OK)
        rc = fail(KD_ERR_CANCELLED, "kd_step cancelled after %lld of the requested steps", (long long)done);
    if (s->tc_fault) {   // an injected fault lasts one call (finish_step has synchronised)
        s->tc_fault = 0;
        clear_graphs(s);
    }
    return rc;
}

int kd_inject_fault(kd_sim* s, int32_t kind) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (kind != 0 && kind != KD_FAULT_TC_WAIT && kind != KD_FAULT_PERSIST_HOLD)
        return fail(KD_ERR_ARG, "unknown fault kind %d", kind);
    if (kind == KD_FAULT_TC_WAIT && !s->tc) return fail(KD_ERR_ARG, "not a KD_FP32_TC simulation");
    s->tc_fault = kind == KD_FAULT_TC_WAIT;
    s->persist_hold = kind == KD_FAULT_PERSIST_HOLD;
    clear_graphs(s);
    return KD_OK;
}

int kd_cancel(kd_sim* s) {
    if (!s) return fail(KD_ERR_ARG, "null simulation");
    s->cancel.store(1);
    return KD_OK;
}

int kd_inject_alloc_failure(int32_t after) {
    if (after < -1) return fail(KD_ERR_ARG, "after must be >= -1");
    g_alloc_fail_after.store(after);
    return KD_OK;
}

}  // extern "C"

struct kd_batch {
    std::vector<kd_sim*> sims;
    cudaStream_t stream = nullptr;   // caller's stream
    cudaStream_t cap = nullptr;      // capture origin
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    int device = 0;
    // one graph per chunk shape: all simulations' chunks as concurrent branches
    std::map<GraphKey, std::pair<cudaGraphExec_t, std::vector<int64_t>>> graphs;
    std::vector<uint64_t> gens;      // simulations' graph generations the graphs were built on
    // persistent form (kd_batch_set_mode): member descriptors, prefix sums of the work
    // items, queue head + per-member completion counters, abort flag
    bool persistent = false;
    PersistMember* d_members = nullptr;
    int* d_pre = nullptr;            // [2 (n + 1)]: y items, x items
    unsigned* d_ctr = nullptr;       // [1 + n]: queue head, then completion counters
    int* d_abort = nullptr;
    int y_items = 0, x_items = 0;
    int hold_item = -1;              // withheld completion of the current step call (test hook)
    int persist_group = 1;           // CTA-fulls per work item (kd_batch_autotune)
};

namespace {

// Persistent form: each member's launch variants become the ones the kernel runs for it
// (its own where the kernel holds them, else the axis default), so that the sweep
// arguments (the twiddle tables follow the variant's radix schedule) and the sweeps that
// run outside the kernel (half sweeps at chunk ends, read-outs) use those same variants.
void persist_map_variants(kd_batch* b) {
    for (kd_sim* s : b->sims)
        for (int ax = 0; ax < 2; ++ax) {
            const int logn = ax == AXIS_X ? s->lx : s->ly;
            int v0, v1;
            persist_variants(ax, logn, &v0, &v1);
            const int ran = persist_variant_alt(ax, s->var[ax], logn) ? v1 : v0;
            if (s->var[ax] != ran) {
                s->var[ax] = ran;
                clear_graphs(s);
            }
        }
}

// Persistent form: uploads this call's member descriptors and the work items' prefix
// sums, clears the abort flag, and finds the item whose completion the test hook withholds
// (the first y item of the first held member in the call's first chunk).
int persist_upload(kd_batch* b, const std::vector<StepPlan>& plans, bool* hold) {
    const size_t n = b->sims.size();
    std::vector<PersistMember> hm(n);
    std::vector<int> pre(2 * (n + 1), 0);
    b->hold_item = -1;
    for (size_t i = 0; i < n; ++i) {
        kd_sim* s = b->sims[i];
        PersistMember& m = hm[i];
        m.y = make_args(s, AXIS_Y, OP_KINETIC, s->psi, s->psi, 0, 0.0, false);
        m.x = make_args(s, AXIS_X, OP_POTENTIAL, s->psi, s->psi, 0, plans[i].dt, false);
        m.xc = make_args(s, AXIS_X, OP_POTENTIAL, s->psi, s->psi, 0, 0.5 * plans[i].dt, false);
        m.lx = s->lx;
        m.ly = s->ly;
        // the member's own launch variants where the kernel holds them, else its defaults;
        // the same number of CTA-fulls per work item for every member (uneven groups let
        // the large members' items set the pace of every sweep)
        m.vx_alt = persist_variant_alt(AXIS_X, s->var[AXIS_X], s->lx);
        m.vy_alt = persist_variant_alt(AXIS_Y, s->var[AXIS_Y], s->ly);
        m.cy = persist_ctas(AXIS_Y, m.vy_alt, s->ly, s->g.nx);
        m.cx = persist_ctas(AXIS_X, m.vx_alt, s->lx, s->g.ny);
        m.gy = m.gx = b->persist_group;
        m.iy = (m.cy + m.gy - 1) / m.gy;
        m.ix = (m.cx + m.gx - 1) / m.gx;
        m.status = s->status;
        pre[i + 1] = pre[i] + m.iy;
        pre[n + 1 + i + 1] = pre[n + 1 + i] + m.ix;
        if (s->persist_hold && b->hold_item < 0) b->hold_item = pre[i];
    }
    b->y_items = pre[n];
    b->x_items = pre[2 * n + 1];
    *hold = b->hold_item >= 0;
    KD_CUDA(cudaMemcpyAsync(b->d_members, hm.data(), n * sizeof(PersistMember), cudaMemcpyHostToDevice,
                            b->stream));
    KD_CUDA(cudaMemcpyAsync(b->d_pre, pre.data(), pre.size() * sizeof(int), cudaMemcpyHostToDevice,
                            b->stream));
    KD_CUDA(cudaMemsetAsync(b->d_abort, 0, sizeof(int), b->stream));
    KD_CUDA(cudaStreamSynchronize(b->stream));   // the host vectors go out of scope
    return KD_OK;
}

PersistPlan persist_plan(const kd_batch* b, int chunk, bool closing, int hold_item) {
    const int n = (int)b->sims.size();
    PersistPlan p{};
    p.members = b->d_members;
    p.n = n;
    p.pre_y = b->d_pre;
    p.pre_x = b->d_pre + n + 1;
    p.y_items = b->y_items;
    p.items_per_step = b->y_items + b->x_items;
    p.chunk = chunk;
    p.closing = closing ? 1 : 0;
    p.next = b->d_ctr;
    p.done = b->d_ctr + 1;
    p.abort = b->d_abort;
    p.budget_cycles = 2000000000LL;   // ~1 s at the GB300's clocks
    p.hold_item = hold_item;
    return p;
}

// A member's work after the persistent launch of a chunk (the launch ran its steps and, on
// a closing chunk, the closing half sweep): observation, the next opening half sweep, and
// the device clock, as enqueue_chunk does after its last step.
int persist_tail(kd_sim* s, const StepPlan& p, int chunk, bool last, bool obs) {
    if (last || obs) {
        if (obs) {
            int rc = observe_launch(s, p.w, s->spec.basis, true, chunk, 0.0, p.obs_every, p.cap, s->obs_dev);
            if (rc) return rc;
        }
        if (!last) KD_LAUNCH(sweep(s, AXIS_X, SHAPE_F2, OP_POTENTIAL, s->psi, s->psi, chunk, 0.5 * p.dt));
    }
    k_advance_clock<<<1, 1, 0, s->stream>>>(s->clock, chunk);
    KD_CUDA(cudaGetLastError());
    ++s->launches;
    return KD_OK;
}

void clear_batch_graphs(kd_batch* b) {
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second.first);
    b->graphs.clear();
}

// Runs fn(sim, i) with every simulation's work forked from `origin` onto the
// simulation's own capture stream and joined back, so that the simulations' kernels are
// independent branches (of a capture, or of the stream graph).
template <typename F> int fork_join(kd_batch* b, cudaStream_t origin, F fn) {
    KD_CUDA(cudaEventRecord(b->fork, origin));
    for (size_t i = 0; i < b->sims.size(); ++i) {
        kd_sim* s = b->sims[i];
        KD_CUDA(cudaStreamWaitEvent(s->cap_stream, b->fork, 0));
        cudaStream_t saved = s->stream;
        s->stream = s->cap_stream;
        int rc = fn(s, i);
        s->stream = saved;
        if (rc) return rc;
        KD_CUDA(cudaEventRecord(b->join[i], s->cap_stream));
        KD_CUDA(cudaStreamWaitEvent(origin, b->join[i], 0));
    }
    return KD_OK;
}

}  // namespace

extern "C" {

int kd_batch_create(kd_sim* const* sims, int32_t n, void* cuda_stream, kd_batch** out) {
    g_err.clear();
    if (!sims || !out || n <= 0) return fail(KD_ERR_ARG, "need n > 0 simulations and an output pointer");
    *out = nullptr;
    int dev = -1;
    for (int32_t i = 0; i < n; ++i) {
        if (!sims[i]) return fail(KD_ERR_ARG, "simulation %d is null", i);
        if (dev >= 0 && sims[i]->device != dev) return fail(KD_ERR_ARG, "simulations live on different devices");
        dev = sims[i]->device;
        for (int32_t j = 0; j < i; ++j)
            if (sims[j] == sims[i]) return fail(KD_ERR_ARG, "simulation %d appears twice", i);
    }
    KD_CUDA(cudaSetDevice(dev));
    kd_batch* b = new kd_batch();
    b->sims.assign(sims, sims + n);
    b->stream = (cudaStream_t)cuda_stream;
    b->device = dev;
    b->join.assign(n, nullptr);
    bool ok = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int32_t i = 0; ok && i < n; ++i)
        ok = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        kd_batch_destroy(b);
        return fail(KD_ERR_CUDA, "stream/event creation failed");
    }
    b->gens.assign(n, ~0ull);
    *out = b;
    return KD_OK;
}

void kd_batch_destroy(kd_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    clear_batch_graphs(b);
    void* bufs[] = {b->d_members, b->d_pre, b->d_ctr, b->d_abort};
    for (void* p : bufs)
        if (p) cudaFree(p);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

int kd_batch_step(kd_batch* b, const double* dt, int64_t nsteps, int64_t obs_every,
                  kd_obs* obs_out, int64_t obs_cap, int64_t* n_obs) {
    if (!b || !dt) return fail(KD_ERR_ARG, "null batch or dt");
    KD_CUDA(cudaSetDevice(b->device));
    if (n_obs) *n_obs = 0;
    const size_t n = b->sims.size();
    if (b->persistent) persist_map_variants(b);
    std::vector<StepPlan> plans(n);
    for (size_t i = 0; i < n; ++i) {
        int rc = prepare_step(b->sims[i], dt[i], nsteps, obs_every,
                              obs_out ? obs_out + i * (size_t)obs_cap : nullptr, obs_cap, &plans[i]);
        if (rc) return rc;
    }
    if (nsteps == 0) return KD_OK;
    for (size_t i = 0; i < n; ++i)
        if (b->gens[i] != b->sims[i]->graph_gen) {
            clear_batch_graphs(b);
            for (size_t k = 0; k < n; ++k) b->gens[k] = b->sims[k]->graph_gen;
            break;
        }
    int rc = fork_join(b, b->stream, [&](kd_sim* s, size_t i) { return enqueue_prologue(s, plans[i]); });
    if (rc) return rc;
    // persistent form: this call's member descriptors (dt, tables, per-step scalars), the
    // withheld-completion test hook, a cleared abort flag
    bool hold = false;
    if (b->persistent) {
        rc = persist_upload(b, plans, &hold);
        if (rc) return rc;
    }
    bool first_chunk = true;
    rc = for_each_chunk(plans[0], [&](int chunk, bool last, bool obs) -> int {
        GraphKey key{chunk, last ? 1 : 0, obs ? 1 : 0};
        const bool held = hold && first_chunk;   // this chunk's graph carries the hook
        first_chunk = false;
        if (held) clear_batch_graphs(b);
        auto it = b->graphs.find(key);
        if (it == b->graphs.end()) {
            std::vector<int64_t> nodes(n, 0);
            cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return fail(KD_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
            int crc = KD_OK;
            if (b->persistent) {
                // one launch for every member's steps of the chunk, then the members'
                // observation / opening tails and clocks as branches
                PersistPlan pl = persist_plan(b, chunk, last || obs, held ? b->hold_item : -1);
                if (cudaMemsetAsync(b->d_ctr, 0, (1 + n) * sizeof(unsigned), b->cap) != cudaSuccess ||
                    launch_persist(pl, b->cap) != cudaSuccess)
                    crc = fail(KD_ERR_CUDA, "persistent batch launch failed");
                b->sims[0]->launches += 1;
                nodes[0] += 1;
            }
            if (crc == KD_OK) crc = fork_join(b, b->cap, [&](kd_sim* s, size_t i) {
                const int64_t before = s->launches;
                int r = b->persistent ? persist_tail(s, plans[i], chunk, last, obs)
                                      : enqueue_chunk(s, plans[i].dt, chunk, last, obs, plans[i].w,
                                                      plans[i].obs_every, plans[i].cap);
                nodes[i] += s->launches - before;
                s->launches = before;
                return r;
            });
            cudaGraph_t graph = nullptr;
            e = cudaStreamEndCapture(b->cap, &graph);
            if (crc) { if (graph) cudaGraphDestroy(graph); return crc; }
            if (e != cudaSuccess) return fail(KD_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
            cudaGraphExec_t exec = nullptr;
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return fail(KD_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
            it = b->graphs.emplace(key, std::make_pair(exec, nodes)).first;
        }
        KD_CUDA(cudaGraphLaunch(it->second.first, b->stream));
        for (size_t i = 0; i < n; ++i) b->sims[i]->launches += it->second.second[i];
        if (held) clear_batch_graphs(b);   // the hook lasts one chunk of one call
        return KD_OK;
    });
    if (rc) return rc;
    int first_err = KD_OK;
    if (b->persistent) {
        int ab = 0;
        KD_CUDA(cudaMemcpyAsync(&ab, b->d_abort, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
        KD_CUDA(cudaStreamSynchronize(b->stream));
        for (kd_sim* s : b->sims) s->persist_hold = 0;
        if (ab) first_err = fail(KD_ERR_TIMEOUT, "persistent batch: a bounded wait for a member's "
                                                 "previous sweep gave up (states are not valid)");
    }
    for (size_t i = 0; i < n; ++i) {
        kd_sim* s = b->sims[i];
        cudaStream_t saved = s->stream;
        s->stream = b->stream;   // all branches are joined on the batch stream
        int r = finish_step(s, plans[i], obs_out ? obs_out + i * (size_t)obs_cap : nullptr, n_obs);
        if (r && first_err == KD_ERR_TIMEOUT) r = KD_OK;   // already reported
        s->stream = saved;
        if (r && !first_err) first_err = r;
        if (s->tc_fault) {   // an injected fault lasts one step call, batched or not
            s->tc_fault = 0;
            clear_graphs(s);
        }
    }
    return first_err;
}

int kd_batch_set_mode(kd_batch* b, int32_t mode) {
    if (!b) return fail(KD_ERR_ARG, "null batch");
    if (mode != KD_BATCH_GRAPH && mode != KD_BATCH_PERSISTENT) return fail(KD_ERR_ARG, "unknown batch mode %d", mode);
    KD_CUDA(cudaSetDevice(b->device));
    if (mode == KD_BATCH_PERSISTENT) {
        for (size_t i = 0; i < b->sims.size(); ++i) {
            const kd_sim* s = b->sims[i];
            if (s->prec != KD_FP32 || s->tc || s->dw)
                return fail(KD_ERR_UNSUPPORTED_SIZE, "persistent batch: member %zu is not a KD_FP32 simulation", i);
            if (!persist_supported(s->lx) || !persist_supported(s->ly))
                return fail(KD_ERR_UNSUPPORTED_SIZE, "persistent batch: member %zu grid %dx%d outside 16..512 per axis",
                            i, s->g.nx, s->g.ny);
        }
        const size_t n = b->sims.size();
        if (!b->d_members) {
            KD_CUDA(dev_alloc((void**)&b->d_members, n * sizeof(PersistMember)));
            KD_CUDA(dev_alloc((void**)&b->d_pre, 2 * (n + 1) * sizeof(int)));
            KD_CUDA(dev_alloc((void**)&b->d_ctr, (1 + n) * sizeof(unsigned)));
            KD_CUDA(dev_alloc((void**)&b->d_abort, sizeof(int)));
        }
    }
    KD_CUDA(cudaStreamSynchronize(b->stream));
    b->persistent = mode == KD_BATCH_PERSISTENT;
    if (b->persistent) persist_map_variants(b);
    clear_batch_graphs(b);
    return KD_OK;
}

int kd_batch_autotune(kd_batch* b, const double* dt, int32_t steps, int32_t* variants) {
    if (!b || !dt) return fail(KD_ERR_ARG, "null batch or dt");
    if (steps < 1 || steps > 4096) return fail(KD_ERR_ARG, "steps must be in [1, 4096]");
    KD_CUDA(cudaSetDevice(b->device));
    const size_t n = b->sims.size();
    for (size_t i = 0; i < n; ++i) {
        if (!(dt[i] > 0) || !isfinite(dt[i])) return fail(KD_ERR_ARG, "dt[%zu] must be positive and finite", i);
        int rc = reject_capture(b->sims[i], "kd_batch_autotune");
        if (rc) return rc;
    }
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(b->stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
            return fail(KD_ERR_ARG, "kd_batch_autotune: the batch stream is being captured");
        cudaGetLastError();
    }
    // every compiled variant launched once outside any capture (kernel attributes), then
    // the current variants back; warm_variants writes only the work buffers
    std::vector<std::pair<int, int>> keep(n);
    for (size_t i = 0; i < n; ++i) {
        kd_sim* s = b->sims[i];
        keep[i] = {s->var[0], s->var[1]};
        if (s->prec == KD_FP64) continue;
        for (int v = 0; v < KD_SWEEP_VARIANTS; ++v) {
            s->var[0] = s->var[1] = v;
            int rc = warm_variants(s);
            if (rc) return rc;
        }
        s->var[0] = keep[i].first;
        s->var[1] = keep[i].second;
    }
    // the states and clocks are restored afterwards: states parked in the work buffers
    struct Clk { double t0, dt_clock; int64_t step; };
    std::vector<Clk> clk(n);
    for (size_t i = 0; i < n; ++i) {
        kd_sim* s = b->sims[i];
        KD_CUDA(cudaStreamSynchronize(s->stream));
        KD_CUDA(cudaMemcpyAsync(s->work, s->psi, spinor_bytes(s), cudaMemcpyDeviceToDevice, b->stream));
        clk[i] = {s->t0, s->dt_clock, s->step};
    }
    cudaEvent_t ev[2] = {nullptr, nullptr};
    KD_CUDA(cudaEventCreate(&ev[0]));
    KD_CUDA(cudaEventCreate(&ev[1]));
    auto timed = [&](float* ms) -> int {
        int rc = kd_batch_step(b, dt, steps, 0, nullptr, 0, nullptr);   // captures the graphs
        if (rc) return rc;
        KD_CUDA(cudaEventRecord(ev[0], b->stream));
        rc = kd_batch_step(b, dt, steps, 0, nullptr, 0, nullptr);
        if (rc) return rc;
        KD_CUDA(cudaEventRecord(ev[1], b->stream));
        KD_CUDA(cudaEventSynchronize(ev[1]));
        KD_CUDA(cudaEventElapsedTime(ms, ev[0], ev[1]));
        return KD_OK;
    };
    auto set_var = [&](size_t i, int ax, int v) {
        kd_sim* s = b->sims[i];
        if (s->var[ax] != v) {
            s->var[ax] = v;
            clear_graphs(s);
        }
    };
    // greedy: per axis, per group of members with the same grid and form, the variant
    // with the shortest batch time (kept only when > 2 % faster than the group's current)
    std::map<std::tuple<int, int, int>, std::vector<size_t>> groups;
    for (size_t i = 0; i < n; ++i) {
        kd_sim* s = b->sims[i];
        if (s->prec != KD_FP64) groups[std::make_tuple(s->g.nx, s->g.ny, (int)s->tc)].push_back(i);
    }
    int rc = KD_OK;
    float base = 0.0f;
    if (!groups.empty()) rc = timed(&base);
    for (int ax = 0; ax < 2 && !rc; ++ax)
        for (auto& kv : groups) {
            if (rc) break;
            const int cur = b->sims[kv.second[0]]->var[ax];
            int best = cur;
            float best_ms = base;
            for (int v = 0; v < KD_SWEEP_VARIANTS && !rc; ++v) {
                if (v == cur) continue;
                if (b->persistent) {   // the variants the persistent kernel holds
                    int v0, v1;
                    const kd_sim* s0 = b->sims[kv.second[0]];
                    persist_variants(ax, ax == AXIS_X ? s0->lx : s0->ly, &v0, &v1);
                    if (v != v0 && v != v1) continue;
                }
                for (size_t i : kv.second) set_var(i, ax, v);
                float ms = 0.0f;
                rc = timed(&ms);
                if (!rc && ms < 0.98f * best_ms) { best = v; best_ms = ms; }
            }
            for (size_t i : kv.second) set_var(i, ax, best);
            base = best_ms;
        }
    // persistent form: the work item size (CTA-fulls per item), same rule
    if (b->persistent && !rc) {
        int best = b->persist_group;
        float best_ms = base;
        for (int g : {1, 2, 4}) {
            if (g == b->persist_group || rc) continue;
            const int cur = b->persist_group;
            b->persist_group = g;
            clear_batch_graphs(b);
            float ms = 0.0f;
            rc = timed(&ms);
            b->persist_group = cur;
            if (!rc && ms < 0.98f * best_ms) { best = g; best_ms = ms; }
        }
        b->persist_group = best;
        clear_batch_graphs(b);
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    // states and clocks back (whatever happened above)
    for (size_t i = 0; i < n; ++i) {
        kd_sim* s = b->sims[i];
        cudaMemcpyAsync(s->psi, s->work, spinor_bytes(s), cudaMemcpyDeviceToDevice, b->stream);
        s->t0 = clk[i].t0;
        s->dt_clock = clk[i].dt_clock;
        s->step = clk[i].step;
        clear_graphs(s);
    }
    KD_CUDA(cudaStreamSynchronize(b->stream));
    if (rc) {
        for (size_t i = 0; i < n; ++i) {
            b->sims[i]->var[0] = keep[i].first;
            b->sims[i]->var[1] = keep[i].second;
        }
        return rc;
    }
    if (variants)
        for (size_t i = 0; i < n; ++i) {
            variants[2 * i] = b->sims[i]->var[0];
            variants[2 * i + 1] = b->sims[i]->var[1];
        }
    return KD_OK;
}

int kd_observe(kd_sim* s, const kd_obs_spec* spec, kd_obs* out) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (!out) return fail(KD_ERR_ARG, "null output");
    if (!spec && !s->has_spec) return fail(KD_ERR_ARG, "no observation spec");
    const kd_obs_spec* sp = spec ? spec : &s->spec;
    ObsWin w;
    rc = make_window(s, sp, &w);
    if (rc) return rc;
    rc = ensure_obs(s, 1);
    if (rc) return rc;
    const double t = s->t0 + (double)s->step * s->dt_clock;
    rc = observe_launch(s, w, sp->basis, false, 0, t, 1, 1, s->obs_dev);
    if (rc) return rc;
    KD_CUDA(cudaMemcpyAsync(out, s->obs_dev, sizeof(kd_obs), cudaMemcpyDeviceToHost, s->stream));
    KD_CUDA(cudaStreamSynchronize(s->stream));
    return KD_OK;
}

int kd_get_momentum_density(kd_sim* s, int32_t basis, double* out, int32_t where) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (!out || (where != KD_HOST && where != KD_DEVICE) || (basis != 0 && basis != 1))
        return fail(KD_ERR_ARG, "bad output pointer, where or basis");
    double* dst = out;
    if (where == KD_HOST) {
        rc = ensure_md(s);
        if (rc) return rc;
        dst = s->md;
    }
    rc = momentum_density_launch(s, basis, dst);
    if (rc) return rc;
    if (where == KD_HOST) {
        KD_CUDA(cudaMemcpyAsync(out, s->md, s->P * 3 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        KD_CUDA(cudaStreamSynchronize(s->stream));
    }
    return KD_OK;
}

int kd_get_density_x(kd_sim* s, double* out, int32_t where) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (!out || (where != KD_HOST && where != KD_DEVICE)) return fail(KD_ERR_ARG, "bad output pointer or where");
    double* dst = out;
    if (where == KD_HOST) {
        rc = ensure_md(s);
        if (rc) return rc;
        dst = s->md;
    }
    const double dy = (s->g.y_max - s->g.y_min) / s->g.ny;
    const void* st = nullptr;
    rc = state_view(s, &st);
    if (rc) return rc;
    if (s->prec == KD_FP64) k_density_x<double><<<grid_blocks(s->g.nx, 128), 128, 0, s->stream>>>((const double*)st, s->g.nx, s->g.ny, dy, dst);
    else k_density_x<float><<<grid_blocks(s->g.nx, 128), 128, 0, s->stream>>>((const float*)s->psi, s->g.nx, s->g.ny, dy, dst);
    KD_CUDA(cudaGetLastError());
    ++s->launches;
    if (where == KD_HOST) {
        KD_CUDA(cudaMemcpyAsync(out, dst, s->g.nx * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        KD_CUDA(cudaStreamSynchronize(s->stream));
    }
    return KD_OK;
}

int kd_bench_sweep(kd_sim* s, int32_t kind, int32_t reps) {
    int rc = check_sim(s);
    if (rc) return rc;
    if ((kind != 0 && kind != 1) || reps < 0) return fail(KD_ERR_ARG, "kind must be 0 or 1, reps >= 0");
    if (s->ktab_dt == 0.0 || !s->steps) return fail(KD_ERR_ARG, "call kd_step once before kd_bench_sweep");
    // the launches are captured once into a graph (per kind and count) and replayed, so
    // that the GPU runs them back to back without host launch overhead
    GraphKey key{-1 - kind, reps, 0};
    auto it = s->graphs.find(key);
    if (it == s->graphs.end()) {
        cudaStream_t user = s->stream;
        s->stream = s->cap_stream;
        cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            s->stream = user;
            return fail(KD_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
        }
        const int64_t before = s->launches;
        cudaError_t el = cudaSuccess;
        k_set_clock<<<1, 1, 0, s->stream>>>(s->clock, 0);
        ++s->launches;
        for (int32_t i = 0; i < reps && el == cudaSuccess; ++i)
            el = kind == 0 ? sweep(s, AXIS_X, SHAPE_F1F2, OP_POTENTIAL, s->psi, s->psi, 0, s->ktab_dt)
                           : sweep(s, AXIS_Y, SHAPE_F1F2, OP_KINETIC, s->psi, s->psi, 0, 0.0);
        const int64_t nodes = s->launches - before;
        s->launches = before;
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(s->stream, &graph);
        s->stream = user;
        if (el != cudaSuccess || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(KD_ERR_CUDA, "bench capture: %s", cudaGetErrorString(el != cudaSuccess ? el : e));
        }
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(KD_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        it = s->graphs.emplace(key, std::make_pair(exec, nodes)).first;
    }
    KD_CUDA(cudaGraphLaunch(it->second.first, s->stream));
    s->launches += it->second.second;
    return KD_OK;
}

int kd_set_sweep_variants(kd_sim* s, int32_t variant_x, int32_t variant_y) {
    int rc = check_sim(s);
    if (rc) return rc;
    const int nv = s->prec == KD_FP64 ? 1 : KD_SWEEP_VARIANTS;
    if (variant_x < 0 || variant_x >= nv || variant_y < 0 || variant_y >= nv)
        return fail(KD_ERR_ARG, "sweep variant out of range [0, %d)", nv);
    if (s->var[0] == variant_x && s->var[1] == variant_y) return KD_OK;
    rc = reject_capture(s, "kd_set_sweep_variants");
    if (rc) return rc;
    s->var[0] = variant_x;
    s->var[1] = variant_y;
    clear_graphs(s);
    return warm_variants(s);
}

int kd_get_sweep_variants(kd_sim* s, int32_t* variant_x, int32_t* variant_y) {
    if (!s || !variant_x || !variant_y) return fail(KD_ERR_ARG, "null argument");
    *variant_x = s->var[0];
    *variant_y = s->var[1];
    return KD_OK;
}

int kd_autotune(kd_sim* s, double dt, int32_t reps, int32_t flags, int32_t* variant_x,
                int32_t* variant_y, float* times_ms) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (!(dt > 0) || !isfinite(dt)) return fail(KD_ERR_ARG, "dt must be positive and finite");
    if (reps < 1 || reps > 4096) return fail(KD_ERR_ARG, "reps must be in [1, 4096]");
    if (flags & ~KD_TUNE_FORCE) return fail(KD_ERR_ARG, "unknown flags");
    rc = reject_capture(s, "kd_autotune");
    if (rc) return rc;
    TuneResult res{};
    for (auto& a : res.ms)
        for (float& m : a) m = -1.0f;
    if (s->prec == KD_FP64) {   // one compiled variant: nothing to choose
        rc = kd_set_sweep_variants(s, 0, 0);
        if (rc) return rc;
    } else {
        const TuneKey key{s->device, s->g.nx, s->g.ny, s->f.kind, s->f.longitudinal, (int)s->tc};
        bool cached = false;
        if (!(flags & KD_TUNE_FORCE)) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune.find(key);
            if (it != g_tune.end()) { res = it->second; cached = true; }
        }
        if (!cached) {
            // the step's tables and one step's scalars for dt at the current time
            if (dt != s->ktab_dt) {
                rc = build_dt_tables(s, dt);
                if (rc) return rc;
                clear_graphs(s);
            }
            rc = ensure_steps(s, 1);
            if (rc) return rc;
            const double omega = s->u.c * s->f.k_L;
            k_step_scalars<<<1, 256, 0, s->stream>>>(s->steps, 1, s->t0 + (double)s->step * s->dt_clock, 0,
                                                     dt, s->f.a0, omega, s->f.phase0, s->f.env_T,
                                                     s->f.box_vy, s->g.y_min);
            KD_CUDA(cudaGetLastError());
            k_set_clock<<<1, 1, 0, s->stream>>>(s->clock, 0);
            KD_CUDA(cudaGetLastError());
            s->launches += 2;
            const int keep[2] = {s->var[0], s->var[1]};
            for (int ax = 0; ax < 2 && !rc; ++ax) {
                for (int v = 0; v < KD_SWEEP_VARIANTS && !rc; ++v) {
                    s->var[ax] = v;
                    rc = warm_variants(s);
                    if (!rc) rc = time_sweep(s, ax, reps, dt, &res.ms[ax][v]);
                }
                // the default stays unless another variant is faster by more than 2 %
                int best = 0;
                for (int v = 1; v < KD_SWEEP_VARIANTS; ++v)
                    if (res.ms[ax][v] < 0.98f * res.ms[ax][best]) best = v;
                res.var[ax] = best;
                s->var[ax] = keep[ax];
            }
            if (rc) {
                s->var[0] = keep[0];
                s->var[1] = keep[1];
                return rc;
            }
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune[key] = res;
        }
        rc = kd_set_sweep_variants(s, res.var[0], res.var[1]);
        if (rc) return rc;
    }
    if (variant_x) *variant_x = s->var[0];
    if (variant_y) *variant_y = s->var[1];
    if (times_ms)
        for (int ax = 0; ax < 2; ++ax)
            for (int v = 0; v < KD_SWEEP_VARIANTS; ++v) times_ms[ax * KD_SWEEP_VARIANTS + v] = res.ms[ax][v];
    return KD_OK;
}

int kd_get_launch_count(kd_sim* s, int64_t* n) {
    if (!s || !n) return fail(KD_ERR_ARG, "null argument");
    *n = s->launches;
    return KD_OK;
}

int kd_get_state(kd_sim* s, void* buf, size_t* size) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (!size) return fail(KD_ERR_ARG, "null size");
    const size_t need = sizeof(StateHeader) + spinor_bytes(s);
    if (!buf || *size < need) {
        *size = need;
        return buf ? fail(KD_ERR_ARG, "buffer too small (%zu < %zu)", *size, need) : KD_OK;
    }
    StateHeader h{};
    h.magic = 0x3153444bu;  // "KDS1"
    h.version = 1;
    h.nx = s->g.nx;
    h.ny = s->g.ny;
    h.prec = s->prec;
    h.hash = param_hash(s);
    h.t0 = s->t0;
    h.dt_clock = s->dt_clock;
    h.step = s->step;
    h.payload = spinor_bytes(s);
    memcpy(buf, &h, sizeof h);
    rc = copy_out(s, (char*)buf + sizeof h, KD_HOST);
    if (rc) return rc;
    *size = need;
    return KD_OK;
}

int kd_set_state(kd_sim* s, const void* buf, size_t size) {
    int rc = check_sim(s);
    if (rc) return rc;
    if (!buf || size < sizeof(StateHeader)) return fail(KD_ERR_ARG, "state buffer too small");
    StateHeader h;
    memcpy(&h, buf, sizeof h);
    if (h.magic != 0x3153444bu || h.version != 1) return fail(KD_ERR_STATE_MISMATCH, "not a kd state");
    if (h.nx != s->g.nx || h.ny != s->g.ny || h.prec != s->prec || h.hash != param_hash(s) ||
        h.payload != spinor_bytes(s) || size < sizeof h + h.payload)
        return fail(KD_ERR_STATE_MISMATCH, "state was taken from a different simulation");
    rc = copy_in(s, (const char*)buf + sizeof h, KD_HOST);
    if (rc) return rc;
    s->t0 = h.t0;
    s->dt_clock = h.dt_clock;
    s->step = h.step;
    clear_graphs(s);
    return KD_OK;
}

}  // extern "C"
