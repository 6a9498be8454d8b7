// kd_noalloc.cu -- kd_density_noalloc: position-space norm and y-integrated density of a
// caller's spinor, for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: hosts that hand the library a fixed memory budget
// (another framework's pool already owns the device memory), real-time loops that must
// never wait on the allocator (cudaMalloc and cudaFree can synchronise the device), and
// plug-ins that run inside a runtime which forbids them to allocate.  This entry point
// needs no kd_sim (which owns allocated buffers): its only scratch, the per-row partial
// sums of the norm, lives in the file-scope device array below, which every GPU that
// loads the library holds until the process exits.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "../../include/kd.h"

namespace kd {
int set_error(int code, const char* msg);  // kd_api.cu: message for kd_last_error()
void clear_error();                         // kd_api.cu: kd_last_error() becomes ""
}

namespace {

// One double per grid row; 4096 rows = 32 KiB per device.
constexpr int kMaxRows = KD_NOALLOC_MAX_ROWS;
static __device__ __align__(256) double g_row_scratch[kMaxRows];

// Device address of g_row_scratch per device ordinal, looked up once per device and
// context: the unique id of the context the address was taken in is kept beside it, so
// that a new primary context on that device (after cudaDeviceReset) is noticed and the
// address looked up again instead of being used stale.
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};
std::mutex g_setup_mu;

// The two driver calls that identify the current context, found through the runtime
// (the library links no driver library of its own, so it also loads where none exists).
PFN_cuCtxGetCurrent_v4000 p_ctx_get_current = nullptr;
PFN_cuCtxGetId_v12000 p_ctx_get_id = nullptr;

bool driver_calls() {
    if (p_ctx_get_current && p_ctx_get_id) return true;
    void* a = nullptr;
    void* b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 4000, cudaEnableDefault, &qa) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) != cudaSuccess ||
        qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
        return false;
    p_ctx_get_current = (PFN_cuCtxGetCurrent_v4000)a;
    p_ctx_get_id = (PFN_cuCtxGetId_v12000)b;
    return true;
}

// Sum of |psi|^2 over one row of a [ny][nx][4] complex spinor, fixed-order tree.
template <typename T>
__global__ void k_row_norm(const T* psi, int nx, double* rows) {
    __shared__ double red[256];
    const T* p = psi + (size_t)blockIdx.x * nx * 8;
    double acc = 0.0;
    for (int i = threadIdx.x; i < nx * 8; i += blockDim.x) acc += (double)p[i] * (double)p[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) rows[blockIdx.x] = red[0];
}

__global__ void k_sum_rows(const double* rows, int ny, double cell, double* out) {
    __shared__ double red[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < ny; i += blockDim.x) acc += rows[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] * cell;
}

// Phi(x) = sum_y |psi|^2 dy, one thread per column, rows in order.
template <typename T>
__global__ void k_col_density(const T* psi, int nx, int ny, double dy, double* out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    double acc = 0.0;
    for (int y = 0; y < ny; ++y) {
        const T* p = psi + ((size_t)y * nx + x) * 8;
        double s = 0.0;
        for (int i = 0; i < 8; ++i) s += (double)p[i] * (double)p[i];
        acc += s;
    }
    out[x] = acc * dy;
}

int noalloc_fail(int code, const char* msg) { return kd::set_error(code, msg); }

}  // namespace

extern "C" int kd_density_noalloc(const void* psi, int32_t nx, int32_t ny, int32_t precision,
                                  double dx, double dy, double* norm_out, double* density_x_out,
                                  void* cuda_stream) {
    if (!psi || (!norm_out && !density_x_out))
        return noalloc_fail(KD_ERR_ARG, "kd_density_noalloc: null spinor or no output requested");
    if (precision != KD_FP64 && precision != KD_FP32)
        return noalloc_fail(KD_ERR_ARG, "kd_density_noalloc: precision must be KD_FP64 or KD_FP32");
    if (nx <= 0 || ny <= 0 || nx > 4096)
        return noalloc_fail(KD_ERR_UNSUPPORTED_SIZE, "kd_density_noalloc: nx must be in [1, 4096] and ny > 0");
    if (ny > kMaxRows)
        return noalloc_fail(KD_ERR_UNSUPPORTED_SIZE,
                            "kd_density_noalloc: ny exceeds the static scratch of KD_NOALLOC_MAX_ROWS (4096) rows");
    if (!isfinite(dx) || !isfinite(dy)) return noalloc_fail(KD_ERR_ARG, "kd_density_noalloc: dx, dy must be finite");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return noalloc_fail(KD_ERR_CUDA, "kd_density_noalloc: no usable current CUDA device");
    CUcontext ctx = nullptr;
    unsigned long long ctx_id = 0;
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!driver_calls())
            return noalloc_fail(KD_ERR_CUDA, "kd_density_noalloc: the CUDA driver's context calls are unavailable");
    }
    if (p_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) {
        // this thread has not used the runtime yet: setting the current device again
        // initialises the driver and the device's primary context (allocating nothing)
        if (cudaSetDevice(dev) != cudaSuccess || p_ctx_get_current(&ctx) != CUDA_SUCCESS)
            return noalloc_fail(KD_ERR_CUDA, "kd_density_noalloc: the device's context is not usable");
    }
    if (!ctx || p_ctx_get_id(ctx, &ctx_id) != CUDA_SUCCESS)
        return noalloc_fail(KD_ERR_CUDA, "kd_density_noalloc: no current CUDA context");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double* rows = nullptr;
    {
        // once per device (and again after the device's context was replaced), with that
        // device current: the host-side name g_row_scratch is only a stand-in, the
        // kernels need the device address
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx_id) {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
                return noalloc_fail(KD_ERR_CUDA,
                                    "kd_density_noalloc: the first call on a device (or after its "
                                    "context was reset) must not be made on a capturing stream");
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_row_scratch);
            if (e != cudaSuccess || !p)
                return noalloc_fail(KD_ERR_CUDA, "kd_density_noalloc: cudaGetSymbolAddress failed");
            g_scratch_addr[dev] = (double*)p;
            g_scratch_ctx[dev] = ctx_id;
        }
        rows = g_scratch_addr[dev];
    }
    // drop an earlier launch error of unrelated work on this thread, so that the check
    // after our launches reports only our own
    (void)cudaGetLastError();
    if (norm_out) {
        // every row of the scratch that k_sum_rows reads is written first, so nothing
        // needs clearing between calls
        if (precision == KD_FP64) k_row_norm<double><<<ny, 256, 0, s>>>((const double*)psi, nx, rows);
        else k_row_norm<float><<<ny, 256, 0, s>>>((const float*)psi, nx, rows);
        k_sum_rows<<<1, 256, 0, s>>>(rows, ny, dx * dy, norm_out);
    }
    if (density_x_out) {
        const int blocks = (nx + 127) / 128;
        if (precision == KD_FP64) k_col_density<double><<<blocks, 128, 0, s>>>((const double*)psi, nx, ny, dy, density_x_out);
        else k_col_density<float><<<blocks, 128, 0, s>>>((const float*)psi, nx, ny, dy, density_x_out);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(KD_ERR_CUDA, cudaGetErrorString(e));
    kd::clear_error();
    return KD_OK;
}
