// sgl_noalloc.cu -- sgl_trig_coeffs_noalloc: the trigonometric coefficients eta without any
// device allocation, for callers that cannot call cudaMalloc.
//
// Who needs it: applications whose device memory is owned by their own pool allocator
// (a framework's caching allocator that has reserved most of the GPU, an embedded or
// real-time runtime with a fixed memory budget) cannot let a library call cudaMalloc or
// cudaFree: those calls may fail once the pool holds the memory, and they can synchronize
// the device in the middle of the caller's work.  A plan (sgl_plan_create) allocates its
// workspace, so such callers use this entry point instead.
//
// All scratch -- the polar matrices and cosine tables of every B <= SGL_NOALLOC_MAX_B, the
// radial values and matrices, beta, zeta and the reduction cell for rho -- lives in one
// file-scope __device__ array (about 6.9 MB).  Every GPU that loads libsgl.so holds that array
// until the process exits.  The caller passes inputs and outputs only.  The tables are built on
// the host once per process (in static storage) and copied into the array once per device, by
// the first call on that device; later calls issue only kernels and one memset.
#include "sgl_internal.cuh"

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

namespace sgl {
namespace {

constexpr int kMaxB = SGL_NOALLOC_MAX_B;
constexpr size_t round32(size_t n) { return (n + 31) / 32 * 32; }     // regions start on 256-byte boundaries
// the tables of bandwidth B start at table_offset(B): sum over b < B of (b^3 + 8b), rounded up
constexpr size_t table_offset(int B) {
    size_t o = 0;
    for (int b = 1; b < B; ++b) o += round32((size_t)b * b * b + (size_t)8 * b);
    return o;
}
constexpr size_t kRegTables = table_offset(kMaxB + 1);
constexpr size_t kRegRadv = round32((size_t)kMaxB * kMaxB * (kMaxB + 1));
constexpr size_t kRegKmat = round32((size_t)(2 * kMaxB - 1) * kMaxB * (kMaxB + 1) / 2);
constexpr size_t kRegBeta = round32((size_t)2 * (2 * kMaxB - 1) * (2 * kMaxB - 1) * kMaxB);   // double2 as 2 doubles
constexpr size_t kRegZeta = round32((size_t)2 * (2 * kMaxB - 1) * kMaxB * (2 * kMaxB - 1));
constexpr size_t kRegCell = 32;                                                                // r2max bits + flags
constexpr size_t kScratchDoubles = kRegTables + kRegRadv + kRegKmat + kRegBeta + kRegZeta + kRegCell;

}  // namespace
}  // namespace sgl

// The shared scratch.  Host code must not use this name as a pointer: it only stands
// for the symbol; the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_scratch[sgl::kScratchDoubles];

namespace sgl {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_on_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

// The conversion tables of every B <= kMaxB in host static storage (no heap use), built once per
// process by the plan's own builder (conversion_tables); the Legendre scratch is static too.
std::mutex g_host_mu;
bool g_host_built = false;
double g_host_tables[kRegTables];
double g_leg[2 * kMaxB * kMaxB * kMaxB];
bool g_dev_tables[kMaxDevices] = {};

void build_host_tables() {
    for (int B = 1; B <= kMaxB; ++B) {
        double *P = g_host_tables + table_offset(B);
        conversion_tables(B, P, P + (size_t)B * B * B, g_leg);
    }
    g_host_built = true;
}

// Set-up of the current device (once): the scratch address and one copy of the tables into it
// on stream s, which is then synchronized (so that calls on any stream find the tables in
// place).  Refused while s is being captured (the copy and the wait cannot be captured).
cudaError_t setup_current_device(cudaStream_t s, double **out, bool *capture_refused) {
    *capture_refused = false;
    cudaError_t e = scratch_on_current_device(out);
    if (e != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_host_mu);
    if (g_dev_tables[dev]) return cudaSuccess;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(s, &cs)) != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusNone) {
        *capture_refused = true;
        return cudaErrorStreamCaptureUnsupported;
    }
    if (!g_host_built) build_host_tables();
    if ((e = cudaMemcpyAsync(*out, g_host_tables, sizeof(g_host_tables), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    g_dev_tables[dev] = true;
    return cudaSuccess;
}

}  // namespace
}  // namespace sgl

extern "C" int sgl_noalloc_max_b(void) { return sgl::kMaxB; }

extern "C" sgl_status sgl_trig_coeffs_noalloc(int B, const double *xyz_dev, int64_t M, const double *coef_dev,
                                              double *eta_dev, void *cuda_stream) {
    using namespace sgl;
    if (B < 1 || B > kMaxB)
        return set_error(SGL_ERR_ARG, "sgl_trig_coeffs_noalloc: B must be in [1, " + std::to_string(kMaxB) +
                                          "] (its static scratch is sized for B <= " + std::to_string(kMaxB) + ")");
    if (M < 0) return set_error(SGL_ERR_ARG, "sgl_trig_coeffs_noalloc: M must be >= 0");
    if ((M > 0 && (!xyz_dev || ((uintptr_t)xyz_dev & 7u))) || !coef_dev || !eta_dev || ((uintptr_t)coef_dev & 7u) ||
        ((uintptr_t)eta_dev & 7u))
        return set_error(SGL_ERR_ARG, "sgl_trig_coeffs_noalloc: buffers must be non-NULL, 8-byte aligned device pointers");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double *base = nullptr;
    bool refused = false;
    cudaError_t e = setup_current_device(s, &base, &refused);
    if (refused)
        return set_error(SGL_ERR_STATE, "sgl_trig_coeffs_noalloc: the first call on a device copies its tables and "
                                        "cannot run inside a stream capture; call it once before capturing");
    if (e != cudaSuccess) return set_error(SGL_ERR_CUDA, std::string("set-up of the static scratch: ") + cudaGetErrorString(e));
    double *P = base + table_offset(B);
    double *costab = P + (size_t)B * B * B;
    double *radv = base + kRegTables;
    double *Kmat = radv + kRegRadv;
    double2 *beta = reinterpret_cast<double2 *>(Kmat + kRegKmat);
    double2 *zeta = reinterpret_cast<double2 *>(Kmat + kRegKmat + kRegBeta);
    unsigned long long *r2max = reinterpret_cast<unsigned long long *>(Kmat + kRegKmat + kRegBeta + kRegZeta);
    int *flags = reinterpret_cast<int *>(r2max + 1);
    // the reduction cell starts at zero for every call
    if ((e = cudaMemsetAsync(r2max, 0, 2 * sizeof(unsigned long long), s)) != cudaSuccess)
        return set_error(SGL_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    if ((e = launch_max_radius_raw(s, xyz_dev, M, r2max, flags)) != cudaSuccess)
        return set_error(SGL_ERR_CUDA, std::string("max radius: ") + cudaGetErrorString(e));
    if ((e = launch_trig_raw(s, B, r2max, costab, P, radv, Kmat, beta, zeta, (const double2 *)coef_dev,
                             (double2 *)eta_dev)) != cudaSuccess)
        return set_error(SGL_ERR_CUDA, std::string("conversions: ") + cudaGetErrorString(e));
    set_error(SGL_OK, "");
    return SGL_OK;
}
