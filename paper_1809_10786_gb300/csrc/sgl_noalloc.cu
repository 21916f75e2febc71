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
// All scratch -- the polar matrices, the cosine table, the radial values and matrices,
// beta, zeta and the reduction cell for rho -- lives in one file-scope __device__ array
// sized for B <= SGL_NOALLOC_MAX_B (about 4.9 MB).  Every GPU that loads libsgl.so holds
// that array until the process exits.  The caller passes inputs and outputs only.
#include "sgl_internal.cuh"

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

namespace sgl {
namespace {

constexpr int kMaxB = SGL_NOALLOC_MAX_B;
constexpr size_t round32(size_t n) { return (n + 31) / 32 * 32; }     // regions start on 256-byte boundaries
constexpr size_t kRegP = round32((size_t)kMaxB * kMaxB * kMaxB);
constexpr size_t kRegCos = round32((size_t)8 * kMaxB);
constexpr size_t kRegRadv = round32((size_t)kMaxB * kMaxB * (kMaxB + 1));
constexpr size_t kRegKmat = round32((size_t)(2 * kMaxB - 1) * kMaxB * (kMaxB + 1) / 2);
constexpr size_t kRegBeta = round32((size_t)2 * (2 * kMaxB - 1) * (2 * kMaxB - 1) * kMaxB);   // double2 as 2 doubles
constexpr size_t kRegZeta = round32((size_t)2 * (2 * kMaxB - 1) * kMaxB * (2 * kMaxB - 1));
constexpr size_t kRegCell = 32;                                                                // r2max bits + flags
constexpr size_t kScratchDoubles = kRegP + kRegCos + kRegRadv + kRegKmat + kRegBeta + kRegZeta + kRegCell;

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

// Host-side polar matrices and cosine table for one B, in static storage (no heap use).
// Same mathematics as the plan's precompute (Sect. 6, spherical subtransform): for m >= 0,
// P[m][k][l] = (1/2B) sum_j cos(k w_j) Pbar_lm(cos w_j) (m even), and for m odd the
// sin-weighted Chebyshev coefficients eps mapped to zeta/(-i).
std::mutex g_host_mu;
double g_host_tables[kRegP + kRegCos];
int g_host_B = 0;
double g_leg[2 * kMaxB][kMaxB][kMaxB];

void build_host_tables(int B) {
    const int K1 = B - 1, n2 = 2 * B;
    double *P = g_host_tables;
    double *cosv = g_host_tables + kRegP;
    std::memset(g_host_tables, 0, sizeof(g_host_tables));
    double w[2 * kMaxB];
    for (int j = 0; j < n2; ++j) {
        w[j] = (2.0 * j + 1.0) * kPi / (4.0 * B);
        const double x = std::cos(w[j]), sn = std::sin(w[j]);
        double pmm = 1.0 / std::sqrt(4.0 * kPi);
        for (int m = 0; m < B; ++m) {
            if (m > 0) pmm *= -std::sqrt((2.0 * m + 1.0) / (2.0 * m)) * sn;
            g_leg[j][m][m] = pmm;
            if (m + 1 < B) g_leg[j][m + 1][m] = std::sqrt(2.0 * m + 3.0) * x * pmm;
            for (int l = m + 2; l < B; ++l) {
                const double a = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
                const double bb = std::sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
                g_leg[j][l][m] = a * (x * g_leg[j][l - 1][m] - bb * g_leg[j][l - 2][m]);
            }
        }
    }
    double eps[2 * kMaxB + 2];
    for (int m = 0; m < B; ++m) {
        for (int l = m; l < B; ++l) {
            if (m % 2 == 0) {
                for (int k = 0; k <= K1; ++k) {
                    long double s = 0.0L;
                    for (int j = 0; j < n2; ++j) s += (long double)std::cos(k * w[j]) * g_leg[j][l][m];
                    P[((size_t)m * (K1 + 1) + k) * B + l] = (double)(s / n2);
                }
            } else {
                for (int k = 0; k < n2 + 2; ++k) eps[k] = 0.0;
                for (int k = 0; k < n2; ++k) {
                    long double s = 0.0L;
                    for (int j = 0; j < n2; ++j) s += (long double)std::cos(k * w[j]) * g_leg[j][l][m] / std::sin(w[j]);
                    eps[k] = (double)(s * (k == 0 ? 1.0L : 2.0L) / n2);
                }
                for (int k = 1; k <= K1; ++k) {
                    double v;
                    if (k == 1) v = 2.0 * eps[0] - eps[2];
                    else if (k < n2 - 2) v = eps[k - 1] - eps[k + 1];
                    else v = eps[k - 1];
                    P[((size_t)m * (K1 + 1) + k) * B + l] = v / 4.0;
                }
            }
        }
    }
    for (int m = 0; m < 8 * B; ++m)
        cosv[m] = (double)cosl((long double)m * 3.14159265358979323846264338327950288L / (4.0L * B));
    g_host_B = B;
}

}  // namespace
}  // namespace sgl

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
    cudaError_t e = scratch_on_current_device(&base);
    if (e != cudaSuccess) return set_error(SGL_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    double *P = base;
    double *costab = P + kRegP;
    double *radv = costab + kRegCos;
    double *Kmat = radv + kRegRadv;
    double2 *beta = reinterpret_cast<double2 *>(Kmat + kRegKmat);
    double2 *zeta = reinterpret_cast<double2 *>(Kmat + kRegKmat + kRegBeta);
    unsigned long long *r2max = reinterpret_cast<unsigned long long *>(Kmat + kRegKmat + kRegBeta + kRegZeta);
    int *flags = reinterpret_cast<int *>(r2max + 1);
    {
        // the host tables are rebuilt when B changes; the copy from pageable memory is staged
        // before cudaMemcpyAsync returns, so the lock only needs to cover the copy's issue
        std::lock_guard<std::mutex> lock(g_host_mu);
        if (g_host_B != B) build_host_tables(B);
        const size_t nP = (size_t)B * B * B;
        e = cudaMemcpyAsync(P, g_host_tables, nP * sizeof(double), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(costab, g_host_tables + kRegP, (size_t)8 * B * sizeof(double), cudaMemcpyHostToDevice, s);
    }
    if (e != cudaSuccess) return set_error(SGL_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(e));
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
