// sgl_inverse.cu -- the inverse transform (iNFSGLFT): SGL Fourier coefficients from scattered
// samples by conjugate gradients on the normal equations, one forward and one adjoint
// transform per iteration (Sect. 2, end, for the iNFFT; Sect. 7, end, for the NFSGLFT).
//
//   M >= Nc: least squares min ||f - Lambda c||, Lambda^H Lambda c = Lambda^H f: CGNR
//            (Golub and Van Loan, Alg. 10.4.1);
//   M <  Nc: minimum-norm solution, Lambda Lambda^H g = f, c = Lambda^H g: CGNE (Alg. 10.4.2).
//
// Vectors stay on the device; the squared norms are reduced per block in FP64 and summed on
// the host in long double, so the scalars alpha and beta are formed in extended precision as in
// the paper's last test.  Work vectors are allocated on the first call and owned by the plan.
#include "sgl_internal.cuh"

#include <algorithm>
#include <cmath>
#include <new>
#include <string>

namespace sgl {
namespace {

constexpr int kThreads = 256;

int blocks_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 1024));
}

// y += a x (complex vectors, real a)
__global__ void k_axpy(int64_t n, double a, const double2 *__restrict__ x, double2 *__restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = x[i];
        y[i].x = fma(a, v.x, y[i].x);
        y[i].y = fma(a, v.y, y[i].y);
    }
}

// y = x + b y
__global__ void k_xpby(int64_t n, const double2 *__restrict__ x, double b, double2 *__restrict__ y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = x[i];
        y[i].x = fma(b, y[i].x, v.x);
        y[i].y = fma(b, y[i].y, v.y);
    }
}

// z = x - y
__global__ void k_sub(int64_t n, const double2 *__restrict__ x, const double2 *__restrict__ y, double2 *__restrict__ z) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = make_double2(x[i].x - y[i].x, x[i].y - y[i].y);
}

// z = w x (real weights)
__global__ void k_weight(int64_t n, const double *__restrict__ w, const double2 *__restrict__ x, double2 *__restrict__ z) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z[i] = make_double2(w[i] * x[i].x, w[i] * x[i].y);
}

// per-block partial sums of |x_i|^2
__global__ void k_norm2_partials(int64_t n, const double2 *__restrict__ x, double *__restrict__ part) {
    __shared__ double red[kThreads / 32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = x[i];
        s = fma(v.x, v.x, fma(v.y, v.y, s));
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

}  // namespace

struct InverseWork {
    double2 *r = nullptr, *w = nullptr, *z = nullptr, *p = nullptr;
    double *part = nullptr;
    double *part_host = nullptr;
};

}  // namespace sgl

namespace {

using namespace sgl;

sgl_status cuda_fail(cudaError_t e, const char *what) {
    return set_error(SGL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ||x||^2, blocks reduced on the device, summed on the host in long double
sgl_status norm2(sgl_plan *p, const double2 *x, int64_t n, long double *out) {
    const int nb = blocks_for(n);
    k_norm2_partials<<<nb, kThreads, 0, p->stream>>>(n, x, p->inv->part);
    p->launches += 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->inv->part_host, p->inv->part, sizeof(double) * nb, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "norm");
    long double s = 0.0L;
    for (int b = 0; b < nb; ++b) s += (long double)p->inv->part_host[b];
    *out = s;
    return SGL_OK;
}

sgl_status ensure_work(sgl_plan *p) {
    if (p->inv) return SGL_OK;
    InverseWork *w = new (std::nothrow) InverseWork();
    if (!w) return set_error(SGL_ERR_ALLOC, "host allocation failed");
    const size_t Mc = (size_t)std::max<int64_t>(p->M_max, 1), Nc = (size_t)p->Nc;
    cudaError_t e = device_malloc((void **)&w->r, sizeof(double2) * Mc);
    if (e == cudaSuccess) e = device_malloc((void **)&w->w, sizeof(double2) * Mc);
    if (e == cudaSuccess) e = device_malloc((void **)&w->z, sizeof(double2) * Nc);
    if (e == cudaSuccess) e = device_malloc((void **)&w->p, sizeof(double2) * Nc);
    if (e == cudaSuccess) e = device_malloc((void **)&w->part, sizeof(double) * 1024);
    if (e == cudaSuccess) e = cudaMallocHost(&w->part_host, sizeof(double) * 1024);
    if (e != cudaSuccess) {
        cudaFree(w->r); cudaFree(w->w); cudaFree(w->z); cudaFree(w->p); cudaFree(w->part);
        if (w->part_host) cudaFreeHost(w->part_host);
        delete w;
        return set_error(SGL_ERR_ALLOC, std::string("inverse work vectors: ") + cudaGetErrorString(e));
    }
    p->inv = w;
    p->work_bytes += (int64_t)(sizeof(double2) * (2 * Mc + 2 * Nc) + sizeof(double) * 1024);
    return SGL_OK;
}

#define INV_TRY(expr) do { if (sgl_status _s = (expr)) return _s; } while (0)
#define INV_LAUNCH(k, n, ...) do { k<<<blocks_for(n), kThreads, 0, p->stream>>>(n, __VA_ARGS__); p->launches += 1; \
    if (cudaError_t _e = cudaGetLastError()) return cuda_fail(_e, #k); } while (0)

}  // namespace

namespace sgl {
void inverse_work_free(sgl_plan *p) {
    if (!p || !p->inv) return;
    cudaFree(p->inv->r);
    cudaFree(p->inv->w);
    cudaFree(p->inv->z);
    cudaFree(p->inv->p);
    cudaFree(p->inv->part);
    cudaFreeHost(p->inv->part_host);
    delete p->inv;
    p->inv = nullptr;
}
}  // namespace sgl

extern "C" {

sgl_status sgl_inverse(sgl_plan *p, const double *vals_dev, double *coef_dev, int iters, double tol, int method,
                       double *residual_out, int *iters_out) {
    if (!p) return set_error(SGL_ERR_ARG, "plan is NULL");
    if (!p->points_set) return set_error(SGL_ERR_STATE, "sgl_set_points has not been called");
    if (!coef_dev || ((uintptr_t)coef_dev & 7u) || (p->M > 0 && (!vals_dev || ((uintptr_t)vals_dev & 7u))))
        return set_error(SGL_ERR_ARG, "vals and coef must be non-NULL, 8-byte aligned device pointers");
    if (iters < 0 || !(tol >= 0.0)) return set_error(SGL_ERR_ARG, "iters must be >= 0 and tol >= 0");
    if (method < 0 || method > 2) return set_error(SGL_ERR_ARG, "method must be 0 (automatic), 1 (CGNR) or 2 (CGNE)");
    const int64_t M = p->M, Nc = p->Nc;
    const bool cgne = method == 2 || (method == 0 && M < Nc);
    INV_TRY(ensure_work(p));
    InverseWork &v = *p->inv;
    const double2 *f = (const double2 *)vals_dev;
    double2 *c = (double2 *)coef_dev;
    long double ff = 0.0L, rr = 0.0L;
    INV_TRY(norm2(p, f, M, &ff));
    // r = f - Lambda c0
    INV_TRY(sgl_forward(p, coef_dev, (double *)v.w));
    INV_LAUNCH(k_sub, M, f, v.w, v.r);
    INV_TRY(norm2(p, v.r, M, &rr));
    const long double stop = (long double)tol * (long double)tol * ff;
    int k = 0;
    if (!cgne) {
        // CGNR: z = Lambda^H r, p = z
        long double zz = 0.0L;
        INV_TRY(sgl_adjoint(p, (const double *)v.r, (double *)v.z));
        if (cudaError_t e = cudaMemcpyAsync(v.p, v.z, sizeof(double2) * Nc, cudaMemcpyDeviceToDevice, p->stream)) return cuda_fail(e, "copy");
        INV_TRY(norm2(p, v.z, Nc, &zz));
        for (; k < iters && rr > stop && zz > 0.0L; ++k) {
            long double ww = 0.0L;
            INV_TRY(sgl_forward(p, (const double *)v.p, (double *)v.w));          // w = Lambda p
            INV_TRY(norm2(p, v.w, M, &ww));
            if (!(ww > 0.0L)) break;
            const long double alpha = zz / ww;
            INV_LAUNCH(k_axpy, Nc, (double)alpha, v.p, c);                          // c += alpha p
            INV_LAUNCH(k_axpy, M, -(double)alpha, v.w, v.r);                        // r -= alpha w
            INV_TRY(sgl_adjoint(p, (const double *)v.r, (double *)v.z));          // z = Lambda^H r
            long double zz_new = 0.0L;
            INV_TRY(norm2(p, v.z, Nc, &zz_new));
            const long double beta = zz_new / zz;
            INV_LAUNCH(k_xpby, Nc, v.z, (double)beta, v.p);                         // p = z + beta p
            zz = zz_new;
            INV_TRY(norm2(p, v.r, M, &rr));
        }
    } else {
        // CGNE: p = Lambda^H r
        INV_TRY(sgl_adjoint(p, (const double *)v.r, (double *)v.p));
        for (; k < iters && rr > stop; ++k) {
            long double pp = 0.0L;
            INV_TRY(norm2(p, v.p, Nc, &pp));
            if (!(pp > 0.0L)) break;
            const long double alpha = rr / pp;
            INV_LAUNCH(k_axpy, Nc, (double)alpha, v.p, c);                          // c += alpha p
            INV_TRY(sgl_forward(p, (const double *)v.p, (double *)v.w));          // w = Lambda p
            INV_LAUNCH(k_axpy, M, -(double)alpha, v.w, v.r);                        // r -= alpha w
            long double rr_new = 0.0L;
            INV_TRY(norm2(p, v.r, M, &rr_new));
            const long double beta = rr_new / rr;
            INV_TRY(sgl_adjoint(p, (const double *)v.r, (double *)v.z));          // z = Lambda^H r
            INV_LAUNCH(k_xpby, Nc, v.z, (double)beta, v.p);                         // p = z + beta p
            rr = rr_new;
        }
    }
    if (residual_out) *residual_out = ff > 0.0L ? (double)std::sqrt(rr / ff) : 0.0;
    if (iters_out) *iters_out = k;
    return sgl_sync(p);
}

sgl_status sgl_midpoint_guess(sgl_plan *p, const double *vals_dev, const double *weights_dev, double *coef_dev) {
    if (!p) return set_error(SGL_ERR_ARG, "plan is NULL");
    if (!p->points_set) return set_error(SGL_ERR_STATE, "sgl_set_points has not been called");
    if (!coef_dev || ((uintptr_t)coef_dev & 7u) ||
        (p->M > 0 && (!vals_dev || !weights_dev || ((uintptr_t)vals_dev & 7u) || ((uintptr_t)weights_dev & 7u))))
        return set_error(SGL_ERR_ARG, "vals, weights and coef must be non-NULL, 8-byte aligned device pointers");
    INV_TRY(ensure_work(p));
    const int64_t M = p->M;
    INV_LAUNCH(k_weight, M, weights_dev, (const double2 *)vals_dev, p->inv->r);
    return sgl_adjoint(p, (const double *)p->inv->r, coef_dev);
}

}  // extern "C"
