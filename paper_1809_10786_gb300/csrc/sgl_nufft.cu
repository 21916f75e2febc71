// sgl_nufft.cu -- windowed interpolation (NFFT step 3, Sect. 2), its adjoint (spreading),
// and the window-derivative interpolation that gives the point gradient.
//
//   s(t) = sum_{l : |u_d - l_d| <= q} alpha_l prod_d psi_d(u_d - l_d),   u_d = N_d t_d / (2 pi)
//
// with psi the truncated, peak-normalized window (Kaiser-Bessel sinh form or the
// Gaussian of Sect. 2).  Taps per axis: l = floor(u) - q + 1 ... floor(u) + q (2q taps).
// A group of G lanes (G = 8, 16 or 32 >= 2q) handles one point: lane c owns the
// azimuthal tap c, loops over the (2q)^2 rows (axis 0, axis 1), and the group
// reduces with the azimuthal weights at the end.  Points are visited in bin order.
#include "sgl_internal.cuh"

namespace sgl {
namespace {

template <typename T> struct CT;
template <> struct CT<float> { using type = float2; };
template <> struct CT<double> { using type = double2; };
template <typename T> using C2 = typename CT<T>::type;

__device__ __forceinline__ float d_exp(float x) { return expf(x); }
__device__ __forceinline__ double d_exp(double x) { return exp(x); }
__device__ __forceinline__ float d_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double d_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float d_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double d_sqrt(double x) { return sqrt(x); }

// Window parameters of one axis, precomputed on the host.
struct WinAxis {
    double par;    // KB: shape b; Gauss: lambda
    double norm;   // KB: q / (1 - exp(-2 b q)); Gauss: unused
};

// psi(x) and d psi / dx for |x| <= q (0 outside); peak-normalized: psi(0) = 1.
// KB:    psi = [sinh(b s)/s] / [sinh(b q)/q],  s = sqrt(q^2 - x^2)
//           = norm * exp(b (s - q)) * (1 - exp(-2 b s)) / s
// Gauss: psi = exp(-x^2 / (2 lambda))
template <int WIN, typename T>
__device__ __forceinline__ T window(T x, T q, T par, T norm) {
    if (fabs(x) > q) return (T)0;
    if (WIN == SGL_WIN_KB) {
        const T s = d_sqrt(q * q - x * x);
        const T ratio = (s > (T)1e-6) ? -d_expm1(-(T)2 * par * s) / s : (T)2 * par;
        return norm * d_exp(par * (s - q)) * ratio;
    } else {
        return d_exp(-x * x / ((T)2 * par));
    }
}

template <int WIN, typename T>
__device__ __forceinline__ T window_deriv(T x, T q, T par, T norm) {
    if (fabs(x) > q) return (T)0;
    if (WIN == SGL_WIN_KB) {
        // d/dx [sinh(b s)/s] = -x (b s cosh(b s) - sinh(b s)) / s^3
        const T s = d_sqrt(q * q - x * x);
        if (s < (T)1e-4) return -x * norm * d_exp(-par * q) * ((T)2 / (T)3) * par * par * par;
        const T em = d_exp(-(T)2 * par * s);
        const T num = par * s * ((T)1 + em) - ((T)1 - em);
        return -x * norm * d_exp(par * (s - q)) * num / (s * s * s);
    } else {
        return -x / par * d_exp(-x * x / ((T)2 * par));
    }
}

struct NGeom {
    int N[3], rows[3], first[3];
    int q;
    double par[3], norm[3];
};

// storage row of grid index t on an axis (windowed rows start at first = -q, periodic rows wrap)
__device__ __forceinline__ int row_of(int t, int first, int rows, int N) {
    int r = t - first;
    if (r < 0) r += N;
    if (r >= rows) r -= N;
    return r;
}

template <typename T, int WIN, int G>
__global__ void __launch_bounds__(256) k_interp(NGeom g, int64_t M, const double *__restrict__ u_sorted,
                                                const int *__restrict__ perm, const C2<T> *__restrict__ grid,
                                                double2 *__restrict__ vals) {
    const int lane = threadIdx.x & 31;
    const int gl = lane % G;
    const int q2 = 2 * g.q;
    const T qT = (T)g.q;
    const int64_t ppw = 32 / G;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) / 32;
    const int64_t s1 = g.N[2], s0 = (int64_t)g.rows[1] * g.N[2];
    for (int64_t base = warp0 * ppw; base < M; base += nwarps * ppw) {
        const int64_t i = base + lane / G;
        const bool live = i < M;
        const int64_t ii = live ? i : M - 1;
        const double u0 = u_sorted[3 * ii], u1 = u_sorted[3 * ii + 1], u2 = u_sorted[3 * ii + 2];
        const int a0 = (int)floor(u0) - g.q + 1, a1 = (int)floor(u1) - g.q + 1, a2 = (int)floor(u2) - g.q + 1;
        T w1[G];
#pragma unroll
        for (int b = 0; b < G; ++b) w1[b] = (b < q2) ? window<WIN, T>((T)(u1 - (a1 + b)), qT, (T)g.par[1], (T)g.norm[1]) : (T)0;
        const T w2 = (gl < q2) ? window<WIN, T>((T)(u2 - (a2 + gl)), qT, (T)g.par[2], (T)g.norm[2]) : (T)0;
        int c = a2 + gl;
        if (c < 0) c += g.N[2];
        if (c >= g.N[2]) c -= g.N[2];
        if (gl >= q2) c = 0;
        T ax = 0, ay = 0;
        for (int a = 0; a < q2; ++a) {
            const T w0 = window<WIN, T>((T)(u0 - (a0 + a)), qT, (T)g.par[0], (T)g.norm[0]);
            const int r0 = row_of(a0 + a, g.first[0], g.rows[0], g.N[0]);
            const C2<T> *rowp = grid + r0 * s0 + c;
#pragma unroll
            for (int b = 0; b < G; ++b) {
                if (b < q2) {
                    const int r1 = row_of(a1 + b, g.first[1], g.rows[1], g.N[1]);
                    const C2<T> v = rowp[r1 * s1];
                    const T w = w0 * w1[b];
                    ax += w * v.x;
                    ay += w * v.y;
                }
            }
        }
        ax *= w2;
        ay *= w2;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            ax += __shfl_xor_sync(0xffffffffu, ax, o);
            ay += __shfl_xor_sync(0xffffffffu, ay, o);
        }
        if (live && gl == 0) vals[perm[i]] = make_double2((double)ax, (double)ay);
    }
}

__device__ __forceinline__ void atomic_add_c(float2 *p, float x, float y) { atomicAdd(&p->x, x); atomicAdd(&p->y, y); }
__device__ __forceinline__ void atomic_add_c(double2 *p, double x, double y) { atomicAdd(&p->x, x); atomicAdd(&p->y, y); }

template <typename T, int WIN, int G>
__global__ void __launch_bounds__(256) k_spread(NGeom g, int64_t M, const double *__restrict__ u_sorted,
                                                const int *__restrict__ perm, const double2 *__restrict__ vals,
                                                C2<T> *__restrict__ grid) {
    const int lane = threadIdx.x & 31;
    const int gl = lane % G;
    const int q2 = 2 * g.q;
    const T qT = (T)g.q;
    const int64_t ppw = 32 / G;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) / 32;
    const int64_t s1 = g.N[2], s0 = (int64_t)g.rows[1] * g.N[2];
    for (int64_t base = warp0 * ppw; base < M; base += nwarps * ppw) {
        const int64_t i = base + lane / G;
        if (i >= M || gl >= q2) continue;
        const double u0 = u_sorted[3 * i], u1 = u_sorted[3 * i + 1], u2 = u_sorted[3 * i + 2];
        const int a0 = (int)floor(u0) - g.q + 1, a1 = (int)floor(u1) - g.q + 1, a2 = (int)floor(u2) - g.q + 1;
        const double2 y = vals[perm[i]];
        const T w2 = window<WIN, T>((T)(u2 - (a2 + gl)), qT, (T)g.par[2], (T)g.norm[2]);
        const T yx = (T)y.x * w2, yy = (T)y.y * w2;
        int c = a2 + gl;
        if (c < 0) c += g.N[2];
        if (c >= g.N[2]) c -= g.N[2];
        for (int a = 0; a < q2; ++a) {
            const T w0 = window<WIN, T>((T)(u0 - (a0 + a)), qT, (T)g.par[0], (T)g.norm[0]);
            const int r0 = row_of(a0 + a, g.first[0], g.rows[0], g.N[0]);
            C2<T> *rowp = grid + r0 * s0 + c;
            for (int b = 0; b < q2; ++b) {
                const T w = w0 * window<WIN, T>((T)(u1 - (a1 + b)), qT, (T)g.par[1], (T)g.norm[1]);
                const int r1 = row_of(a1 + b, g.first[1], g.rows[1], g.N[1]);
                atomic_add_c(rowp + r1 * s1, w * yx, w * yy);
            }
        }
    }
}

// gxyz[perm[i]] = Re(conj(g_i) grad_x s(t(x_i))): window derivatives give ds/du_d; the
// chain rule goes through t0 = arccos(2r/rho - 1), t1 = theta, t2 = phi.
template <typename T, int WIN, int G>
__global__ void __launch_bounds__(256) k_grad(NGeom g, int64_t M, const double *__restrict__ u_sorted,
                                              const int *__restrict__ perm, const unsigned long long *__restrict__ r2max,
                                              const C2<T> *__restrict__ grid, const double2 *__restrict__ gout,
                                              double *__restrict__ gxyz) {
    const int lane = threadIdx.x & 31;
    const int gl = lane % G;
    const int q2 = 2 * g.q;
    const T qT = (T)g.q;
    const int64_t ppw = 32 / G;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) / 32;
    const int64_t s1 = g.N[2], s0 = (int64_t)g.rows[1] * g.N[2];
    double rho = sqrt(__longlong_as_double((long long)*r2max)) * (1.0 + 0x1p-20);
    if (!(rho > 0.0)) rho = 1.0;
    for (int64_t base = warp0 * ppw; base < M; base += nwarps * ppw) {
        const int64_t i = base + lane / G;
        const bool live = i < M;
        const int64_t ii = live ? i : M - 1;
        const double u0 = u_sorted[3 * ii], u1 = u_sorted[3 * ii + 1], u2 = u_sorted[3 * ii + 2];
        const int a0 = (int)floor(u0) - g.q + 1, a1 = (int)floor(u1) - g.q + 1, a2 = (int)floor(u2) - g.q + 1;
        T w1[G], d1[G];
#pragma unroll
        for (int b = 0; b < G; ++b) {
            const T x = (T)(u1 - (a1 + b));
            w1[b] = (b < q2) ? window<WIN, T>(x, qT, (T)g.par[1], (T)g.norm[1]) : (T)0;
            d1[b] = (b < q2) ? window_deriv<WIN, T>(x, qT, (T)g.par[1], (T)g.norm[1]) : (T)0;
        }
        const T x2 = (T)(u2 - (a2 + gl));
        const T w2 = (gl < q2) ? window<WIN, T>(x2, qT, (T)g.par[2], (T)g.norm[2]) : (T)0;
        const T d2 = (gl < q2) ? window_deriv<WIN, T>(x2, qT, (T)g.par[2], (T)g.norm[2]) : (T)0;
        int c = a2 + gl;
        if (c < 0) c += g.N[2];
        if (c >= g.N[2]) c -= g.N[2];
        if (gl >= q2) c = 0;
        T fx = 0, fy = 0, ax = 0, ay = 0, bx = 0, by = 0;   // s, ds/du0, ds/du1 before the axis-2 weight
        for (int a = 0; a < q2; ++a) {
            const T x0 = (T)(u0 - (a0 + a));
            const T w0 = window<WIN, T>(x0, qT, (T)g.par[0], (T)g.norm[0]);
            const T dw0 = window_deriv<WIN, T>(x0, qT, (T)g.par[0], (T)g.norm[0]);
            const int r0 = row_of(a0 + a, g.first[0], g.rows[0], g.N[0]);
            const C2<T> *rowp = grid + r0 * s0 + c;
            T rx = 0, ry = 0, sx = 0, sy = 0;
#pragma unroll
            for (int b = 0; b < G; ++b) {
                if (b < q2) {
                    const int r1 = row_of(a1 + b, g.first[1], g.rows[1], g.N[1]);
                    const C2<T> v = rowp[r1 * s1];
                    rx += w1[b] * v.x; ry += w1[b] * v.y;
                    sx += d1[b] * v.x; sy += d1[b] * v.y;
                }
            }
            fx += w0 * rx; fy += w0 * ry;
            ax += dw0 * rx; ay += dw0 * ry;
            bx += w0 * sx; by += w0 * sy;
        }
        // d/du of psi(u - l) is psi'(u - l)
        T f2x = d2 * fx, f2y = d2 * fy;
        fx *= w2; fy *= w2; ax *= w2; ay *= w2; bx *= w2; by *= w2;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            ax += __shfl_xor_sync(0xffffffffu, ax, o);
            ay += __shfl_xor_sync(0xffffffffu, ay, o);
            bx += __shfl_xor_sync(0xffffffffu, bx, o);
            by += __shfl_xor_sync(0xffffffffu, by, o);
            f2x += __shfl_xor_sync(0xffffffffu, f2x, o);
            f2y += __shfl_xor_sync(0xffffffffu, f2y, o);
        }
        if (live && gl == 0) {
            const double twopi = 2.0 * kPi;
            // ds/dt_d = (N_d / 2 pi) ds/du_d
            const double g0x = ax * (g.N[0] / twopi), g0y = ay * (g.N[0] / twopi);
            const double g1x = bx * (g.N[1] / twopi), g1y = by * (g.N[1] / twopi);
            const double g2x = f2x * (g.N[2] / twopi), g2y = f2y * (g.N[2] / twopi);
            const double t0 = twopi * u0 / g.N[0], t1 = twopi * u1 / g.N[1], t2 = twopi * u2 / g.N[2];
            const double ch = cos(0.5 * t0);
            const double r = rho * ch * ch;                 // r = rho (1 + cos t0) / 2
            const double st0 = sin(t0), st1 = sin(t1), ct1 = cos(t1), sp = sin(t2), cp = cos(t2);
            const double dt0dr = (st0 > 0.0) ? -2.0 / (rho * st0) : 0.0;
            const double ir = (r > 0.0) ? 1.0 / r : 0.0;
            const double irs = (r > 0.0 && st1 > 0.0) ? 1.0 / (r * st1) : 0.0;
            const double er[3] = {st1 * cp, st1 * sp, ct1}, et[3] = {ct1 * cp, ct1 * sp, -st1}, ep[3] = {-sp, cp, 0.0};
            const double2 gv = gout[perm[i]];
            double *outp = gxyz + 3 * (int64_t)perm[i];
            for (int d = 0; d < 3; ++d) {
                const double vx = g0x * dt0dr * er[d] + g1x * ir * et[d] + g2x * irs * ep[d];
                const double vy = g0y * dt0dr * er[d] + g1y * ir * et[d] + g2y * irs * ep[d];
                outp[d] = gv.x * vx + gv.y * vy;          // Re(conj(g) v)
            }
        }
    }
}

NGeom make_geom(const sgl_plan *p) {
    NGeom g{};
    for (int d = 0; d < 3; ++d) {
        g.N[d] = p->ax[d].N;
        g.rows[d] = p->ax[d].rows;
        g.first[d] = p->ax[d].first;
        g.par[d] = p->ax[d].wpar;
        g.norm[d] = (p->window == SGL_WIN_KB) ? p->q / (-expm1(-2.0 * p->ax[d].wpar * p->q)) : 1.0;
    }
    g.q = p->q;
    return g;
}

int nufft_blocks(int64_t M, int G) {
    const int64_t ppb = 256 / G;                 // points per block per sweep
    int64_t b = (M + ppb - 1) / ppb;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

template <typename T, int WIN>
cudaError_t interp_t(sgl_plan *p, double2 *vals) {
    NGeom g = make_geom(p);
    const C2<T> *grid = (const C2<T> *)p->b.bufA;
    const int q2 = 2 * p->q;
    if (q2 <= 8) k_interp<T, WIN, 8><<<nufft_blocks(p->M, 8), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, grid, vals);
    else if (q2 <= 16) k_interp<T, WIN, 16><<<nufft_blocks(p->M, 16), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, grid, vals);
    else k_interp<T, WIN, 32><<<nufft_blocks(p->M, 32), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, grid, vals);
    p->launches += 1;
    return cudaGetLastError();
}

template <typename T, int WIN>
cudaError_t spread_t(sgl_plan *p, const double2 *vals) {
    NGeom g = make_geom(p);
    C2<T> *grid = (C2<T> *)p->b.bufA;
    const int q2 = 2 * p->q;
    if (q2 <= 8) k_spread<T, WIN, 8><<<nufft_blocks(p->M, 8), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, vals, grid);
    else if (q2 <= 16) k_spread<T, WIN, 16><<<nufft_blocks(p->M, 16), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, vals, grid);
    else k_spread<T, WIN, 32><<<nufft_blocks(p->M, 32), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, vals, grid);
    p->launches += 1;
    return cudaGetLastError();
}

template <typename T, int WIN>
cudaError_t grad_t(sgl_plan *p, const double2 *gout, double *gxyz) {
    NGeom g = make_geom(p);
    const C2<T> *grid = (const C2<T> *)p->b.bufA;
    const int q2 = 2 * p->q;
    if (q2 <= 8) k_grad<T, WIN, 8><<<nufft_blocks(p->M, 8), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, p->b.r2max, grid, gout, gxyz);
    else if (q2 <= 16) k_grad<T, WIN, 16><<<nufft_blocks(p->M, 16), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, p->b.r2max, grid, gout, gxyz);
    else k_grad<T, WIN, 32><<<nufft_blocks(p->M, 32), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, p->b.r2max, grid, gout, gxyz);
    p->launches += 1;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_interp(sgl_plan *p, double2 *vals) {
    if (p->M == 0) return cudaSuccess;
    const bool f32 = p->prec == SGL_FP32_MIXED, kb = p->window == SGL_WIN_KB;
    if (f32) return kb ? interp_t<float, SGL_WIN_KB>(p, vals) : interp_t<float, SGL_WIN_GAUSS>(p, vals);
    return kb ? interp_t<double, SGL_WIN_KB>(p, vals) : interp_t<double, SGL_WIN_GAUSS>(p, vals);
}

cudaError_t launch_spread(sgl_plan *p, const double2 *vals) {
    if (p->M == 0) return cudaSuccess;
    const bool f32 = p->prec == SGL_FP32_MIXED, kb = p->window == SGL_WIN_KB;
    if (f32) return kb ? spread_t<float, SGL_WIN_KB>(p, vals) : spread_t<float, SGL_WIN_GAUSS>(p, vals);
    return kb ? spread_t<double, SGL_WIN_KB>(p, vals) : spread_t<double, SGL_WIN_GAUSS>(p, vals);
}

cudaError_t launch_grad(sgl_plan *p, const double2 *gout, double *gxyz) {
    if (p->M == 0) return cudaSuccess;
    const bool f32 = p->prec == SGL_FP32_MIXED, kb = p->window == SGL_WIN_KB;
    if (f32) return kb ? grad_t<float, SGL_WIN_KB>(p, gout, gxyz) : grad_t<float, SGL_WIN_GAUSS>(p, gout, gxyz);
    return kb ? grad_t<double, SGL_WIN_KB>(p, gout, gxyz) : grad_t<double, SGL_WIN_GAUSS>(p, gout, gxyz);
}

}  // namespace sgl
