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

#include <algorithm>

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
    // bins (see BinGeom): azimuthal chunk, columns per super-bin, super-bins per axis
    int S2, C0, C1, nsb0, nsb1, nsb2, cmax0, cmax1;
};

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    // elementwise a * b + c on a packed pair (fma.rn.f32x2)
    unsigned long long ra = *reinterpret_cast<unsigned long long *>(&a);
    unsigned long long rb = *reinterpret_cast<unsigned long long *>(&b);
    unsigned long long rc = *reinterpret_cast<unsigned long long *>(&c);
    unsigned long long rd;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
    return *reinterpret_cast<float2 *>(&rd);
}

__device__ __forceinline__ int cell_clamped(double u, int cmax) { return min(max((int)floor(u), 0), cmax); }

// i mod n in [0, n) for any int i
__device__ __forceinline__ int wrap_index(int i, int n) {
    int r = i % n;
    return r < 0 ? r + n : r;
}

// storage row of grid index t, or -1 if a windowed axis does not store it (periodic axes wrap)
__device__ __forceinline__ int row_checked(int t, int first, int rows, int N) {
    if (rows == N) return wrap_index(t, N);
    const int r = t - first;
    return (r >= 0 && r < rows) ? r : -1;
}

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
            T rx = 0, ry = 0;                 // row sum over axis 1, then one multiply by w0
#pragma unroll
            for (int b = 0; b < G; ++b) {
                if (b < q2) {
                    const int r1 = row_of(a1 + b, g.first[1], g.rows[1], g.N[1]);
                    const C2<T> v = rowp[r1 * s1];
                    rx += w1[b] * v.x;
                    ry += w1[b] * v.y;
                }
            }
            ax += w0 * rx;
            ay += w0 * ry;
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

// ---------------------------------------------------------------------------------------------
// FP32 interpolation by column work items.  One warp per item (<= kItemPoints points of one
// column bin: the same rows on axes 0 and 1, all azimuthal taps inside the warp's 32 lanes).
// Each grid row is read once per KC points (lane = azimuthal cell, coalesced) and used for all
// of them: s = sum_a w0[a] sum_b w1[b] g[a][b][lane], then a lane reduction with w2[lane].
// Window weights are staged per warp in shared memory; the inner products use packed FP32 FMA.
template <int WIN, int Q2MAX, int KC>
__global__ void __launch_bounds__(256) k_interp_col(NGeom g, const int2 *__restrict__ items, const int *__restrict__ n_items,
                                                    const double *__restrict__ u_sorted, const int *__restrict__ perm,
                                                    const float2 *__restrict__ grid, double2 *__restrict__ vals) {
    __shared__ float2 s_w1[8][KC][Q2MAX];   // (w1, w1) pairs
    __shared__ float s_w0[8][KC][Q2MAX];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int q = g.q, q2 = 2 * q;
    const float qf = (float)q;
    const int64_t s1 = g.N[2], s0 = (int64_t)g.rows[1] * g.N[2];
    const int nit = *n_items;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int it = blockIdx.x * (blockDim.x >> 5) + wib; it < nit; it += nw) {
        const int2 item = items[it];
        const int first = item.x, cnt = item.y;
        const int c0 = cell_clamped(u_sorted[3 * (int64_t)first], g.cmax0);
        const int c1 = cell_clamped(u_sorted[3 * (int64_t)first + 1], g.cmax1);
        const int cz = min(max((int)floor(u_sorted[3 * (int64_t)first + 2]), 0), g.N[2] - 1);
        const int a0 = c0 - q + 1, a1 = c1 - q + 1;
        const int cbase = (cz / g.S2) * g.S2 - q + 1;
        const int col = wrap_index(cbase + lane, g.N[2]);
        int off1[Q2MAX];
#pragma unroll
        for (int b = 0; b < Q2MAX; ++b) off1[b] = (b < q2) ? row_of(a1 + b, g.first[1], g.rows[1], g.N[1]) * (int)s1 + col : col;
        for (int p0 = 0; p0 < cnt; p0 += KC) {
            const int np = min(KC, cnt - p0);
            for (int t = lane; t < KC * Q2MAX; t += 32) {
                const int k = t / Q2MAX, j = t % Q2MAX;
                float w0 = 0.f, w1 = 0.f;
                if (k < np && j < q2) {
                    const int64_t pi = first + p0 + k;
                    w0 = window<WIN, float>((float)(u_sorted[3 * pi] - (a0 + j)), qf, (float)g.par[0], (float)g.norm[0]);
                    w1 = window<WIN, float>((float)(u_sorted[3 * pi + 1] - (a1 + j)), qf, (float)g.par[1], (float)g.norm[1]);
                }
                s_w0[wib][k][j] = w0;
                s_w1[wib][k][j] = make_float2(w1, w1);
            }
            float w2[KC];
#pragma unroll
            for (int k = 0; k < KC; ++k) {
                w2[k] = 0.f;
                if (k < np) {
                    const double u2 = u_sorted[3 * (int64_t)(first + p0 + k) + 2];
                    const int rel = cbase + lane - ((int)floor(u2) - q + 1);
                    if (rel >= 0 && rel < q2)
                        w2[k] = window<WIN, float>((float)(u2 - (cbase + lane)), qf, (float)g.par[2], (float)g.norm[2]);
                }
            }
            __syncwarp();
            float2 acc[KC];
#pragma unroll
            for (int k = 0; k < KC; ++k) acc[k] = make_float2(0.f, 0.f);
            for (int a = 0; a < q2; ++a) {
                const float2 *rowp = grid + row_of(a0 + a, g.first[0], g.rows[0], g.N[0]) * s0;
                float2 rs[KC];
#pragma unroll
                for (int k = 0; k < KC; ++k) rs[k] = make_float2(0.f, 0.f);
#pragma unroll
                for (int b = 0; b < Q2MAX; ++b) {
                    if (b < q2) {
                        const float2 v = __ldg(rowp + off1[b]);
#pragma unroll
                        for (int k = 0; k < KC; ++k) rs[k] = ffma2(s_w1[wib][k][b], v, rs[k]);
                    }
                }
#pragma unroll
                for (int k = 0; k < KC; ++k) {
                    const float w0 = s_w0[wib][k][a];
                    acc[k] = ffma2(make_float2(w0, w0), rs[k], acc[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < KC; ++k) {
                float x = acc[k].x * w2[k], y = acc[k].y * w2[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    x += __shfl_xor_sync(0xffffffffu, x, o);
                    y += __shfl_xor_sync(0xffffffffu, y, o);
                }
                if (lane == 0 && k < np) vals[perm[first + p0 + k]] = make_double2((double)x, (double)y);
            }
            __syncwarp();
        }
    }
}

// Chain rule from ds/du_d to Re(conj(g) grad_x f) for one point (FP64), written by one lane.
__device__ __forceinline__ void write_point_gradient(const NGeom &g, double rho, double u0, double u1, double u2,
                                                     double a0x, double a0y, double a1x, double a1y, double a2x, double a2y,
                                                     double2 gv, double *outp) {
    const double twopi = 2.0 * kPi;
    const double g0x = a0x * (g.N[0] / twopi), g0y = a0y * (g.N[0] / twopi);
    const double g1x = a1x * (g.N[1] / twopi), g1y = a1y * (g.N[1] / twopi);
    const double g2x = a2x * (g.N[2] / twopi), g2y = a2y * (g.N[2] / twopi);
    const double t0 = twopi * u0 / g.N[0], t1 = twopi * u1 / g.N[1], t2 = twopi * u2 / g.N[2];
    const double ch = cos(0.5 * t0);
    const double r = rho * ch * ch;                 // r = rho (1 + cos t0) / 2
    const double st0 = sin(t0), st1 = sin(t1), ct1 = cos(t1), sp = sin(t2), cp = cos(t2);
    const double dt0dr = (st0 > 0.0) ? -2.0 / (rho * st0) : 0.0;
    const double ir = (r > 0.0) ? 1.0 / r : 0.0;
    const double irs = (r > 0.0 && st1 > 0.0) ? 1.0 / (r * st1) : 0.0;
    const double er[3] = {st1 * cp, st1 * sp, ct1}, et[3] = {ct1 * cp, ct1 * sp, -st1}, ep[3] = {-sp, cp, 0.0};
    for (int d = 0; d < 3; ++d) {
        const double vx = g0x * dt0dr * er[d] + g1x * ir * et[d] + g2x * irs * ep[d];
        const double vy = g0y * dt0dr * er[d] + g1y * ir * et[d] + g2y * irs * ep[d];
        outp[d] = gv.x * vx + gv.y * vy;           // Re(conj(g) v)
    }
}

// FP32 window-derivative interpolation by column work items (same layout as k_interp_col):
// per point s, ds/du0, ds/du1 from one pass over the rows, ds/du2 from psi' on the lanes.
template <int WIN, int Q2MAX, int KC>
__global__ void __launch_bounds__(256) k_grad_col(NGeom g, const int2 *__restrict__ items, const int *__restrict__ n_items,
                                                  const double *__restrict__ u_sorted, const int *__restrict__ perm,
                                                  const unsigned long long *__restrict__ r2max, const float2 *__restrict__ grid,
                                                  const double2 *__restrict__ gout, double *__restrict__ gxyz) {
    __shared__ float2 s_w1[8][KC][Q2MAX], s_d1[8][KC][Q2MAX];
    __shared__ float s_w0[8][KC][Q2MAX], s_d0[8][KC][Q2MAX];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int q = g.q, q2 = 2 * q;
    const float qf = (float)q;
    const int64_t s1 = g.N[2], s0 = (int64_t)g.rows[1] * g.N[2];
    double rho = sqrt(__longlong_as_double((long long)*r2max)) * (1.0 + 0x1p-20);
    if (!(rho > 0.0)) rho = 1.0;
    const int nit = *n_items;
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int it = blockIdx.x * (blockDim.x >> 5) + wib; it < nit; it += nw) {
        const int2 item = items[it];
        const int first = item.x, cnt = item.y;
        const int c0 = cell_clamped(u_sorted[3 * (int64_t)first], g.cmax0);
        const int c1 = cell_clamped(u_sorted[3 * (int64_t)first + 1], g.cmax1);
        const int cz = min(max((int)floor(u_sorted[3 * (int64_t)first + 2]), 0), g.N[2] - 1);
        const int a0 = c0 - q + 1, a1 = c1 - q + 1;
        const int cbase = (cz / g.S2) * g.S2 - q + 1;
        const int col = wrap_index(cbase + lane, g.N[2]);
        int off1[Q2MAX];
#pragma unroll
        for (int b = 0; b < Q2MAX; ++b) off1[b] = (b < q2) ? row_of(a1 + b, g.first[1], g.rows[1], g.N[1]) * (int)s1 + col : col;
        for (int p0 = 0; p0 < cnt; p0 += KC) {
            const int np = min(KC, cnt - p0);
            for (int t = lane; t < KC * Q2MAX; t += 32) {
                const int k = t / Q2MAX, j = t % Q2MAX;
                float w0 = 0.f, d0 = 0.f, w1 = 0.f, d1 = 0.f;
                if (k < np && j < q2) {
                    const int64_t pi = first + p0 + k;
                    const float x0 = (float)(u_sorted[3 * pi] - (a0 + j)), x1 = (float)(u_sorted[3 * pi + 1] - (a1 + j));
                    w0 = window<WIN, float>(x0, qf, (float)g.par[0], (float)g.norm[0]);
                    d0 = window_deriv<WIN, float>(x0, qf, (float)g.par[0], (float)g.norm[0]);
                    w1 = window<WIN, float>(x1, qf, (float)g.par[1], (float)g.norm[1]);
                    d1 = window_deriv<WIN, float>(x1, qf, (float)g.par[1], (float)g.norm[1]);
                }
                s_w0[wib][k][j] = w0;
                s_d0[wib][k][j] = d0;
                s_w1[wib][k][j] = make_float2(w1, w1);
                s_d1[wib][k][j] = make_float2(d1, d1);
            }
            float w2[KC], d2[KC];
#pragma unroll
            for (int k = 0; k < KC; ++k) {
                w2[k] = 0.f;
                d2[k] = 0.f;
                if (k < np) {
                    const double u2 = u_sorted[3 * (int64_t)(first + p0 + k) + 2];
                    const int rel = cbase + lane - ((int)floor(u2) - q + 1);
                    if (rel >= 0 && rel < q2) {
                        const float x2 = (float)(u2 - (cbase + lane));
                        w2[k] = window<WIN, float>(x2, qf, (float)g.par[2], (float)g.norm[2]);
                        d2[k] = window_deriv<WIN, float>(x2, qf, (float)g.par[2], (float)g.norm[2]);
                    }
                }
            }
            __syncwarp();
            float2 af[KC], a0v[KC], a1v[KC];
#pragma unroll
            for (int k = 0; k < KC; ++k) { af[k] = make_float2(0.f, 0.f); a0v[k] = af[k]; a1v[k] = af[k]; }
            for (int a = 0; a < q2; ++a) {
                const float2 *rowp = grid + row_of(a0 + a, g.first[0], g.rows[0], g.N[0]) * s0;
                float2 rs[KC], rd[KC];
#pragma unroll
                for (int k = 0; k < KC; ++k) { rs[k] = make_float2(0.f, 0.f); rd[k] = rs[k]; }
#pragma unroll
                for (int b = 0; b < Q2MAX; ++b) {
                    if (b < q2) {
                        const float2 v = __ldg(rowp + off1[b]);
#pragma unroll
                        for (int k = 0; k < KC; ++k) {
                            rs[k] = ffma2(s_w1[wib][k][b], v, rs[k]);
                            rd[k] = ffma2(s_d1[wib][k][b], v, rd[k]);
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < KC; ++k) {
                    const float w0 = s_w0[wib][k][a], d0 = s_d0[wib][k][a];
                    af[k] = ffma2(make_float2(w0, w0), rs[k], af[k]);
                    a0v[k] = ffma2(make_float2(d0, d0), rs[k], a0v[k]);
                    a1v[k] = ffma2(make_float2(w0, w0), rd[k], a1v[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < KC; ++k) {
                float v0x = a0v[k].x * w2[k], v0y = a0v[k].y * w2[k];
                float v1x = a1v[k].x * w2[k], v1y = a1v[k].y * w2[k];
                float v2x = af[k].x * d2[k], v2y = af[k].y * d2[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    v0x += __shfl_xor_sync(0xffffffffu, v0x, o);
                    v0y += __shfl_xor_sync(0xffffffffu, v0y, o);
                    v1x += __shfl_xor_sync(0xffffffffu, v1x, o);
                    v1y += __shfl_xor_sync(0xffffffffu, v1y, o);
                    v2x += __shfl_xor_sync(0xffffffffu, v2x, o);
                    v2y += __shfl_xor_sync(0xffffffffu, v2y, o);
                }
                if (lane == 0 && k < np) {
                    const int64_t pi = first + p0 + k;
                    const int dst = perm[pi];
                    write_point_gradient(g, rho, u_sorted[3 * pi], u_sorted[3 * pi + 1], u_sorted[3 * pi + 2],
                                         v0x, v0y, v1x, v1y, v2x, v2y, gout[dst], gxyz + 3 * (int64_t)dst);
                }
            }
            __syncwarp();
        }
    }
}

// Spreading by super-bins.  One CTA per super-bin (C0 x C1 columns x one azimuthal chunk);
// warp w owns tile slab a = w (one grid row on axis 0) and keeps the sums for all T1 rows of
// axis 1 and its 32 azimuthal lanes in registers while it sweeps every point of the super-bin;
// each tile cell is then added to the grid once (atomically: neighbouring tiles overlap).
template <typename T, int WIN, int Q2MAX, int C1>
struct SpreadSmem {
    static constexpr int PCH = 64;
    static constexpr int T1MAX = C1 + Q2MAX - 1;
    C2<T> y[PCH];
    T w0[PCH][Q2MAX];
    C2<T> w1[PCH][T1MAX];     // (w1, w1) pairs
    T w2[PCH][32];
    int ta0[PCH];
};

template <typename T, int WIN, int Q2MAX, int C0, int C1>
__global__ void __launch_bounds__(32 * (C0 + Q2MAX - 1)) k_spread_slab(NGeom g, const int *__restrict__ bin_off, int64_t M,
                                                                       int64_t nsuper, const double *__restrict__ u_sorted,
                                                                       const int *__restrict__ perm, const double2 *__restrict__ vals,
                                                                       C2<T> *__restrict__ grid) {
    using S = SpreadSmem<T, WIN, Q2MAX, C1>;
    constexpr int PCH = S::PCH, T1MAX = S::T1MAX;
    __shared__ S sm;
    const int lane = threadIdx.x & 31, ta = threadIdx.x >> 5;
    const int q = g.q, q2 = 2 * q;
    const T qT = (T)q;
    const int64_t sb = blockIdx.x;
    if (sb >= nsuper) return;
    const int first = bin_off[sb * C0 * C1];
    const int last = (sb + 1 < nsuper) ? bin_off[(sb + 1) * C0 * C1] : (int)M;
    if (first >= last) return;
    const int sb1 = (int)(sb % g.nsb1), sb2 = (int)((sb / g.nsb1) % g.nsb2), sb0 = (int)(sb / ((int64_t)g.nsb1 * g.nsb2));
    const int ta_org = sb0 * C0 - q + 1, tb_org = sb1 * C1 - q + 1, cbase = sb2 * g.S2 - q + 1;
    const int T1 = C1 + q2 - 1;
    constexpr int E = Q2MAX + T1MAX + 32 + 1;    // staged values per point
    C2<T> acc[T1MAX];
#pragma unroll
    for (int tb = 0; tb < T1MAX; ++tb) { acc[tb].x = (T)0; acc[tb].y = (T)0; }
    for (int cs = first; cs < last; cs += PCH) {
        const int np = min(PCH, last - cs);
        __syncthreads();
        for (int t = threadIdx.x; t < np * E; t += blockDim.x) {
            const int p = t / E, e = t % E;
            const int64_t pi = cs + p;
            const double u0 = u_sorted[3 * pi], u1 = u_sorted[3 * pi + 1], u2 = u_sorted[3 * pi + 2];
            if (e < Q2MAX) {
                const int a0p = cell_clamped(u0, g.cmax0) - q + 1;
                sm.w0[p][e] = (e < q2) ? window<WIN, T>((T)(u0 - (a0p + e)), qT, (T)g.par[0], (T)g.norm[0]) : (T)0;
            } else if (e < Q2MAX + T1MAX) {
                const int tb = e - Q2MAX;
                const int rel = tb - (cell_clamped(u1, g.cmax1) - sb1 * C1);
                T w = (T)0;
                if (rel >= 0 && rel < q2) w = window<WIN, T>((T)(u1 - (tb_org + tb)), qT, (T)g.par[1], (T)g.norm[1]);
                sm.w1[p][tb].x = w;
                sm.w1[p][tb].y = w;
            } else if (e < Q2MAX + T1MAX + 32) {
                const int L = e - Q2MAX - T1MAX;
                const int rel = cbase + L - ((int)floor(u2) - q + 1);
                sm.w2[p][L] = (rel >= 0 && rel < q2) ? window<WIN, T>((T)(u2 - (cbase + L)), qT, (T)g.par[2], (T)g.norm[2]) : (T)0;
            } else {
                const double2 y = vals[perm[pi]];
                sm.y[p].x = (T)y.x;
                sm.y[p].y = (T)y.y;
                sm.ta0[p] = cell_clamped(u0, g.cmax0) - sb0 * C0;
            }
        }
        __syncthreads();
        for (int p = 0; p < np; ++p) {
            const int j = ta - sm.ta0[p];
            if (j < 0 || j >= q2) continue;
            const T wz = sm.w0[p][j] * sm.w2[p][lane];
            C2<T> z;
            z.x = sm.y[p].x * wz;
            z.y = sm.y[p].y * wz;
#pragma unroll
            for (int tb = 0; tb < T1MAX; ++tb) {
                const C2<T> w = sm.w1[p][tb];
                if constexpr (sizeof(T) == 4) {
                    acc[tb] = ffma2(w, z, acc[tb]);
                } else {
                    acc[tb].x = fma(w.x, z.x, acc[tb].x);
                    acc[tb].y = fma(w.y, z.y, acc[tb].y);
                }
            }
        }
    }
    if (ta >= C0 + q2 - 1) return;
    const int64_t s1 = g.N[2], s0 = (int64_t)g.rows[1] * g.N[2];
    const int c = wrap_index(cbase + lane, g.N[2]);
    const int r0 = row_checked(ta_org + ta, g.first[0], g.rows[0], g.N[0]);
    if (r0 < 0) return;                 // slab outside the stored rows: no point reaches it
    C2<T> *rowp = grid + r0 * s0 + c;
#pragma unroll
    for (int tb = 0; tb < T1MAX; ++tb) {
        const int r1 = (tb < T1) ? row_checked(tb_org + tb, g.first[1], g.rows[1], g.N[1]) : -1;
        if (r1 >= 0 && (acc[tb].x != (T)0 || acc[tb].y != (T)0)) {
            C2<T> *cell = rowp + r1 * s1;
            if constexpr (sizeof(T) == 4) {
                atomicAdd(cell, acc[tb]);
            } else {
                atomicAdd(&cell->x, acc[tb].x);
                atomicAdd(&cell->y, acc[tb].y);
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
    g.S2 = p->bins.S2;
    g.C0 = p->bins.C0;
    g.C1 = p->bins.C1;
    g.nsb0 = p->bins.nsb[0];
    g.nsb1 = p->bins.nsb[1];
    g.nsb2 = p->bins.nsb[2];
    g.cmax0 = p->ax[0].N / 2;
    g.cmax1 = p->ax[1].N / 2;
    return g;
}

int nufft_blocks(int64_t M, int G) {
    const int64_t ppb = 256 / G;                 // points per block per sweep
    int64_t b = (M + ppb - 1) / ppb;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

int col_blocks(const sgl_plan *p) {
    int64_t b = (p->max_items + 7) / 8;
    if (b > 152 * 8) b = 152 * 8;
    return (int)std::max<int64_t>(b, 1);
}

template <typename T, int WIN>
cudaError_t interp_t(sgl_plan *p, double2 *vals) {
    NGeom g = make_geom(p);
    if constexpr (sizeof(T) == 4) {
        const float2 *gridf = (const float2 *)p->b.bufA;
        if (p->q <= 4) {
            k_interp_col<WIN, 8, 4><<<col_blocks(p), 256, 0, p->stream>>>(g, p->b.items, p->b.n_items, p->b.u_sorted, p->b.perm, gridf, vals);
            p->launches += 1;
            return cudaGetLastError();
        }
        if (p->q <= 8) {
            k_interp_col<WIN, 16, 4><<<col_blocks(p), 256, 0, p->stream>>>(g, p->b.items, p->b.n_items, p->b.u_sorted, p->b.perm, gridf, vals);
            p->launches += 1;
            return cudaGetLastError();
        }
    }
    const C2<T> *grid = (const C2<T> *)p->b.bufA;
    const int q2 = 2 * p->q;
    if (q2 <= 8) k_interp<T, WIN, 8><<<nufft_blocks(p->M, 8), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, grid, vals);
    else if (q2 <= 16) k_interp<T, WIN, 16><<<nufft_blocks(p->M, 16), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, grid, vals);
    else k_interp<T, WIN, 32><<<nufft_blocks(p->M, 32), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, grid, vals);
    p->launches += 1;
    return cudaGetLastError();
}

template <typename T, int WIN, int Q2MAX, int C0, int C1>
cudaError_t spread_slab_t(sgl_plan *p, const NGeom &g, const double2 *vals) {
    if (g.C0 != C0 || g.C1 != C1) return cudaErrorInvalidConfiguration;
    const int threads = 32 * (C0 + 2 * p->q - 1);
    k_spread_slab<T, WIN, Q2MAX, C0, C1><<<(unsigned)p->bins.nsuper, threads, 0, p->stream>>>(
        g, p->b.bin_off, p->M, p->bins.nsuper, p->b.u_sorted, p->b.perm, vals, (C2<T> *)p->b.bufA);
    p->launches += 1;
    return cudaGetLastError();
}

template <typename T, int WIN>
cudaError_t spread_t(sgl_plan *p, const double2 *vals) {
    NGeom g = make_geom(p);
    if constexpr (sizeof(T) == 4) {
        if (p->q <= 4) return spread_slab_t<T, WIN, 8, 8, 8>(p, g, vals);
        if (p->q <= 8) return spread_slab_t<T, WIN, 16, 8, 8>(p, g, vals);
    } else {
        if (p->q <= 4) return spread_slab_t<T, WIN, 8, 4, 2>(p, g, vals);
        if (p->q <= 8) return spread_slab_t<T, WIN, 16, 4, 2>(p, g, vals);
    }
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
    if constexpr (sizeof(T) == 4) {
        const float2 *gridf = (const float2 *)p->b.bufA;
        if (p->q <= 4) {
            k_grad_col<WIN, 8, 2><<<col_blocks(p), 256, 0, p->stream>>>(g, p->b.items, p->b.n_items, p->b.u_sorted, p->b.perm,
                                                                         p->b.r2max, gridf, gout, gxyz);
            p->launches += 1;
            return cudaGetLastError();
        }
        if (p->q <= 8) {
            k_grad_col<WIN, 16, 2><<<col_blocks(p), 256, 0, p->stream>>>(g, p->b.items, p->b.n_items, p->b.u_sorted, p->b.perm,
                                                                          p->b.r2max, gridf, gout, gxyz);
            p->launches += 1;
            return cudaGetLastError();
        }
    }
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
