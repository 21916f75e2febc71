// sgl_nufft_common.cuh -- window functions, grid geometry and index helpers shared by the
// interpolation / spreading kernels (SIMT in sgl_nufft.cu, tensor-core in sgl_nufft_tc.cu).
#pragma once

#include "sgl_dfl.cuh"
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
    float parf[3], normf[3];   // the same in binary32 (read from the parameter bank by the FP32 kernels)
    const double *wtab;        // tabulated windows (FP64 plans; see kWinNI)
    const float2 *wtab_df;     // the same coefficients as double-float pairs (h, l)
    double wh, winv;           // piece width q / kWinNI of the table, and its reciprocal
    float whf, winvf;          // the same in binary32 (exact: q / kWinNI is a short binary fraction)
    double tpn[3], ntp[3];     // 2 pi / N_d and N_d / (2 pi)
    // bins (see BinGeom): azimuthal chunk, columns per super-bin, super-bins per axis
    int S2, C0, C1, nsb0, nsb1, nsb2, cmax0, cmax1;
};

// psi (D = 0) or psi' (D = 1) of axis d from the table: the piece of |x| and its polynomial in the
// offset from the piece's midpoint (Horner); psi is even, psi' odd; zero for |x| > q
template <int D>
__device__ __forceinline__ double window_tab(const NGeom &g, int d, double x) {
    const double ax = fabs(x);
    if (ax > (double)g.q) return 0.0;
    const int i = min((int)(ax * g.winv), kWinNI - 1);
    const double t = ax - (i + 0.5) * g.wh;
    const double *c = g.wtab + ((d * 2 + D) * kWinNI + i) * (kWinDeg + 1);
    double r = __ldg(c + kWinDeg);
#pragma unroll
    for (int k = kWinDeg - 1; k >= 0; --k) r = fma(r, t, __ldg(c + k));
    return (D == 1 && x < 0.0) ? -r : r;
}

// window_tab for a double-float argument, from the double-float copy of the table, in
// double-float arithmetic on the FP32 pipe: |t| <= q / (2 kWinNI), so the terms of degree >= 8
// are below 1e-9 of psi's peak and take binary32 Horner steps; the others take double-float ones
template <int D>
__device__ __forceinline__ dfl window_tab_df(const NGeom &g, int d, dfl x) {
    const bool neg = x.h < 0.f;
    const dfl ax = neg ? -x : x;
    const float qf = (float)g.q;
    if (ax.h > qf || (ax.h == qf && ax.l > 0.f)) return dfl(0.f, 0.f);
    const int i = min((int)(ax.h * g.winvf), kWinNI - 1);
    const dfl t = ax - dfl(((float)i + 0.5f) * g.whf);         // the midpoint is exact in binary32
    const float2 *c = g.wtab_df + ((d * 2 + D) * kWinNI + i) * (kWinDeg + 1);
    float rf = __ldg(c + kWinDeg).x;
#pragma unroll
    for (int k = kWinDeg - 1; k >= 8; --k) rf = fmaf(rf, t.h, __ldg(c + k).x);
    dfl r(rf, 0.f);
#pragma unroll
    for (int k = 7; k >= 0; --k) {
        const float2 ck = __ldg(c + k);
        r = r * t + dfl(ck.x, ck.y);
    }
    return (D == 1 && neg) ? -r : r;
}

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

__device__ __forceinline__ void atomic_add_c(float2 *p, float x, float y) { atomicAdd(&p->x, x); atomicAdd(&p->y, y); }
__device__ __forceinline__ void atomic_add_c(double2 *p, double x, double y) { atomicAdd(&p->x, x); atomicAdd(&p->y, y); }

__device__ __forceinline__ void unpack_cells(float w, int &c0, int &c1, int &c2) {
    const int v = __float_as_int(w);
    c0 = v & 1023;
    c1 = (v >> 10) & 1023;
    c2 = (v >> 20) & 1023;
}

inline NGeom make_geom(const sgl_plan *p) {
    NGeom g{};
    for (int d = 0; d < 3; ++d) {
        g.N[d] = p->ax[d].N;
        g.rows[d] = p->ax[d].rows;
        g.first[d] = p->ax[d].first;
        g.par[d] = p->ax[d].wpar;
        g.norm[d] = (p->window == SGL_WIN_KB) ? p->q / (-expm1(-2.0 * p->ax[d].wpar * p->q)) : 1.0;
        g.parf[d] = (float)g.par[d];
        g.normf[d] = (float)g.norm[d];
        g.tpn[d] = 2.0 * kPi / p->ax[d].N;
        g.ntp[d] = p->ax[d].N / (2.0 * kPi);
    }
    g.q = p->q;
    g.wtab = p->b.wtab;
    g.wtab_df = p->b.wtab_df;
    g.wh = (double)p->q / kWinNI;
    g.winv = kWinNI / (double)p->q;
    g.whf = (float)g.wh;
    g.winvf = (float)g.winv;
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

// Chain rule in FP32 for one point: from the window-derivative sums v_d = ds/du_d (complex) to
// Re(conj(g) grad_x s), written as three doubles.  t_d = 2 pi u_d / N_d are the torus angles
// (r = rho (1 + cos t0) / 2, theta = t1, phi = t2); sincospi of t_d / pi keeps it in FP32.
__device__ __forceinline__ void grad_chain32(const NGeom &g, float rho, int c0, int c1, int c2, float f0, float f1, float f2,
                                             float v0x, float v0y, float v1x, float v1y, float v2x, float v2y, double2 gv,
                                             double *out) {
    // ds/dt_d = (N_d / 2 pi) ds/du_d;  t_d / pi = 2 u_d / N_d
    const float k0 = g.N[0] * 0.15915494309189535f, k1 = g.N[1] * 0.15915494309189535f, k2 = g.N[2] * 0.15915494309189535f;
    const float h0 = 2.f * ((float)c0 + f0) / g.N[0], h1 = 2.f * ((float)c1 + f1) / g.N[1], h2 = 2.f * ((float)c2 + f2) / g.N[2];
    float st0, ct0h, sth, st1, ct1, sp, cp;
    sincospif(h0, &st0, &ct0h);
    sincospif(0.5f * h0, &sth, &ct0h);          // cos(t0 / 2)
    sincospif(h1, &st1, &ct1);
    sincospif(h2, &sp, &cp);
    const float r = rho * ct0h * ct0h;            // r = rho (1 + cos t0) / 2
    const float dt0dr = (st0 > 0.f) ? -2.f / (rho * st0) : 0.f;
    const float ir = (r > 0.f) ? 1.f / r : 0.f;
    const float irs = (r > 0.f && st1 > 0.f) ? 1.f / (r * st1) : 0.f;
    const float er[3] = {st1 * cp, st1 * sp, ct1}, et[3] = {ct1 * cp, ct1 * sp, -st1}, ep[3] = {-sp, cp, 0.f};
    const float gx = (float)gv.x, gy = (float)gv.y;
    const float A = k0 * dt0dr, Bq = k1 * ir, Cq = k2 * irs;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float vx = A * v0x * er[d] + Bq * v1x * et[d] + Cq * v2x * ep[d];
        const float vy = A * v0y * er[d] + Bq * v1y * et[d] + Cq * v2y * ep[d];
        out[d] = (double)(gx * vx + gy * vy);     // Re(conj(g) v)
    }
}

// rho = max |x| (1 + 2^-20) from the bit pattern of max |x|^2 (1 if no point is away from the origin)
__device__ __forceinline__ float rho_from_r2max(const unsigned long long *r2max) {
    double rhod = sqrt(__longlong_as_double((long long)*r2max)) * (1.0 + 0x1p-20);
    if (!(rhod > 0.0)) rhod = 1.0;
    return (float)rhod;
}


// psi(x) and psi'(x) in FP32 for |x| <= q (zero outside), well-conditioned and branch-free
// (straight-line code, so the 16 taps of a point interleave): the Kaiser-Bessel exponent
// b (s - q) is evaluated as -b x^2 / (s + q), which has no cancellation near the peak.
// KB:    psi  = norm e^(b (s - q)) (1 - e^(-2 b s)) / s,   s = sqrt(q^2 - x^2)
//        psi' = -x norm e^(b (s - q)) (b s (1 + e^(-2bs)) - (1 - e^(-2bs))) / s^3
//        (limits s -> 0: psi -> 2 b norm e^(-bq), psi' -> -x (2/3) b^3 norm e^(-bq))
// Gauss: psi = exp(-x^2 / (2 lambda)),  psi' = -x / lambda psi.
template <int WIN>
__device__ __forceinline__ float2 window_pair32(float x, float q, float par, float norm) {
    const float s2 = fmaf(-x, x, q * q);
    float v, d;
    if (WIN == SGL_WIN_KB) {
        const float sv = sqrtf(fmaxf(s2, 0.f));
        const float e1 = expf(-__fdividef(par * x * x, sv + q));
        const float em = expf(-2.f * par * sv), om = 1.f - em;
        const float is = __fdividef(1.f, sv);
        const bool tiny = sv < 1e-3f;
        const float ebq = expf(-par * q);
        v = tiny ? 2.f * par * norm * ebq : norm * e1 * om * is;
        d = tiny ? -x * norm * ebq * (2.f / 3.f) * par * par * par : -x * norm * e1 * (par * sv * (1.f + em) - om) * is * is * is;
    } else {
        v = expf(-__fdividef(x * x, 2.f * par));
        d = -__fdividef(x, par) * v;
    }
    return (s2 >= 0.f) ? make_float2(v, d) : make_float2(0.f, 0.f);
}

// Point-parallel spreading for 2q > 16 (both precisions): G lanes per point, atomic adds per tap.
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

// blocks of 256 threads for a grid-stride sweep over the points
int nufft_blocks(int64_t M, int G) {
    const int64_t ppb = 256 / G;                 // points per block per sweep
    int64_t b = (M + ppb - 1) / ppb;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}


}  // namespace
}  // namespace sgl
