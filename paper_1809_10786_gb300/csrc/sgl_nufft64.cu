// sgl_nufft64.cu -- FP64 windowed interpolation (NFFT step 3, Sect. 2), its adjoint
// (spreading) and the window-derivative interpolation of the point gradient.
//
//   s(t) = sum_{l : |u_d - l_d| <= q} alpha_l prod_d psi_d(u_d - l_d),   u_d = N_d t_d / (2 pi)
//
// Taps per axis: l = floor(u) - q + 1 ... floor(u) + q (2q taps).  The FP64 pipe of GB300 runs
// at 1/64 of the FP32 rate, so it bounds every binary64 kernel here.  By default the three hot
// loops therefore run in double-float arithmetic instead: a value is the unevaluated sum hi + lo
// of two FP32 numbers, products and sums are carried out with the error-free transformations
// TwoProduct (Dekker; exact with a fused multiply-add) and TwoSum (Knuth), so every tap costs
// about a dozen FP32 operations and keeps a relative rounding error of order 2^-48 (binary64:
// 2^-53).  Their window values are binary64, read from per-axis polynomial tables (see kWinNI:
// a dozen FP64 operations instead of a square root, exponentials and a division); the final lane
// reductions and the chain rule stay binary64; the grid is split into (hi, lo) pairs in place by
// one pass before the interpolation, and spreading adds its double-float sums to the binary64
// grid.  SGL_FLAG_NATIVE_FP64 selects the binary64 loops (k_interp64, k_grad64, k_spread_slab64),
// which evaluate the windows directly.
#include "sgl_nufft_common.cuh"

namespace sgl {
namespace {

// ---- double-float helpers (rounded operations that the compiler may not fuse or reorder)
__device__ __forceinline__ void df_split(double x, float &h, float &l) {
    h = __double2float_rn(x);
    l = __double2float_rn(x - (double)h);
}

// acc += w * v for double-float w = wh + wl, v = vh + vl.  acc is kept as a running binary32
// sum ah (updated by TwoSum, exactly) and the accumulated rounding terms al; (double)ah +
// (double)al is the value.
__device__ __forceinline__ void df_fma(float &ah, float &al, float wh, float wl, float vh, float vl) {
    const float p = __fmul_rn(wh, vh);
    float e = fmaf(wh, vh, -p);                 // TwoProduct: wh vh = p + e exactly
    e = fmaf(wh, vl, e);
    e = fmaf(wl, vh, e);
    const float s = __fadd_rn(ah, p);          // TwoSum: ah + p = s + t exactly
    const float bv = __fsub_rn(s, ah);
    const float t = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bv)), __fsub_rn(p, bv));
    al = __fadd_rn(al, __fadd_rn(t, e));
    ah = s;
}

// (ph, pl) = w * v (double-float product, unnormalized)
__device__ __forceinline__ void df_mul(float &ph, float &pl, float wh, float wl, float vh, float vl) {
    ph = __fmul_rn(wh, vh);
    float e = fmaf(wh, vh, -ph);
    e = fmaf(wh, vl, e);
    pl = fmaf(wl, vh, e);
}

__device__ __forceinline__ double df_value(float h, float l) { return (double)h + (double)l; }

// a running pair (ah, al) of df_fma as a normalized double-float number (|ah| >= |al| holds for the
// sums here; a zero ah gives al itself)
__device__ __forceinline__ dfl df_norm(float ah, float al) { return fast_two_sum(ah, al); }
__device__ __forceinline__ dfl shfl_xor_df(dfl v, int o) {
    return dfl(__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o));
}
// the double-float window argument u - (c - q + 1 + j) = (u - c) + (q - 1 - j) (u - c exact in binary64)
__device__ __forceinline__ dfl tap_arg(double u, int c, int q, int j) { return df_split_bits(u - c) + dfl((float)(q - 1 - j)); }

// Double-float has the exponent range of binary32, and the SGL basis functions are polynomials
// that grow like r^(2B) (they are orthonormal under the weight e^{-|x|^2}), so grids and values
// of 1e40 and more are ordinary at moderate B.  Every double-float pass therefore works on
// data scaled by an exact power of two: max |x| over its input (the grid, or the values to
// spread) is reduced on the device and the pass multiplies by 2^-e on entry and by 2^e on exit,
// with max |x| 2^-e in [1/2, 1).  (Parts below max |x| 2^-100 would lose bits; relative to the
// sum they are below binary64's own rounding.)
__global__ void __launch_bounds__(256) k_max_abs(const double *__restrict__ x, int64_t n, unsigned long long *__restrict__ out) {
    __shared__ double ws[8];
    double m = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(x[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) m = fmax(m, ws[w]);
        atomicMax(out, (unsigned long long)__double_as_longlong(m));   // non-negative doubles order as integers
    }
}

// the exponent e of the scale for max |x| (0 when it is zero or not finite)
__device__ __forceinline__ int df_exponent(const unsigned long long *bits) {
    const double m = __longlong_as_double((long long)__ldg(bits));
    int e = 0;
    if (m > 0.0 && m <= 1.7976931348623157e308) frexp(m, &e);
    return e;
}

// binary64 grid -> double-float grid of grid * 2^-e, in place: cell (re, im) becomes
// (re_hi, im_hi, re_lo, im_lo)
__global__ void __launch_bounds__(256) k_split_grid(double2 *__restrict__ grid, int64_t n, const unsigned long long *__restrict__ maxbits) {
    float4 *out = reinterpret_cast<float4 *>(grid);
    const double sc = ldexp(1.0, -df_exponent(maxbits));
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = grid[i];
        float4 o;
        df_split(v.x * sc, o.x, o.z);
        df_split(v.y * sc, o.y, o.w);
        out[i] = o;
    }
}

// Chain rule from ds/du_d to Re(conj(g) grad_x f) for one point (FP64), called by every lane of
// the point's group of G lanes (gl = lane within the group), written by the group's lane 0 when
// `write`.  The transcendental functions and reciprocals are spread over lanes 0-2 of the group
// (one sincos and one reciprocal each) and gathered by shuffle: an FP64 warp instruction costs
// the FP64 pipe the same however few lanes are active.
template <int G>
__device__ __forceinline__ void point_gradient_lanes(const NGeom &g, int gl, double rho, double u0, double u1, double u2,
                                                     double a0x, double a0y, double a1x, double a1y, double a2x,
                                                     double a2y, bool write, double2 gv, double *outp) {
    const int lane = threadIdx.x & 31, base = lane - gl;
    const int sel = min(gl, 2);
    const double ud = sel == 0 ? u0 : (sel == 1 ? u1 : u2);
    double sn, cs;
    // lane 0: t0 / 2, lane 1: t1, lane 2: t2, as multiples of pi (t_d / pi = 2 u_d / N_d), so that the
    // singular places r = 0 (t0 = pi) and sin theta = 0 give exact zeros below
    sincospi(sel == 0 ? ud / g.N[0] : 2.0 * ud / g.N[sel], &sn, &cs);
    const double sh = __shfl_sync(0xffffffffu, sn, base, 32), ch = __shfl_sync(0xffffffffu, cs, base, 32);
    const double st1 = __shfl_sync(0xffffffffu, sn, base + 1, 32), ct1 = __shfl_sync(0xffffffffu, cs, base + 1, 32);
    const double sp = __shfl_sync(0xffffffffu, sn, base + 2, 32), cp = __shfl_sync(0xffffffffu, cs, base + 2, 32);
    const double st0 = 2.0 * sh * ch;                // sin t0
    const double r = rho * ch * ch;                  // r = rho (1 + cos t0) / 2
    // lane 0: dt0/dr = -2 / (rho sin t0); lane 1: 1 / r; lane 2: 1 / (r sin t1); zero where singular
    const double den = sel == 0 ? rho * st0 : (sel == 1 ? r : r * st1);
    const double num = sel == 0 ? -2.0 : 1.0;
    const double rec = den > 0.0 ? num / den : 0.0;
    const double dt0dr = __shfl_sync(0xffffffffu, rec, base, 32);
    const double ir = __shfl_sync(0xffffffffu, rec, base + 1, 32);
    const double irs = __shfl_sync(0xffffffffu, rec, base + 2, 32);
    if (!write) return;
    const double g0x = a0x * g.ntp[0], g0y = a0y * g.ntp[0];
    const double g1x = a1x * g.ntp[1], g1y = a1y * g.ntp[1];
    const double g2x = a2x * g.ntp[2], g2y = a2y * g.ntp[2];
    const double er[3] = {st1 * cp, st1 * sp, ct1}, et[3] = {ct1 * cp, ct1 * sp, -st1}, ep[3] = {-sp, cp, 0.0};
    for (int d = 0; d < 3; ++d) {
        const double vx = g0x * dt0dr * er[d] + g1x * ir * et[d] + g2x * irs * ep[d];
        const double vy = g0y * dt0dr * er[d] + g1y * ir * et[d] + g2y * irs * ep[d];
        outp[d] = gv.x * vx + gv.y * vy;           // Re(conj(g) v)
    }
}

// FP64 spreading.  The FP64 pipe is the bound (1/64 of the FP32 rate), so no lane may spend a
// DFMA on a zero weight: warp w owns tile slab a = w as above, but each half-warp h keeps the
// tile rows tb = 2i + h of axis 1, and lane l of a half the two azimuthal cells l and l + 16 of
// the 32-cell tile.  A point's 2q <= 16 taps on axis 2 start at tile cell s (its cell within the
// chunk), so [s, s + 2q) meets exactly one of each lane's two cells -- l if l >= s, else l + 16 --
// and the lane updates that accumulator (chosen by selects, on the integer pipe).
template <int Q2MAX, int C1>
struct Spread64Smem {
    static constexpr int PCH = 64;
    static constexpr int T1 = C1 + Q2MAX - 1;     // tile rows on axis 1 at the largest q
    static constexpr int RH = (T1 + 1) / 2;        // rows per half-warp
    double2 y[PCH];
    double w0[PCH][Q2MAX];
    double w1[PCH][2 * RH];   // axis-1 weights on the tile rows (0 off the point's taps)
    double w2[PCH][32];       // axis-2 weights on the 32 tile cells (0 off the point's taps)
    int ta0[PCH];             // the point's first slab within the tile (axis 0)
    int s2[PCH];              // the point's first tile cell on axis 2
};

template <int WIN, int Q2MAX, int C0, int C1>
__global__ void __launch_bounds__(32 * (C0 + Q2MAX - 1)) k_spread_slab64(NGeom g, const int4 *__restrict__ work,
                                                                         const int *__restrict__ work_len,
                                                                         const double *__restrict__ u_sorted,
                                                                         const int *__restrict__ perm, const double2 *__restrict__ vals,
                                                                         double2 *__restrict__ grid) {
    using S = Spread64Smem<Q2MAX, C1>;
    constexpr int PCH = S::PCH, RH = S::RH, T1P = 2 * RH;
    constexpr int E = Q2MAX + T1P + 32 + 1;      // staged values per point
    __shared__ __align__(16) S sm;
    const int lane = threadIdx.x & 31, ta = threadIdx.x >> 5, half = lane >> 4, l16 = lane & 15;
    const int q = g.q, q2 = 2 * q;
    const double qd = (double)q;
    if ((int)blockIdx.x >= __ldg(work_len)) return;
    const int4 piece = __ldg(work + blockIdx.x);
    const int64_t sb = piece.x;
    const int first = piece.y, last = piece.y + piece.z;
    const int sb1 = (int)(sb % g.nsb1), sb2 = (int)((sb / g.nsb1) % g.nsb2), sb0 = (int)(sb / ((int64_t)g.nsb1 * g.nsb2));
    const int ta_org = sb0 * C0 - q + 1, tb_org = sb1 * C1 - q + 1, cbase = sb2 * g.S2 - q + 1;
    const int T1 = C1 + q2 - 1;
    double2 lo[RH], hi[RH];
#pragma unroll
    for (int i = 0; i < RH; ++i) { lo[i] = make_double2(0.0, 0.0); hi[i] = make_double2(0.0, 0.0); }
    for (int cs = first; cs < last; cs += PCH) {
        const int np = min(PCH, last - cs);
        __syncthreads();
        for (int t = threadIdx.x; t < np * E; t += blockDim.x) {
            const int p = t / E, e = t % E;
            const int64_t pi = cs + p;
            const double u0 = u_sorted[3 * pi], u1 = u_sorted[3 * pi + 1], u2 = u_sorted[3 * pi + 2];
            const int c0 = cell_clamped(u0, g.cmax0), c1 = cell_clamped(u1, g.cmax1);
            const int c2 = min(max((int)floor(u2), 0), g.N[2] - 1);
            if (e < Q2MAX) {
                sm.w0[p][e] = (e < q2) ? window<WIN, double>(u0 - c0 + (double)(q - 1 - e), qd, g.par[0], g.norm[0]) : 0.0;
            } else if (e < Q2MAX + T1P) {
                const int tb = e - Q2MAX;
                const int rel = tb - (c1 - sb1 * C1);
                sm.w1[p][tb] = (rel >= 0 && rel < q2 && tb < T1)
                                   ? window<WIN, double>(u1 - c1 + (double)(q - 1 - rel), qd, g.par[1], g.norm[1]) : 0.0;
            } else if (e < Q2MAX + T1P + 32) {
                const int L = e - Q2MAX - T1P;
                const int rel = cbase + L - (c2 - q + 1);
                sm.w2[p][L] = (rel >= 0 && rel < q2) ? window<WIN, double>(u2 - c2 + (double)(q - 1 - rel), qd, g.par[2], g.norm[2])
                                                     : 0.0;
            } else {
                sm.y[p] = vals[perm[pi]];
                sm.ta0[p] = c0 - sb0 * C0;
                sm.s2[p] = c2 - q + 1 - cbase;
            }
        }
        __syncthreads();
        for (int p = 0; p < np; ++p) {
            const int j = ta - sm.ta0[p];
            if (j < 0 || j >= q2) continue;
            const bool up = l16 < sm.s2[p];
            const double wz = sm.w0[p][j] * sm.w2[p][up ? l16 + 16 : l16];
            const double2 y = sm.y[p];
            const double zx = y.x * wz, zy = y.y * wz;
#pragma unroll
            for (int i = 0; i < RH; ++i) {
                const double w = sm.w1[p][2 * i + half];
                double tx = up ? hi[i].x : lo[i].x, ty = up ? hi[i].y : lo[i].y;
                tx = fma(w, zx, tx);
                ty = fma(w, zy, ty);
                hi[i].x = up ? tx : hi[i].x;
                hi[i].y = up ? ty : hi[i].y;
                lo[i].x = up ? lo[i].x : tx;
                lo[i].y = up ? lo[i].y : ty;
            }
        }
    }
    if (ta >= C0 + q2 - 1) return;
    const int64_t s1 = g.N[2], s0 = (int64_t)g.rows[1] * g.N[2];
    const int r0 = row_checked(ta_org + ta, g.first[0], g.rows[0], g.N[0]);
    if (r0 < 0) return;                 // slab outside the stored rows: no point reaches it
    const int clo = wrap_index(cbase + l16, g.N[2]), chi = wrap_index(cbase + l16 + 16, g.N[2]);
    double2 *rowp = grid + r0 * s0;
#pragma unroll
    for (int i = 0; i < RH; ++i) {
        const int tb = 2 * i + half;
        const int r1 = (tb < T1) ? row_checked(tb_org + tb, g.first[1], g.rows[1], g.N[1]) : -1;
        if (r1 < 0) continue;
        double2 *row = rowp + r1 * s1;
        if (lo[i].x != 0.0 || lo[i].y != 0.0) {
            atomicAdd(&row[clo].x, lo[i].x);
            atomicAdd(&row[clo].y, lo[i].y);
        }
        if (hi[i].x != 0.0 || hi[i].y != 0.0) {
            atomicAdd(&row[chi].x, hi[i].x);
            atomicAdd(&row[chi].y, hi[i].y);
        }
    }
}

// FP64 path: same lane layout as the FP32 kernels, binary64 throughout (coordinates from the
// double grid coordinates); lane j evaluates tap j's weights once and shares them by shuffle.
template <int WIN, int G>
__global__ void __launch_bounds__(256) k_interp64(NGeom g, int64_t M, const double *__restrict__ u_sorted,
                                                  const int *__restrict__ perm, const double2 *__restrict__ grid,
                                                  double2 *__restrict__ vals) {
    const int lane = threadIdx.x & 31, gl = lane & (G - 1);
    const int q = g.q, q2 = 2 * q;
    const double qd = (double)q;
    const int64_t s1 = g.N[2], s0 = (int64_t)g.rows[1] * g.N[2];
    // warps sweep the bin-sorted points in grid-stride order (consecutive warps: neighbouring points)
    constexpr int PPW = 32 / G;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) / 32;
    const int64_t end = M;
    for (int64_t base = warp0 * PPW; base < M; base += nwarps * PPW) {
        const int64_t i = base + lane / G;
        const bool live = i < M;
        const int64_t ii = live ? i : end - 1;
        const double u0 = u_sorted[3 * ii], u1 = u_sorted[3 * ii + 1], u2 = u_sorted[3 * ii + 2];
        const int a0 = cell_clamped(u0, g.cmax0) - q + 1, a1 = cell_clamped(u1, g.cmax1) - q + 1;
        const int a2 = min(max((int)floor(u2), 0), g.N[2] - 1) - q + 1;
        const bool tap = gl < q2;
        const double w0_own = tap ? window<WIN, double>(u0 - (a0 + gl), qd, g.par[0], g.norm[0]) : 0.0;
        const double w1_own = tap ? window<WIN, double>(u1 - (a1 + gl), qd, g.par[1], g.norm[1]) : 0.0;
        const double w2 = tap ? window<WIN, double>(u2 - (a2 + gl), qd, g.par[2], g.norm[2]) : 0.0;
        const int col = tap ? wrap_index(a2 + gl, g.N[2]) : 0;
        double w1[G];
        int off1[G];
#pragma unroll
        for (int b = 0; b < G; ++b) {
            w1[b] = __shfl_sync(0xffffffffu, w1_own, b, G);
            off1[b] = (b < q2) ? row_of(a1 + b, g.first[1], g.rows[1], g.N[1]) * (int)s1 + col : col;
        }
        double ax = 0.0, ay = 0.0;
        for (int a = 0; a < q2; ++a) {
            const double w0 = __shfl_sync(0xffffffffu, w0_own, a, G);
            const double2 *rowp = grid + row_of(a0 + a, g.first[0], g.rows[0], g.N[0]) * s0;
            double rx = 0.0, ry = 0.0;
#pragma unroll
            for (int b = 0; b < G; ++b)
                if (b < q2) {
                    const double2 v = __ldg(rowp + off1[b]);
                    rx = fma(w1[b], v.x, rx);
                    ry = fma(w1[b], v.y, ry);
                }
            ax = fma(w0, rx, ax);
            ay = fma(w0, ry, ay);
        }
        ax *= w2;
        ay *= w2;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            ax += __shfl_xor_sync(0xffffffffu, ax, o);
            ay += __shfl_xor_sync(0xffffffffu, ay, o);
        }
        if (live && gl == 0) vals[perm[i]] = make_double2(ax, ay);
    }
}

template <int WIN, int G>
__global__ void __launch_bounds__(256) k_grad64(NGeom g, int64_t M, const double *__restrict__ u_sorted,
                                                const int *__restrict__ perm, const unsigned long long *__restrict__ r2max,
                                                const double2 *__restrict__ grid, const double2 *__restrict__ gout,
                                                double *__restrict__ gxyz, double2 *__restrict__ vals) {
    const int lane = threadIdx.x & 31, gl = lane & (G - 1);
    const int q = g.q, q2 = 2 * q;
    const double qd = (double)q;
    const int64_t s1 = g.N[2], s0 = (int64_t)g.rows[1] * g.N[2];
    double rho = sqrt(__longlong_as_double((long long)*r2max)) * (1.0 + 0x1p-20);
    if (!(rho > 0.0)) rho = 1.0;
    // warps sweep the bin-sorted points in grid-stride order (consecutive warps: neighbouring points)
    constexpr int PPW = 32 / G;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) / 32;
    const int64_t end = M;
    for (int64_t base = warp0 * PPW; base < M; base += nwarps * PPW) {
        const int64_t i = base + lane / G;
        const bool live = i < M;
        const int64_t ii = live ? i : end - 1;
        const double u0 = u_sorted[3 * ii], u1 = u_sorted[3 * ii + 1], u2 = u_sorted[3 * ii + 2];
        const int a0 = cell_clamped(u0, g.cmax0) - q + 1, a1 = cell_clamped(u1, g.cmax1) - q + 1;
        const int a2 = min(max((int)floor(u2), 0), g.N[2] - 1) - q + 1;
        const bool tap = gl < q2;
        const double x0 = u0 - (a0 + gl), x1 = u1 - (a1 + gl), x2 = u2 - (a2 + gl);
        const double w0_own = tap ? window<WIN, double>(x0, qd, g.par[0], g.norm[0]) : 0.0;
        const double d0_own = tap ? window_deriv<WIN, double>(x0, qd, g.par[0], g.norm[0]) : 0.0;
        const double w1_own = tap ? window<WIN, double>(x1, qd, g.par[1], g.norm[1]) : 0.0;
        const double d1_own = tap ? window_deriv<WIN, double>(x1, qd, g.par[1], g.norm[1]) : 0.0;
        const double w2 = tap ? window<WIN, double>(x2, qd, g.par[2], g.norm[2]) : 0.0;
        const double d2 = tap ? window_deriv<WIN, double>(x2, qd, g.par[2], g.norm[2]) : 0.0;
        const int col = tap ? wrap_index(a2 + gl, g.N[2]) : 0;
        double fx = 0, fy = 0, ax = 0, ay = 0, bx = 0, by = 0;
        for (int a = 0; a < q2; ++a) {
            const double w0 = __shfl_sync(0xffffffffu, w0_own, a, G);
            const double dw0 = __shfl_sync(0xffffffffu, d0_own, a, G);
            const double2 *rowp = grid + row_of(a0 + a, g.first[0], g.rows[0], g.N[0]) * s0 + col;
            double rx = 0, ry = 0, sx = 0, sy = 0;
#pragma unroll
            for (int b = 0; b < G; ++b) {
                const double w1 = __shfl_sync(0xffffffffu, w1_own, b, G);
                const double d1 = __shfl_sync(0xffffffffu, d1_own, b, G);
                if (b < q2) {
                    const double2 v = __ldg(rowp + row_of(a1 + b, g.first[1], g.rows[1], g.N[1]) * s1);
                    rx = fma(w1, v.x, rx); ry = fma(w1, v.y, ry);
                    sx = fma(d1, v.x, sx); sy = fma(d1, v.y, sy);
                }
            }
            fx = fma(w0, rx, fx); fy = fma(w0, ry, fy);
            ax = fma(dw0, rx, ax); ay = fma(dw0, ry, ay);
            bx = fma(w0, sx, bx); by = fma(w0, sy, by);
        }
        double f2x = d2 * fx, f2y = d2 * fy;
        double sx = w2 * fx, sy = w2 * fy;             // the value s itself (forward with gradient)
        ax *= w2; ay *= w2; bx *= w2; by *= w2;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            ax += __shfl_xor_sync(0xffffffffu, ax, o);
            ay += __shfl_xor_sync(0xffffffffu, ay, o);
            bx += __shfl_xor_sync(0xffffffffu, bx, o);
            by += __shfl_xor_sync(0xffffffffu, by, o);
            f2x += __shfl_xor_sync(0xffffffffu, f2x, o);
            f2y += __shfl_xor_sync(0xffffffffu, f2y, o);
            if (vals) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
            }
        }
        {
            const bool w = live && gl == 0;
            const int dst = w ? perm[i] : 0;
            point_gradient_lanes<G>(g, gl, rho, u0, u1, u2, ax, ay, bx, by, f2x, f2y, w, w ? gout[dst] : make_double2(0.0, 0.0),
                                    gxyz + 3 * (int64_t)dst);
            if (w && vals) vals[dst] = make_double2(sx, sy);
        }
    }
}


// ---- double-float interpolation: same lane layout as k_interp64 (lane = azimuthal tap, the
// (2q)^2 rows of axes 0 and 1 swept by every lane), double-float products and sums.  The axis-1
// weights are shuffled per tap rather than kept in per-point arrays, so that four CTAs fit on an
// SM: the loop is bound by the latency of its grid loads, not by arithmetic.
template <int WIN, int G>
__global__ void __launch_bounds__(256, 4) k_interp64x(NGeom g, int64_t M, const double *__restrict__ u_sorted,
                                                   const int *__restrict__ perm, const float4 *__restrict__ grid,
                                                   const unsigned long long *__restrict__ maxbits, double2 *__restrict__ vals) {
    const int vexp = df_exponent(maxbits);
    const int lane = threadIdx.x & 31, gl = lane & (G - 1);
    const int q = g.q, q2 = 2 * q;
    const int64_t s1 = g.N[2], s0 = (int64_t)g.rows[1] * g.N[2];
    constexpr int PPW = 32 / G;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) / 32;
    for (int64_t base = warp0 * PPW; base < M; base += nwarps * PPW) {
        const int64_t i = base + lane / G;
        const bool live = i < M;
        const int64_t ii = live ? i : M - 1;
        const double u0 = u_sorted[3 * ii], u1 = u_sorted[3 * ii + 1], u2 = u_sorted[3 * ii + 2];
        const int c0 = cell_clamped(u0, g.cmax0), c1 = cell_clamped(u1, g.cmax1), c2 = min(max((int)floor(u2), 0), g.N[2] - 1);
        const int a0 = c0 - q + 1, a1 = c1 - q + 1, a2 = c2 - q + 1;
        const bool tap = gl < q2;
        // this lane's tap on each axis: double-float windows (FP32 pipe)
        const dfl w0 = tap ? window_tab_df<0>(g, 0, tap_arg(u0, c0, q, gl)) : dfl(0.f, 0.f);
        const dfl w1 = tap ? window_tab_df<0>(g, 1, tap_arg(u1, c1, q, gl)) : dfl(0.f, 0.f);
        const dfl w2 = tap ? window_tab_df<0>(g, 2, tap_arg(u2, c2, q, gl)) : dfl(0.f, 0.f);
        const float w0h_own = w0.h, w0l_own = w0.l, w1h_own = w1.h, w1l_own = w1.l;
        const int col = tap ? wrap_index(a2 + gl, g.N[2]) : 0;

        float axh = 0.f, axl = 0.f, ayh = 0.f, ayl = 0.f;
        for (int a = 0; a < q2; ++a) {
            const float w0h = __shfl_sync(0xffffffffu, w0h_own, a, G), w0l = __shfl_sync(0xffffffffu, w0l_own, a, G);
            const float4 *rowp = grid + row_of(a0 + a, g.first[0], g.rows[0], g.N[0]) * s0 + col;
            float rxh = 0.f, rxl = 0.f, ryh = 0.f, ryl = 0.f;
#pragma unroll
            for (int b = 0; b < G; ++b) {
                const float w1h = __shfl_sync(0xffffffffu, w1h_own, b, G), w1l = __shfl_sync(0xffffffffu, w1l_own, b, G);
                if (b < q2) {
                    const float4 v = __ldg(rowp + row_of(a1 + b, g.first[1], g.rows[1], g.N[1]) * s1);
                    df_fma(rxh, rxl, w1h, w1l, v.x, v.z);
                    df_fma(ryh, ryl, w1h, w1l, v.y, v.w);
                }
            }
            df_fma(axh, axl, w0h, w0l, rxh, rxl);
            df_fma(ayh, ayl, w0h, w0l, ryh, ryl);
        }
        dfl ax = df_norm(axh, axl) * w2, ay = df_norm(ayh, ayl) * w2;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            ax = ax + shfl_xor_df(ax, o);
            ay = ay + shfl_xor_df(ay, o);
        }
        if (live && gl == 0) vals[perm[i]] = make_double2(df_to_double_scaled(ax, vexp), df_to_double_scaled(ay, vexp));
    }
}

// ---- double-float window-derivative interpolation (values, ds/du0, ds/du1, ds/du2), layout of k_grad64
template <int WIN, int G>
__global__ void __launch_bounds__(256, G == 8 ? 3 : 4) k_grad64x(NGeom g, int64_t M, const double *__restrict__ u_sorted,
                                                 const int *__restrict__ perm, const unsigned long long *__restrict__ r2max,
                                                 const float4 *__restrict__ grid, const unsigned long long *__restrict__ maxbits,
                                                 const double2 *__restrict__ gout, double *__restrict__ gxyz,
                                                 double2 *__restrict__ vals) {
    const int vexp = df_exponent(maxbits);
    const int lane = threadIdx.x & 31, gl = lane & (G - 1);
    const int q = g.q, q2 = 2 * q;
    const int64_t s1 = g.N[2], s0 = (int64_t)g.rows[1] * g.N[2];
    double rho = sqrt(__longlong_as_double((long long)*r2max)) * (1.0 + 0x1p-20);
    if (!(rho > 0.0)) rho = 1.0;
    constexpr int PPW = 32 / G;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) / 32;
    for (int64_t base = warp0 * PPW; base < M; base += nwarps * PPW) {
        const int64_t i = base + lane / G;
        const bool live = i < M;
        const int64_t ii = live ? i : M - 1;
        const double u0 = u_sorted[3 * ii], u1 = u_sorted[3 * ii + 1], u2 = u_sorted[3 * ii + 2];
        const int c0 = cell_clamped(u0, g.cmax0), c1 = cell_clamped(u1, g.cmax1), c2 = min(max((int)floor(u2), 0), g.N[2] - 1);
        const int a0 = c0 - q + 1, a1 = c1 - q + 1, a2 = c2 - q + 1;
        const bool tap = gl < q2;
        // this lane's tap on each axis: double-float psi and psi' (FP32 pipe)
        // (one axis at a time: the evaluations would otherwise interleave and spill)
        dfl w0(0.f, 0.f), d0 = w0, w1 = w0, d1 = w0, w2 = w0, d2 = w0;
        if (tap) {
#pragma unroll 1
            for (int k = 0; k < 3; ++k) {
                const dfl x = tap_arg(k == 0 ? u0 : (k == 1 ? u1 : u2), k == 0 ? c0 : (k == 1 ? c1 : c2), q, gl);
                const dfl w = window_tab_df<0>(g, k, x), d = window_tab_df<1>(g, k, x);
                if (k == 0) { w0 = w; d0 = d; } else if (k == 1) { w1 = w; d1 = d; } else { w2 = w; d2 = d; }
            }
        }
        const float w0h_own = w0.h, w0l_own = w0.l, d0h_own = d0.h, d0l_own = d0.l;
        const float w1h_own = w1.h, w1l_own = w1.l, d1h_own = d1.h, d1l_own = d1.l;
        const int col = tap ? wrap_index(a2 + gl, g.N[2]) : 0;
        float fxh = 0.f, fxl = 0.f, fyh = 0.f, fyl = 0.f;     // sum psi0 psi1 grid
        float axh = 0.f, axl = 0.f, ayh = 0.f, ayl = 0.f;     // sum psi0' psi1 grid
        float bxh = 0.f, bxl = 0.f, byh = 0.f, byl = 0.f;     // sum psi0 psi1' grid
        for (int a = 0; a < q2; ++a) {
            const float w0h = __shfl_sync(0xffffffffu, w0h_own, a, G), w0l = __shfl_sync(0xffffffffu, w0l_own, a, G);
            const float d0h = __shfl_sync(0xffffffffu, d0h_own, a, G), d0l = __shfl_sync(0xffffffffu, d0l_own, a, G);
            const float4 *rowp = grid + row_of(a0 + a, g.first[0], g.rows[0], g.N[0]) * s0 + col;
            float rxh = 0.f, rxl = 0.f, ryh = 0.f, ryl = 0.f, sxh = 0.f, sxl = 0.f, syh = 0.f, syl = 0.f;
#pragma unroll
            for (int b = 0; b < G; ++b) {
                const float w1h = __shfl_sync(0xffffffffu, w1h_own, b, G), w1l = __shfl_sync(0xffffffffu, w1l_own, b, G);
                const float d1h = __shfl_sync(0xffffffffu, d1h_own, b, G), d1l = __shfl_sync(0xffffffffu, d1l_own, b, G);
                if (b < q2) {
                    const float4 v = __ldg(rowp + row_of(a1 + b, g.first[1], g.rows[1], g.N[1]) * s1);
                    df_fma(rxh, rxl, w1h, w1l, v.x, v.z);
                    df_fma(ryh, ryl, w1h, w1l, v.y, v.w);
                    df_fma(sxh, sxl, d1h, d1l, v.x, v.z);
                    df_fma(syh, syl, d1h, d1l, v.y, v.w);
                }
            }
            df_fma(fxh, fxl, w0h, w0l, rxh, rxl);
            df_fma(fyh, fyl, w0h, w0l, ryh, ryl);
            df_fma(axh, axl, d0h, d0l, rxh, rxl);
            df_fma(ayh, ayl, d0h, d0l, ryh, ryl);
            df_fma(bxh, bxl, w0h, w0l, sxh, sxl);
            df_fma(byh, byl, w0h, w0l, syh, syl);
        }
        // the azimuthal weights and the reduction over the group in double-float, on 2^-vexp data
        const dfl fx = df_norm(fxh, fxl), fy = df_norm(fyh, fyl);
        dfl f2x = d2 * fx, f2y = d2 * fy;
        dfl sx = w2 * fx, sy = w2 * fy;                // the value s itself (forward with gradient)
        dfl ax = df_norm(axh, axl) * w2, ay = df_norm(ayh, ayl) * w2;
        dfl bx = df_norm(bxh, bxl) * w2, by = df_norm(byh, byl) * w2;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            ax = ax + shfl_xor_df(ax, o);
            ay = ay + shfl_xor_df(ay, o);
            bx = bx + shfl_xor_df(bx, o);
            by = by + shfl_xor_df(by, o);
            f2x = f2x + shfl_xor_df(f2x, o);
            f2y = f2y + shfl_xor_df(f2y, o);
            if (vals) {
                sx = sx + shfl_xor_df(sx, o);
                sy = sy + shfl_xor_df(sy, o);
            }
        }
        {
            const bool w = live && gl == 0;
            const int dst = w ? perm[i] : 0;
            point_gradient_lanes<G>(g, gl, rho, u0, u1, u2, df_to_double_scaled(ax, vexp), df_to_double_scaled(ay, vexp),
                                    df_to_double_scaled(bx, vexp), df_to_double_scaled(by, vexp), df_to_double_scaled(f2x, vexp),
                                    df_to_double_scaled(f2y, vexp), w, w ? gout[dst] : make_double2(0.0, 0.0),
                                    gxyz + 3 * (int64_t)dst);
            if (w && vals) vals[dst] = make_double2(df_to_double_scaled(sx, vexp), df_to_double_scaled(sy, vexp));
        }
    }
}

// ---- double-float spreading.  The two-cells-per-lane layout of k_spread_slab64 needs more
// registers in double-float than a CTA of C0 + 2q - 1 warps can give, so this kernel keeps one
// azimuthal cell per lane (the 32-cell tile on the 32 lanes; a point's 2q taps leave the other
// lanes adding zeros -- the FP32 pipe is 64 times the FP64 one, so idle lanes cost less than
// binary64 arithmetic would) and halves the accumulators instead: the whole work piece (at most
// spread_chunk(FP64) points) is staged once, then swept twice, for tile rows [0, RH) and
// [RH, C1 + 2q - 1), each sweep ending with its atomic flush.
template <int Q2MAX, int C1>
struct Spread64xSmem {
    static constexpr int PCH = SGL_SPREAD_CHUNK64;   // a whole work piece
    static constexpr int T1 = C1 + Q2MAX - 1;
    float4 y[PCH];
    float2 w0[PCH][Q2MAX];
    float2 w1[PCH][T1];
    float2 w2[PCH][32];
    int ta0[PCH];
};

template <int WIN, int Q2MAX, int C0, int C1>
__global__ void __launch_bounds__(32 * (C0 + Q2MAX - 1)) k_spread_slab64x(NGeom g, const int4 *__restrict__ work,
                                                                          const int *__restrict__ work_len,
                                                                          const double *__restrict__ u_sorted,
                                                                          const int *__restrict__ perm, const double2 *__restrict__ vals,
                                                                          const unsigned long long *__restrict__ maxbits,
                                                                          double2 *__restrict__ grid) {
    using S = Spread64xSmem<Q2MAX, C1>;
    constexpr int T1M = S::T1, RH = (T1M + 1) / 2;
    constexpr int E = 3 * Q2MAX + 1;             // staged items per point: the taps of three axes, the value
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S &sm = *reinterpret_cast<S *>(smem_raw);
    const int lane = threadIdx.x & 31, ta = threadIdx.x >> 5;
    const int q = g.q, q2 = 2 * q;
    if ((int)blockIdx.x >= __ldg(work_len)) return;
    const int vexp = df_exponent(maxbits);
    const int4 piece = __ldg(work + blockIdx.x);
    const int64_t sb = piece.x;
    const int cs = piece.y, np = min(piece.z, S::PCH);
    const int sb1 = (int)(sb % g.nsb1), sb2 = (int)((sb / g.nsb1) % g.nsb2), sb0 = (int)(sb / ((int64_t)g.nsb1 * g.nsb2));
    const int ta_org = sb0 * C0 - q + 1, tb_org = sb1 * C1 - q + 1, cbase = sb2 * g.S2 - q + 1;
    const int T1 = C1 + q2 - 1;
    // staging: the tile rows and lanes no tap reaches are zero; then only the 2q taps per axis are
    // evaluated (double-float windows on the FP32 pipe), and the values split into pairs with the
    // power-of-two scale 2^-vexp taken out of their exponents
    for (int t = threadIdx.x; t < np * (T1M + 32); t += blockDim.x) {
        const int p = t / (T1M + 32), e = t - p * (T1M + 32);
        if (e < T1M) sm.w1[p][e] = make_float2(0.f, 0.f);
        else sm.w2[p][e - T1M] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < np * E; t += blockDim.x) {
        const int p = t / E, e = t - p * E;
        const int64_t pi = cs + p;
        if (e < 3 * Q2MAX) {
            const int d = e / Q2MAX, j = e - d * Q2MAX;              // axis, tap
            if (j >= q2) continue;
            const double u = u_sorted[3 * pi + d];
            const int c = d == 0 ? cell_clamped(u, g.cmax0) : (d == 1 ? cell_clamped(u, g.cmax1) : min(max((int)floor(u), 0), g.N[d] - 1));
            const dfl x = df_split_bits(u - c) + dfl((float)(q - 1 - j));   // u - c exact; the tap's offset
            const dfl w = window_tab_df<0>(g, d, x);
            const float2 v = make_float2(w.h, w.l);
            if (d == 0) sm.w0[p][j] = v;
            else if (d == 1) sm.w1[p][c - sb1 * C1 + j] = v;
            else sm.w2[p][c - q + 1 + j - cbase] = v;
        } else {
            const double2 y = vals[perm[pi]];
            const dfl yx = df_split_bits(y.x, vexp), yy = df_split_bits(y.y, vexp);
            sm.y[p] = make_float4(yx.h, yy.h, yx.l, yy.l);
            sm.ta0[p] = cell_clamped(u_sorted[3 * pi], g.cmax0) - sb0 * C0;
        }
    }
    __syncthreads();
    if (ta >= C0 + q2 - 1) return;
    const int64_t s1 = g.N[2], s0 = (int64_t)g.rows[1] * g.N[2];
    const int r0 = row_checked(ta_org + ta, g.first[0], g.rows[0], g.N[0]);
    if (r0 < 0) return;                 // slab outside the stored rows: no point reaches it
    double2 *colp = grid + r0 * s0 + wrap_index(cbase + lane, g.N[2]);
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
        float4 acc[RH];
#pragma unroll
        for (int r = 0; r < RH; ++r) acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 2
        for (int p = 0; p < np; ++p) {
            const int j = ta - sm.ta0[p];
            if (j < 0 || j >= q2) continue;
            const float2 a = sm.w0[p][j], c = sm.w2[p][lane];
            const float4 y = sm.y[p];
            float wzh, wzl, zxh, zxl, zyh, zyl;
            df_mul(wzh, wzl, a.x, a.y, c.x, c.y);
            df_mul(zxh, zxl, wzh, wzl, y.x, y.z);
            df_mul(zyh, zyl, wzh, wzl, y.y, y.w);
#pragma unroll
            for (int r = 0; r < RH; ++r) {
                const int tb = pass * RH + r;
                if (tb < T1M) {
                    const float2 w = sm.w1[p][tb];
                    df_fma(acc[r].x, acc[r].y, w.x, w.y, zxh, zxl);
                    df_fma(acc[r].z, acc[r].w, w.x, w.y, zyh, zyl);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < RH; ++r) {
            const int tb = pass * RH + r;
            if (tb >= T1M || tb >= T1) continue;
            const int r1 = row_checked(tb_org + tb, g.first[1], g.rows[1], g.N[1]);
            // cells no point reached: skipped before any FP64 conversion
            if (r1 < 0 || (acc[r].x == 0.f && acc[r].y == 0.f && acc[r].z == 0.f && acc[r].w == 0.f)) continue;
            const double vx = df_to_double_scaled(dfl(acc[r].x, acc[r].y), vexp);
            const double vy = df_to_double_scaled(dfl(acc[r].z, acc[r].w), vexp);
            if (vx != 0.0 || vy != 0.0) {
                atomicAdd(&colp[r1 * s1].x, vx);
                atomicAdd(&colp[r1 * s1].y, vy);
            }
        }
    }
}

// max |x| of n doubles into bits (zeroed first)
cudaError_t max_abs(sgl_plan *p, const double *x, int64_t n, unsigned long long *bits) {
    cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(unsigned long long), p->stream);
    if (e != cudaSuccess) return e;
    k_max_abs<<<nufft_blocks(n, 1), 256, 0, p->stream>>>(x, n, bits);
    p->launches += 1;
    return cudaGetLastError();
}

cudaError_t split_grid(sgl_plan *p) {
    const int64_t n = (int64_t)p->ax[0].rows * p->ax[1].rows * p->ax[2].N;
    cudaError_t e = max_abs(p, (const double *)p->b.bufA, 2 * n, p->b.df_max);
    if (e != cudaSuccess) return e;
    k_split_grid<<<nufft_blocks(n, 1), 256, 0, p->stream>>>((double2 *)p->b.bufA, n, p->b.df_max);
    p->launches += 1;
    return cudaGetLastError();
}

template <int WIN>
cudaError_t interp64_t(sgl_plan *p, double2 *vals) {
    const NGeom g = make_geom(p);
    const double2 *gridd = (const double2 *)p->b.bufA;
    const int q2 = 2 * p->q;
    if (!(p->flags & SGL_FLAG_NATIVE_FP64)) {
        cudaError_t e = split_grid(p);
        if (e != cudaSuccess) return e;
        const float4 *gx = (const float4 *)p->b.bufA;
        if (q2 <= 8) k_interp64x<WIN, 8><<<nufft_blocks(p->M, 8), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, gx, p->b.df_max, vals);
        else if (q2 <= 16) k_interp64x<WIN, 16><<<nufft_blocks(p->M, 16), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, gx, p->b.df_max, vals);
        else k_interp64x<WIN, 32><<<nufft_blocks(p->M, 32), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, gx, p->b.df_max, vals);
        p->launches += 1;
        return cudaGetLastError();
    }
    if (q2 <= 8) k_interp64<WIN, 8><<<nufft_blocks(p->M, 8), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, gridd, vals);
    else if (q2 <= 16) k_interp64<WIN, 16><<<nufft_blocks(p->M, 16), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, gridd, vals);
    else k_interp64<WIN, 32><<<nufft_blocks(p->M, 32), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, gridd, vals);
    p->launches += 1;
    return cudaGetLastError();
}

template <int WIN, int Q2MAX, int C0, int C1, bool DF>
cudaError_t spread_slab64_t(sgl_plan *p, const NGeom &g, const double2 *vals) {
    if (g.C0 != C0 || g.C1 != C1 || g.S2 + 2 * p->q - 1 > 32) return cudaErrorInvalidConfiguration;
    const int threads = 32 * (C0 + 2 * p->q - 1);
    const int64_t blocks = work_list_cap(p->M, p->bins.nsuper, spread_chunk(p->prec));   // entries past work_len[1] return
    if constexpr (DF) {
        auto kern = k_spread_slab64x<WIN, Q2MAX, C0, C1>;
        const int smem = (int)sizeof(Spread64xSmem<Q2MAX, C1>);
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess) e = max_abs(p, (const double *)vals, 2 * p->M, p->b.df_max + 1);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)blocks, threads, smem, p->stream>>>(g, p->b.work[1], p->b.work_len + 1, p->b.u_sorted, p->b.perm, vals,
                                                            p->b.df_max + 1, (double2 *)p->b.bufA);
    } else {
        k_spread_slab64<WIN, Q2MAX, C0, C1><<<(unsigned)blocks, threads, 0, p->stream>>>(
            g, p->b.work[1], p->b.work_len + 1, p->b.u_sorted, p->b.perm, vals, (double2 *)p->b.bufA);
    }
    p->launches += 1;
    return cudaGetLastError();
}

template <int WIN>
cudaError_t spread64_t(sgl_plan *p, const double2 *vals) {
    const NGeom g = make_geom(p);
    const bool native = p->flags & SGL_FLAG_NATIVE_FP64;
    if (p->q <= 4) return native ? spread_slab64_t<WIN, 8, 4, 2, false>(p, g, vals) : spread_slab64_t<WIN, 8, 8, 4, true>(p, g, vals);
    if (p->q <= 8) return native ? spread_slab64_t<WIN, 16, 4, 2, false>(p, g, vals) : spread_slab64_t<WIN, 16, 8, 4, true>(p, g, vals);
    double2 *grid = (double2 *)p->b.bufA;
    k_spread<double, WIN, 32><<<nufft_blocks(p->M, 32), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, vals, grid);
    p->launches += 1;
    return cudaGetLastError();
}

template <int WIN>
cudaError_t grad64_t(sgl_plan *p, const double2 *gout, double *gxyz, double2 *vals) {
    const NGeom g = make_geom(p);
    const double2 *gridd = (const double2 *)p->b.bufA;
    const int q2 = 2 * p->q;
    if (!(p->flags & SGL_FLAG_NATIVE_FP64)) {
        cudaError_t e = split_grid(p);
        if (e != cudaSuccess) return e;
        const float4 *gx = (const float4 *)p->b.bufA;
        const unsigned long long *r2 = p->b.r2max;
        if (q2 <= 8)
            k_grad64x<WIN, 8><<<nufft_blocks(p->M, 8), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, r2, gx, p->b.df_max, gout, gxyz, vals);
        else if (q2 <= 16)
            k_grad64x<WIN, 16><<<nufft_blocks(p->M, 16), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, r2, gx, p->b.df_max, gout, gxyz, vals);
        else
            k_grad64x<WIN, 32><<<nufft_blocks(p->M, 32), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, r2, gx, p->b.df_max, gout, gxyz, vals);
        p->launches += 1;
        return cudaGetLastError();
    }
    if (q2 <= 8)
        k_grad64<WIN, 8><<<nufft_blocks(p->M, 8), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, p->b.r2max, gridd, gout, gxyz, vals);
    else if (q2 <= 16)
        k_grad64<WIN, 16><<<nufft_blocks(p->M, 16), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, p->b.r2max, gridd, gout, gxyz, vals);
    else
        k_grad64<WIN, 32><<<nufft_blocks(p->M, 32), 256, 0, p->stream>>>(g, p->M, p->b.u_sorted, p->b.perm, p->b.r2max, gridd, gout, gxyz, vals);
    p->launches += 1;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_max_abs(sgl_plan *p, const double *x, int64_t n, unsigned long long *bits) { return max_abs(p, x, n, bits); }

cudaError_t launch_interp64(sgl_plan *p, double2 *vals) {
    return p->window == SGL_WIN_KB ? interp64_t<SGL_WIN_KB>(p, vals) : interp64_t<SGL_WIN_GAUSS>(p, vals);
}

cudaError_t launch_spread64(sgl_plan *p, const double2 *vals) {
    return p->window == SGL_WIN_KB ? spread64_t<SGL_WIN_KB>(p, vals) : spread64_t<SGL_WIN_GAUSS>(p, vals);
}

cudaError_t launch_grad64(sgl_plan *p, const double2 *gout, double *gxyz, double2 *vals) {
    return p->window == SGL_WIN_KB ? grad64_t<SGL_WIN_KB>(p, gout, gxyz, vals) : grad64_t<SGL_WIN_GAUSS>(p, gout, gxyz, vals);
}

}  // namespace sgl
