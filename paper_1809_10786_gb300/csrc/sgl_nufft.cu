// sgl_nufft.cu -- windowed interpolation (NFFT step 3, Sect. 2), its adjoint (spreading),
// and the window-derivative interpolation that gives the point gradient: the FP32 kernels on
// the CUDA cores, and the dispatch between them, the tensor-core kernels (sgl_nufft_tc.cu) and
// the FP64 kernels (sgl_nufft64.cu).
//
//   s(t) = sum_{l : |u_d - l_d| <= q} alpha_l prod_d psi_d(u_d - l_d),   u_d = N_d t_d / (2 pi)
//
// with psi the truncated, peak-normalized window (Kaiser-Bessel sinh form or the
// Gaussian of Sect. 2).  Taps per axis: l = floor(u) - q + 1 ... floor(u) + q (2q taps).
// A group of G lanes (G = 8, 16 or 32 >= 2q) handles one point: lane c owns the
// azimuthal tap c, loops over the (2q)^2 rows (axis 0, axis 1), and the group
// reduces with the azimuthal weights at the end.  Points are visited in bin order.
#include "sgl_nufft_common.cuh"

#include <algorithm>

namespace sgl {
namespace {

// ---------------------------------------------------------------------------------------------
// FP32 path.  Points come packed as float4 (fractional grid coordinates, cells in 10-bit fields),
// so window arguments are exact float sums (frac + integer offset) and no FP64 work is left in
// the loops (the FP64 pipe of GB300 runs at 1/64 of the FP32 rate).  G = 8/16/32 >= 2q lanes
// serve one point: lane j evaluates the weights of tap j on each axis and shares them by
// shuffle; the (2q)^2 rows are read once per point, lane = azimuthal tap, packed FP32 FMA.

// N2T: the axis-2 length (the row stride) as a compile-time constant (0: read it from g) -- with
// it the unrolled row loads use immediate offsets instead of per-load address arithmetic
template <int WIN, int G, bool LIN1, int N2T>
__global__ void __launch_bounds__(256) k_interp32(NGeom g, int64_t M, const float4 *__restrict__ pts, const int *__restrict__ perm,
                                                  const float2 *__restrict__ grid, double2 *__restrict__ vals) {
    const int lane = threadIdx.x & 31, gl = lane & (G - 1);
    const int q = g.q, q2 = 2 * q;
    const float qf = (float)q;
    const float par0 = (float)g.par[0], par1 = (float)g.par[1], par2 = (float)g.par[2];
    const float nrm0 = (float)g.norm[0], nrm1 = (float)g.norm[1], nrm2 = (float)g.norm[2];
    const int64_t s1 = N2T ? N2T : g.N[2], s0 = (int64_t)g.rows[1] * s1;
    // warps sweep the bin-sorted points in grid-stride order (consecutive warps: neighbouring points)
    constexpr int PPW = 32 / G;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) / 32;
    const int64_t end = M;
    for (int64_t base = warp0 * PPW; base < M; base += nwarps * PPW) {
        const int64_t i = base + lane / G;
        const bool live = i < M;
        const float4 pt = pts[live ? i : end - 1];
        int c0, c1, c2;
        unpack_cells(pt.w, c0, c1, c2);
        const int a0 = c0 - q + 1, a1 = c1 - q + 1, a2 = c2 - q + 1;
        const bool tap = gl < q2;
        const float off = (float)(q - 1 - gl);          // u - (a + gl) = frac + q - 1 - gl
        const float w0_own = tap ? window<WIN, float>(pt.x + off, qf, par0, nrm0) : 0.f;
        const float w1_own = tap ? window<WIN, float>(pt.y + off, qf, par1, nrm1) : 0.f;
        const float w2 = tap ? window<WIN, float>(pt.z + off, qf, par2, nrm2) : 0.f;
        const int col = tap ? wrap_index(a2 + gl, (int)s1) : 0;
        float2 w1p[G];
#pragma unroll
        for (int b = 0; b < G; ++b) {
            const float w = __shfl_sync(0xffffffffu, w1_own, b, G);
            w1p[b] = make_float2(w, w);
        }
        // LIN1: windowed axis 1, rows a1 + b stored contiguously from row a1 - first
        const int64_t r1base = LIN1 ? (int64_t)(a1 - g.first[1]) * s1 + col : col;
        float2 acc = make_float2(0.f, 0.f);
        for (int a = 0; a < q2; ++a) {
            const float w0 = __shfl_sync(0xffffffffu, w0_own, a, G);
            const float2 *rowp = grid + row_of(a0 + a, g.first[0], g.rows[0], g.N[0]) * s0 + r1base;
            float2 rs = make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < G; ++b)
                if (b < q2) rs = ffma2(w1p[b], __ldg(rowp + (LIN1 ? b * s1 : row_of(a1 + b, g.first[1], g.rows[1], g.N[1]) * s1)), rs);
            acc = ffma2(make_float2(w0, w0), rs, acc);
        }
        float x = acc.x * w2, y = acc.y * w2;
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
        }
        if (live && gl == 0) vals[perm[i]] = make_double2((double)x, (double)y);
    }
}

// FP32 window-derivative interpolation: s, ds/du0, ds/du1 in one sweep of the rows, ds/du2 from
// psi' on the lanes, then the chain rule in FP32 (sincospi of the torus coordinates).
// N2T: the axis-2 length (the row stride) as a compile-time constant (0: read it from g) -- with
// it the unrolled row loads use immediate offsets instead of per-load address arithmetic
template <int WIN, int G, bool LIN1, int N2T>
__global__ void __launch_bounds__(256, 3) k_grad32(NGeom g, int64_t M, const float4 *__restrict__ pts, const int *__restrict__ perm,
                                                const unsigned long long *__restrict__ r2max, const float2 *__restrict__ grid,
                                                const double2 *__restrict__ gout, double *__restrict__ gxyz,
                                                double2 *__restrict__ vals) {
    const int lane = threadIdx.x & 31, gl = lane & (G - 1);
    const int q = g.q, q2 = 2 * q;
    const float qf = (float)q;
    const float par0 = (float)g.par[0], par1 = (float)g.par[1], par2 = (float)g.par[2];
    const float nrm0 = (float)g.norm[0], nrm1 = (float)g.norm[1], nrm2 = (float)g.norm[2];
    const int64_t s1 = N2T ? N2T : g.N[2], s0 = (int64_t)g.rows[1] * s1;
    double rhod = sqrt(__longlong_as_double((long long)*r2max)) * (1.0 + 0x1p-20);
    if (!(rhod > 0.0)) rhod = 1.0;
    const float rho = (float)rhod;
    // warps sweep the bin-sorted points in grid-stride order (consecutive warps: neighbouring points)
    constexpr int PPW = 32 / G;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) / 32;
    const int64_t end = M;
    for (int64_t base = warp0 * PPW; base < M; base += nwarps * PPW) {
        const int64_t i = base + lane / G;
        const bool live = i < M;
        const float4 pt = pts[live ? i : end - 1];
        int c0, c1, c2;
        unpack_cells(pt.w, c0, c1, c2);
        const int a0 = c0 - q + 1, a1 = c1 - q + 1, a2 = c2 - q + 1;
        const bool tap = gl < q2;
        const float off = (float)(q - 1 - gl);
        const float x0 = pt.x + off, x1 = pt.y + off, x2 = pt.z + off;
        const float w0_own = tap ? window<WIN, float>(x0, qf, par0, nrm0) : 0.f;
        const float d0_own = tap ? window_deriv<WIN, float>(x0, qf, par0, nrm0) : 0.f;
        const float w1_own = tap ? window<WIN, float>(x1, qf, par1, nrm1) : 0.f;
        const float d1_own = tap ? window_deriv<WIN, float>(x1, qf, par1, nrm1) : 0.f;
        const float w2 = tap ? window<WIN, float>(x2, qf, par2, nrm2) : 0.f;
        const float d2 = tap ? window_deriv<WIN, float>(x2, qf, par2, nrm2) : 0.f;
        const int col = tap ? wrap_index(a2 + gl, (int)s1) : 0;
        float2 w1p[G], d1p[G];
#pragma unroll
        for (int b = 0; b < G; ++b) {
            const float w = __shfl_sync(0xffffffffu, w1_own, b, G);
            const float d = __shfl_sync(0xffffffffu, d1_own, b, G);
            w1p[b] = make_float2(w, w);
            d1p[b] = make_float2(d, d);
        }
        const int64_t r1base = LIN1 ? (int64_t)(a1 - g.first[1]) * s1 + col : col;
        float2 af = make_float2(0.f, 0.f), ad0 = af, ad1 = af;
        for (int a = 0; a < q2; ++a) {
            const float w0 = __shfl_sync(0xffffffffu, w0_own, a, G);
            const float d0 = __shfl_sync(0xffffffffu, d0_own, a, G);
            const float2 *rowp = grid + row_of(a0 + a, g.first[0], g.rows[0], g.N[0]) * s0 + r1base;
            float2 rs = make_float2(0.f, 0.f), rd = rs;
#pragma unroll
            for (int b = 0; b < G; ++b)
                if (b < q2) {
                    const float2 v = __ldg(rowp + (LIN1 ? b * s1 : row_of(a1 + b, g.first[1], g.rows[1], g.N[1]) * s1));
                    rs = ffma2(w1p[b], v, rs);
                    rd = ffma2(d1p[b], v, rd);
                }
            af = ffma2(make_float2(w0, w0), rs, af);
            ad0 = ffma2(make_float2(d0, d0), rs, ad0);
            ad1 = ffma2(make_float2(w0, w0), rd, ad1);
        }
        float v0x = ad0.x * w2, v0y = ad0.y * w2, v1x = ad1.x * w2, v1y = ad1.y * w2;
        float v2x = af.x * d2, v2y = af.y * d2;
        float sx = af.x * w2, sy = af.y * w2;          // the value s itself (forward with gradient)
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            v0x += __shfl_xor_sync(0xffffffffu, v0x, o);
            v0y += __shfl_xor_sync(0xffffffffu, v0y, o);
            v1x += __shfl_xor_sync(0xffffffffu, v1x, o);
            v1y += __shfl_xor_sync(0xffffffffu, v1y, o);
            v2x += __shfl_xor_sync(0xffffffffu, v2x, o);
            v2y += __shfl_xor_sync(0xffffffffu, v2y, o);
            if (vals) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
            }
        }
        if (live && gl == 0) {
            const int dst = perm[i];
            grad_chain32(g, rho, c0, c1, c2, pt.x, pt.y, pt.z, v0x, v0y, v1x, v1y, v2x, v2y, gout[dst], gxyz + 3 * (int64_t)dst);
            if (vals) vals[dst] = make_double2((double)sx, (double)sy);
        }
    }
}

// Spreading by super-bins.  One CTA per entry of the spreading work list: up to
// spread_chunk(prec) sorted points of one super-bin (C0 x C1 columns x one azimuthal chunk);
// warp w owns tile slab a = w (one grid row on axis 0) and keeps the sums for all T1 rows of
// axis 1 and its 32 azimuthal lanes in registers while it sweeps the entry's points; each tile
// cell is then added to the grid once (atomically: neighbouring tiles, and the other entries of
// a crowded super-bin, overlap it).
// window value for the spreading staging: FP32 takes the branch-free evaluation, FP64 the
// reference form
template <int WIN, typename T>
__device__ __forceinline__ T win_value(T x, T q, T par, T norm) {
    if constexpr (sizeof(T) == 4) return window_pair32<WIN>(x, q, par, norm).x;
    else return window<WIN, T>(x, q, par, norm);
}

template <typename T, int WIN, int Q2MAX, int C1>
struct SpreadSmem {
    static constexpr int PCH = 64;
    static constexpr int PAD = sizeof(T) == 4 ? 4 : 2;         // 128-bit weight loads
    static constexpr int T1MAX = (C1 + Q2MAX - 1 + PAD - 1) / PAD * PAD;
    C2<T> y[PCH];
    T w0[PCH][Q2MAX];
    T w1[PCH][T1MAX];         // axis-1 weights on the tile rows (0 off the point's taps)
    T w2[PCH][32];
    int ta0[PCH];
};

template <typename T, int WIN, int Q2MAX, int C0, int C1>
__global__ void __launch_bounds__(32 * (C0 + Q2MAX - 1)) k_spread_slab(NGeom g, const int4 *__restrict__ work,
                                                                       const int *__restrict__ work_len, const double *__restrict__ u_sorted,
                                                                       const float4 *__restrict__ pts32, const int *__restrict__ perm,
                                                                       const double2 *__restrict__ vals, C2<T> *__restrict__ grid) {
    using S = SpreadSmem<T, WIN, Q2MAX, C1>;
    constexpr int PCH = S::PCH, T1MAX = S::T1MAX;
    constexpr int T1E = C1 + Q2MAX - 1;          // tile rows kept in registers (T1MAX pads the staged rows to 16 B)
    __shared__ __align__(16) S sm;
    const int lane = threadIdx.x & 31, ta = threadIdx.x >> 5;
    const int q = g.q, q2 = 2 * q;
    const T qT = (T)q;
    if ((int)blockIdx.x >= __ldg(work_len)) return;
    const int4 piece = __ldg(work + blockIdx.x);
    const int64_t sb = piece.x;
    const int first = piece.y, last = piece.y + piece.z;
    const int sb1 = (int)(sb % g.nsb1), sb2 = (int)((sb / g.nsb1) % g.nsb2), sb0 = (int)(sb / ((int64_t)g.nsb1 * g.nsb2));
    const int ta_org = sb0 * C0 - q + 1, tb_org = sb1 * C1 - q + 1, cbase = sb2 * g.S2 - q + 1;
    const int T1 = C1 + q2 - 1;
    constexpr int E = Q2MAX + T1MAX + 32 + 1;    // staged values per point
    const T par0 = (T)g.par[0], par1 = (T)g.par[1], par2 = (T)g.par[2];
    const T nrm0 = (T)g.norm[0], nrm1 = (T)g.norm[1], nrm2 = (T)g.norm[2];
    C2<T> acc[T1E];
#pragma unroll
    for (int tb = 0; tb < T1E; ++tb) { acc[tb].x = (T)0; acc[tb].y = (T)0; }
    for (int cs = first; cs < last; cs += PCH) {
        const int np = min(PCH, last - cs);
        __syncthreads();
        for (int t = threadIdx.x; t < np * E; t += blockDim.x) {
            const int p = t / E, e = t % E;
            const int64_t pi = cs + p;
            // cells and fractional coordinates (FP32: from the packed record, no FP64 work)
            int c0, c1, c2;
            T f0, f1, f2;
            if constexpr (sizeof(T) == 4) {
                const float4 pt = pts32[pi];
                unpack_cells(pt.w, c0, c1, c2);
                f0 = pt.x; f1 = pt.y; f2 = pt.z;
            } else {
                const double u0 = u_sorted[3 * pi], u1 = u_sorted[3 * pi + 1], u2 = u_sorted[3 * pi + 2];
                c0 = cell_clamped(u0, g.cmax0);
                c1 = cell_clamped(u1, g.cmax1);
                c2 = min(max((int)floor(u2), 0), g.N[2] - 1);
                f0 = u0 - c0; f1 = u1 - c1; f2 = u2 - c2;
            }
            // window values (FP32: the branch-free, well-conditioned evaluation), one evaluation
            // site for the three axes: tap index rel of this element on its axis
            if (e < Q2MAX + T1MAX + 32) {
                T f, par, nrm, *dst;
                int rel;
                bool ok;
                if (e < Q2MAX) {
                    rel = e; ok = e < q2; f = f0; par = par0; nrm = nrm0; dst = &sm.w0[p][e];
                } else if (e < Q2MAX + T1MAX) {
                    const int tb = e - Q2MAX;
                    rel = tb - (c1 - sb1 * C1);              // tap index of row tb for this point
                    ok = rel >= 0 && rel < q2 && tb < T1; f = f1; par = par1; nrm = nrm1; dst = &sm.w1[p][tb];
                } else {
                    const int L = e - Q2MAX - T1MAX;
                    rel = cbase + L - (c2 - q + 1);
                    ok = rel >= 0 && rel < q2; f = f2; par = par2; nrm = nrm2; dst = &sm.w2[p][L];
                }
                *dst = ok ? win_value<WIN, T>(f + (T)(q - 1 - rel), qT, par, nrm) : (T)0;
            } else {
                const double2 y = vals[perm[pi]];
                sm.y[p].x = (T)y.x;
                sm.y[p].y = (T)y.y;
                sm.ta0[p] = c0 - sb0 * C0;
            }
        }
        __syncthreads();
        // unrolled so that the next points' shared-memory loads overlap this point's FMAs
        // (a CTA has few warps per scheduler to hide that latency with)
#pragma unroll 4
        for (int p = 0; p < np; ++p) {
            const int j = ta - sm.ta0[p];
            if (j < 0 || j >= q2) continue;
            const T wz = sm.w0[p][j] * sm.w2[p][lane];
            C2<T> z;
            z.x = sm.y[p].x * wz;
            z.y = sm.y[p].y * wz;
            if constexpr (sizeof(T) == 4) {
                const float4 *w1v = reinterpret_cast<const float4 *>(&sm.w1[p][0]);
#pragma unroll
                for (int h = 0; h < T1E / 4; ++h) {
                    const float4 w = w1v[h];
                    acc[4 * h] = ffma2(make_float2(w.x, w.x), z, acc[4 * h]);
                    acc[4 * h + 1] = ffma2(make_float2(w.y, w.y), z, acc[4 * h + 1]);
                    acc[4 * h + 2] = ffma2(make_float2(w.z, w.z), z, acc[4 * h + 2]);
                    acc[4 * h + 3] = ffma2(make_float2(w.w, w.w), z, acc[4 * h + 3]);
                }
                constexpr int R = T1E & ~3;              // the last T1E % 4 rows
                if constexpr (T1E % 4 >= 2) {
                    const float2 w = *reinterpret_cast<const float2 *>(&sm.w1[p][R]);
                    acc[R] = ffma2(make_float2(w.x, w.x), z, acc[R]);
                    acc[R + 1] = ffma2(make_float2(w.y, w.y), z, acc[R + 1]);
                }
                if constexpr (T1E % 2) {
                    const float w = sm.w1[p][T1E - 1];
                    acc[T1E - 1] = ffma2(make_float2(w, w), z, acc[T1E - 1]);
                }
            } else {
#pragma unroll
                for (int tb = 0; tb < T1E; ++tb) {
                    const double w = sm.w1[p][tb];
                    acc[tb].x = fma(w, z.x, acc[tb].x);
                    acc[tb].y = fma(w, z.y, acc[tb].y);
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
    for (int tb = 0; tb < T1E; ++tb) {
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

template <typename T, int WIN>
cudaError_t interp_t(sgl_plan *p, double2 *vals) {
    NGeom g = make_geom(p);
    if constexpr (sizeof(T) == 4) {
        const float2 *gridf = (const float2 *)p->b.bufA;
        const int q2 = 2 * p->q;
        const bool lin = p->ax[1].rows < p->ax[1].N;
        const int n2 = p->ax[2].N;
#define SGL_INTERP32(GG, LL, NN) k_interp32<WIN, GG, LL, NN><<<nufft_blocks(p->M, GG), 256, 0, p->stream>>>(g, p->M, p->b.pts32, p->b.perm, gridf, vals)
#define SGL_INTERP32_N(GG)                                                      \
        if (lin && n2 == 128) SGL_INTERP32(GG, true, 128);                      \
        else if (lin && n2 == 256) SGL_INTERP32(GG, true, 256);                 \
        else if (lin && n2 == 512) SGL_INTERP32(GG, true, 512);                 \
        else if (lin) SGL_INTERP32(GG, true, 0);                                \
        else SGL_INTERP32(GG, false, 0);
        if (q2 <= 8) { SGL_INTERP32_N(8) }
        else if (q2 <= 16) { SGL_INTERP32_N(16) }
        else { if (lin) SGL_INTERP32(32, true, 0); else SGL_INTERP32(32, false, 0); }
#undef SGL_INTERP32_N
#undef SGL_INTERP32
        p->launches += 1;
        return cudaGetLastError();
    }
}

template <typename T, int WIN, int Q2MAX, int C0, int C1>
cudaError_t spread_slab_t(sgl_plan *p, const NGeom &g, const double2 *vals) {
    if (g.C0 != C0 || g.C1 != C1) return cudaErrorInvalidConfiguration;
    const int threads = 32 * (C0 + 2 * p->q - 1);
    const int64_t blocks = work_list_cap(p->M, p->bins.nsuper, spread_chunk(p->prec));   // entries past work_len[1] return
    k_spread_slab<T, WIN, Q2MAX, C0, C1><<<(unsigned)blocks, threads, 0, p->stream>>>(
        g, p->b.work[1], p->b.work_len + 1, p->b.u_sorted, p->b.pts32, p->b.perm, vals, (C2<T> *)p->b.bufA);
    p->launches += 1;
    return cudaGetLastError();
}

template <typename T, int WIN>
cudaError_t spread_t(sgl_plan *p, const double2 *vals) {
    NGeom g = make_geom(p);
    if constexpr (sizeof(T) == 4) {
        if (p->q <= 4) return spread_slab_t<T, WIN, 8, 8, 8>(p, g, vals);
        if (p->q <= 8) return spread_slab_t<T, WIN, 16, 8, 8>(p, g, vals);
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
cudaError_t grad_t(sgl_plan *p, const double2 *gout, double *gxyz, double2 *vals) {
    NGeom g = make_geom(p);
    const int q2 = 2 * p->q;
    if constexpr (sizeof(T) == 4) {
        const float2 *gridf = (const float2 *)p->b.bufA;
        const bool lin = p->ax[1].rows < p->ax[1].N;
        const int n2 = p->ax[2].N;
#define SGL_GRAD32(GG, LL, NN) k_grad32<WIN, GG, LL, NN><<<nufft_blocks(p->M, GG), 256, 0, p->stream>>>(g, p->M, p->b.pts32, p->b.perm, p->b.r2max, gridf, gout, gxyz, vals)
#define SGL_GRAD32_N(GG)                                                        \
        if (lin && n2 == 128) SGL_GRAD32(GG, true, 128);                        \
        else if (lin && n2 == 256) SGL_GRAD32(GG, true, 256);                   \
        else if (lin && n2 == 512) SGL_GRAD32(GG, true, 512);                   \
        else if (lin) SGL_GRAD32(GG, true, 0);                                  \
        else SGL_GRAD32(GG, false, 0);
        if (q2 <= 8) { SGL_GRAD32_N(8) }
        else if (q2 <= 16) { SGL_GRAD32_N(16) }
        else { if (lin) SGL_GRAD32(32, true, 0); else SGL_GRAD32(32, false, 0); }
#undef SGL_GRAD32_N
#undef SGL_GRAD32
    }
    p->launches += 1;
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_interp(sgl_plan *p, double2 *vals) {
    if (p->M == 0) return cudaSuccess;
    if (p->tc_interp) return launch_interp_tc(p, vals);
    const bool f32 = p->prec == SGL_FP32_MIXED, kb = p->window == SGL_WIN_KB;
    if (!f32) return launch_interp64(p, vals);
    return kb ? interp_t<float, SGL_WIN_KB>(p, vals) : interp_t<float, SGL_WIN_GAUSS>(p, vals);
}

cudaError_t launch_spread(sgl_plan *p, const double2 *vals) {
    if (p->M == 0) return cudaSuccess;
    if (p->tc_spread) return launch_spread_tc(p, vals);
    const bool f32 = p->prec == SGL_FP32_MIXED, kb = p->window == SGL_WIN_KB;
    if (!f32) return launch_spread64(p, vals);
    return kb ? spread_t<float, SGL_WIN_KB>(p, vals) : spread_t<float, SGL_WIN_GAUSS>(p, vals);
}

cudaError_t launch_grad(sgl_plan *p, const double2 *gout, double *gxyz, double2 *vals) {
    if (p->M == 0) return cudaSuccess;
    if (p->tc_grad) return launch_grad_tc(p, gout, gxyz, vals);
    const bool f32 = p->prec == SGL_FP32_MIXED, kb = p->window == SGL_WIN_KB;
    if (!f32) return launch_grad64(p, gout, gxyz, vals);
    return kb ? grad_t<float, SGL_WIN_KB>(p, gout, gxyz, vals) : grad_t<float, SGL_WIN_GAUSS>(p, gout, gxyz, vals);
}

}  // namespace sgl
