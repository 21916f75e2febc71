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

// FP32 spreading by super-bins, persistent.  One CTA per SM takes entries of the spreading work
// list (at most 1024 sorted points of one super-bin: C0 x C1 = 8 x 8 cell columns x one azimuthal
// chunk) from a device counter until the list is exhausted, and sweeps each entry in chunks of
// PCH points.  Warp ta owns tile slab ta (one grid row of axis 0; the tile has C0 + 2q - 1 of
// them) and keeps the sums of the C1 + Q2M - 1 tile rows of axis 1 and its 32 azimuthal lanes in
// registers.  A point's 2q rows start at its column's row tb0 in [0, C1): rows are swept in
// blocks of four, and the blocks wholly before tb0 = 4 or after the point's last row are left out
// by one warp-uniform branch (every lane serves the same point).  Each tile cell is added to the
// grid once per entry (atomically: neighbouring tiles, and the other entries of a crowded
// super-bin, overlap it).  Point staging (window values) is double-buffered: in one iteration
// every warp stages its share of the next chunk and then sweeps the current one, with one barrier
// per chunk; thread 0 fetches the work one chunk further ahead.  The values come pre-gathered in
// bin order (k_gather_sorted), so staging reads contiguous memory only.
template <int Q2M>
struct RsStage {
    static constexpr int PCH = 64;
    static constexpr int T1P = (8 + Q2M - 1 + 3) / 4 * 4;      // tile rows padded to blocks of four
    float w0[PCH][Q2M];       // axis-0 weights of the point's taps (slab ta0 + j)
    float w1[PCH][T1P];       // axis-1 weights on the tile rows (0 off the point's taps)
    float w2[PCH][32];        // azimuthal weights on the 32 lanes (0 off the point's taps)
    float2 y[PCH];
    int pk[PCH];              // ta0 | tb0 << 8: the point's first slab and first tile row
};

// acc[r] += w1[r] z for the tile rows of blocks B0 .. B1 - 1 (four rows each, rows < T1E)
template <int B0, int B1, int T1E>
__device__ __forceinline__ void rs_rows(float2 (&acc)[T1E], const float *w1, float2 z) {
#pragma unroll
    for (int h = B0; h < B1; ++h) {
        const float4 w = reinterpret_cast<const float4 *>(w1)[h];
        if (4 * h < T1E) acc[4 * h] = ffma2(make_float2(w.x, w.x), z, acc[4 * h]);
        if (4 * h + 1 < T1E) acc[4 * h + 1] = ffma2(make_float2(w.y, w.y), z, acc[4 * h + 1]);
        if (4 * h + 2 < T1E) acc[4 * h + 2] = ffma2(make_float2(w.z, w.z), z, acc[4 * h + 2]);
        if (4 * h + 3 < T1E) acc[4 * h + 3] = ffma2(make_float2(w.w, w.w), z, acc[4 * h + 3]);
    }
}

// the values to spread in bin order, binary32
__global__ void __launch_bounds__(256) k_gather_sorted(int64_t M, const int *__restrict__ perm, const double2 *__restrict__ vals,
                                                       float2 *__restrict__ ys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 y = vals[perm[i]];
        ys[i] = make_float2((float)y.x, (float)y.y);
    }
}

// a chunk's point records and values, copied into shared memory two chunks ahead (cp.async), so
// that staging never waits on DRAM
struct RsRaw {
    float4 pt[64];
    float2 y[64];
};
struct RsDesc { int sb, first, np, flags; };  // flags bit 0: last chunk of its entry; bit 1: no more work

// asynchronous copies of one chunk's records (16 bytes each) and values (8 bytes each) by threads
// 0 .. 2 np - 1, committed as one group
__device__ __forceinline__ void rs_copy_raw(const RsDesc &d, const float4 *__restrict__ pts32, const float2 *__restrict__ ys,
                                            RsRaw &raw) {
    const int t = threadIdx.x;
    if (!(d.flags & 2)) {
        if (t < d.np) {
            const unsigned dst = (unsigned)__cvta_generic_to_shared(&raw.pt[t]);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(pts32 + d.first + t) : "memory");
        } else if (t >= 64 && t < 64 + d.np) {
            const unsigned dst = (unsigned)__cvta_generic_to_shared(&raw.y[t - 64]);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(ys + d.first + (t - 64)) : "memory");
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void rs_copy_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// thread 0 of a spreading CTA: the next chunk of the work list (cursor: super-bin, next point, end,
// done; the entry counter is shared by all CTAs)
__device__ __forceinline__ RsDesc rs_next_desc(int *cursor, const int4 *__restrict__ work, int nwork, int *sched) {
    while (!cursor[3] && cursor[1] >= cursor[2]) {
        const int e = atomicAdd(sched, 1);
        if (e >= nwork) { cursor[3] = 1; break; }
        const int4 piece = __ldg(work + e);
        cursor[0] = piece.x; cursor[1] = piece.y; cursor[2] = piece.y + piece.z;
    }
    RsDesc d{0, 0, 0, 2};
    if (cursor[3]) return d;
    d.sb = cursor[0]; d.first = cursor[1]; d.np = min(64, cursor[2] - cursor[1]);
    cursor[1] += d.np;
    d.flags = (cursor[1] >= cursor[2]) ? 1 : 0;
    return d;
}

// staging of one chunk (all threads of the CTA): window values of the points' taps on the tile
template <int WIN, int Q2M>
__device__ __forceinline__ void rs_stage(const NGeom &g, int sb, int np, const RsRaw &raw, RsStage<Q2M> &b) {
    constexpr int C0 = 8, C1 = 8, T1P = RsStage<Q2M>::T1P;
    constexpr int E = Q2M + T1P + 32 + 1;         // staged items per point
    const int q = g.q, q2 = 2 * q;
    const int sb1 = sb % g.nsb1, sb2 = (sb / g.nsb1) % g.nsb2, sb0 = sb / (g.nsb1 * g.nsb2);
    const int cbase = sb2 * g.S2 - q + 1;
    // the window parameters in registers (the lanes of a warp serve different axes)
    const float par0 = g.parf[0], par1 = g.parf[1], par2 = g.parf[2];
    const float nrm0 = g.normf[0], nrm1 = g.normf[1], nrm2 = g.normf[2];
    // straight-line items, unrolled, so that the window evaluations of several items interleave
#pragma unroll 4
    for (int t = threadIdx.x; t < np * E; t += blockDim.x) {
        const int p = t / E, e = t - p * E;
        const float4 pt = raw.pt[p];
        int c0, c1, c2;
        unpack_cells(pt.w, c0, c1, c2);
        if (e < Q2M + T1P + 32) {
            const int ax = e < Q2M ? 0 : (e < Q2M + T1P ? 1 : 2);
            const int L = e - (ax == 0 ? 0 : (ax == 1 ? Q2M : Q2M + T1P));   // tap (axis 0), tile row (1), lane (2)
            const int rel = ax == 0 ? L : (ax == 1 ? L - (c1 - sb1 * C1) : cbase + L - (c2 - q + 1));
            const float f = ax == 0 ? pt.x : (ax == 1 ? pt.y : pt.z);
            const float par = ax == 0 ? par0 : (ax == 1 ? par1 : par2), nrm = ax == 0 ? nrm0 : (ax == 1 ? nrm1 : nrm2);
            float *dst = ax == 0 ? &b.w0[p][L] : (ax == 1 ? &b.w1[p][L] : &b.w2[p][L]);
            // window_pair32 is zero outside |x| <= q; an off-tap rel gives such an x or is masked
            const float v = window_pair32<WIN>(f + (float)(q - 1 - rel), (float)q, par, nrm).x;
            *dst = (rel >= 0 && rel < q2) ? v : 0.f;
        } else {
            b.y[p] = raw.y[p];
            b.pk[p] = (c0 - sb0 * C0) | ((c1 - sb1 * C1) << 8);
        }
    }
}

// CTAs per SM: two where the smaller tile's registers allow (q <= 4), so that they hide each other's latency
template <int Q2M> constexpr int rs_ctas_per_sm() { return Q2M <= 8 ? 2 : 1; }

template <int WIN, int Q2M>
__global__ void __launch_bounds__(32 * (8 + Q2M - 1), rs_ctas_per_sm<Q2M>()) k_spread_rs(NGeom g, const int4 *__restrict__ work,
                                                                    const int *__restrict__ work_len, const float4 *__restrict__ pts32,
                                                                    const float2 *__restrict__ ys, float2 *__restrict__ grid,
                                                                    int *__restrict__ sched) {
    constexpr int C0 = 8, C1 = 8, T1E = C1 + Q2M - 1, T1P = RsStage<Q2M>::T1P, NB = T1P / 4;
    static_assert(Q2M % 4 == 0 && Q2M <= 16, "taps per axis: a multiple of 4, at most 16");
    static_assert(RsStage<Q2M>::PCH == 64, "chunks of 64 points (two copy threads per point)");
    __shared__ __align__(16) RsStage<Q2M> st[2];
    __shared__ __align__(16) RsRaw raw[2];
    __shared__ RsDesc desc[4];                    // chunks k .. k + 3 (thread 0 fills them three chunks ahead)
    __shared__ int cursor[4];                     // thread 0's place in the work list: super-bin, next point, end, done
    const int lane = threadIdx.x & 31, ta = threadIdx.x >> 5;
    const int nwork = __ldg(work_len + 1);
    if (threadIdx.x == 0) {
        cursor[0] = cursor[1] = cursor[2] = cursor[3] = 0;
        desc[0] = rs_next_desc(cursor, work, nwork, sched);
        desc[1] = rs_next_desc(cursor, work, nwork, sched);
        desc[2] = rs_next_desc(cursor, work, nwork, sched);
    }
    __syncthreads();
    rs_copy_raw(desc[0], pts32, ys, raw[0]);
    rs_copy_raw(desc[1], pts32, ys, raw[1]);
    rs_copy_wait();
    __syncthreads();
    if (!(desc[0].flags & 2)) rs_stage<WIN, Q2M>(g, desc[0].sb, desc[0].np, raw[0], st[0]);
    __syncthreads();
    float2 acc[T1E];
#pragma unroll
    for (int tb = 0; tb < T1E; ++tb) acc[tb] = make_float2(0.f, 0.f);
    for (int k = 0;; ++k) {
        const int cur = k & 3;                    // desc[cur]: the same for every thread, so the loop ends uniformly
        if (desc[cur].flags & 2) break;
        if (threadIdx.x == 0) desc[(k + 3) & 3] = rs_next_desc(cursor, work, nwork, sched);   // slot last read in iteration k - 1
        rs_copy_raw(desc[(k + 2) & 3], pts32, ys, raw[k & 1]);                                // raw[k & 1] was read in iteration k - 1
        if (!(desc[(k + 1) & 3].flags & 2))
            rs_stage<WIN, Q2M>(g, desc[(k + 1) & 3].sb, desc[(k + 1) & 3].np, raw[(k + 1) & 1], st[(k + 1) & 1]);
        const RsStage<Q2M> &b = st[k & 1];
        const int np = desc[cur].np;
        const int q2 = 2 * g.q;
#pragma unroll 4
        for (int p = 0; p < np; ++p) {
            const int pk = b.pk[p];
            const int j = ta - (pk & 255);
            if ((unsigned)j >= (unsigned)q2) continue;
            const float wz = b.w0[p][j] * b.w2[p][lane];
            const float2 y = b.y[p];
            const float2 z = make_float2(y.x * wz, y.y * wz);
            // rows tb0 .. tb0 + q2 - 1 lie in blocks 0 .. NB - 2 when tb0 < 4, in blocks 1 .. NB - 1 otherwise
            if ((pk >> 8) < 4) rs_rows<0, NB - 1, T1E>(acc, &b.w1[p][0], z);
            else rs_rows<1, NB, T1E>(acc, &b.w1[p][0], z);
        }
        if (desc[cur].flags & 1) {                // the entry's last chunk: add the tile to the grid, clear it
            const int sb = desc[cur].sb;
            const int sb1 = sb % g.nsb1, sb2 = (sb / g.nsb1) % g.nsb2, sb0 = sb / (g.nsb1 * g.nsb2);
            const int r0 = row_checked(sb0 * C0 - g.q + 1 + ta, g.first[0], g.rows[0], g.N[0]);
            const int n2 = g.N[2];
            // grid offsets fit in 32 bits (at most 1024^3 / 4 cells per plan)
            const int base = r0 * g.rows[1] * n2 + wrap_index(sb2 * g.S2 - g.q + 1 + lane, n2);
            const bool win1 = g.rows[1] < g.N[1];
            int r1 = sb1 * C1 - g.q + 1 - g.first[1];   // storage row of tile row 0 (windowed axis 1)
            const int nrow = C1 + q2 - 1;
#pragma unroll
            for (int tb = 0; tb < T1E; ++tb, ++r1) {
                const float2 v = acc[tb];
                acc[tb] = make_float2(0.f, 0.f);
                if (r0 < 0 || tb >= nrow || (v.x == 0.f && v.y == 0.f)) continue;
                const int rr = win1 ? r1 : wrap_index(r1 + g.first[1], g.N[1]);
                if (rr >= 0 && rr < g.rows[1]) atomicAdd(grid + (base + rr * n2), v);
            }
        }
        rs_copy_wait();                           // this thread's copies of chunk k + 2
        __syncthreads();
    }
    rs_copy_wait();
}

// FP32 spreading with a sliding azimuthal window (2q <= 16, C0 = C1 = 8).  One CTA per work-list
// entry (at most spread_chunk points of one super-bin).  The entry's points are sorted by their
// first azimuthal tap s (tile column) in shared memory.  Warp w keeps tile slabs w SPW ... w SPW +
// SPW - 1 (LG lanes each: 16, or 8 for 2q <= 8), and lane k of a slab keeps, for every tile row of
// axis 1, the one tile column c = k (mod LG) inside the window [cur, cur + LG).  A point's taps
// [s, s + 2q) lie inside the window once cur = s + 2q - LG; since the points come in s order the
// window only moves forward, and a column that leaves it has received all its taps: it is added
// to the grid then (atomically; neighbouring entries overlap it) and the lane takes column c + LG.
// So every lane of a slab the point reaches does one useful multiply-add per tile row (none on a
// zero weight when 2q = LG), and each tile cell goes to the grid once per entry.  A point's rows of
// axis 1 start at tb0 in [0, 8): a switch on tb0 picks the statically indexed registers.
template <int Q2M>
struct CwGeom {
    static constexpr int LG = Q2M <= 8 ? 8 : 16;       // lanes per slab (a power of two)
    static constexpr int SPW = 32 / LG;                // slabs per warp
    static constexpr int SLABS = 8 + Q2M - 1;          // tile slabs (axis 0)
    static constexpr int NW = (SLABS + SPW - 1) / SPW;  // warps
    static constexpr int SLABP = NW * SPW;             // slabs with a lane group (the last may be padding)
    static constexpr int T1E = 8 + Q2M - 1;            // tile rows (axis 1)
    static constexpr int PCH = 64;                     // points per staged chunk
    static constexpr int PMAX = SGL_SPREAD_CHUNK32;    // points per work-list entry
};

// A staged chunk: the point's value times its 2q axis-0 window values, its 2q window values on
// axes 1 and 2 (zero past 2q), and where its taps start.
template <int Q2M>
struct CwStage {
    float2 yw0[64][Q2M];      // y psi_0(tap j)
    float w1[64][Q2M];
    float w2[64][Q2M];
    int meta[64];             // first slab ta0 | first tile row tb0 << 8 | first tile column s << 16
};

template <int Q2M>
struct CwSmem {
    float4 pt[CwGeom<Q2M>::PMAX];
    float2 y[CwGeom<Q2M>::PMAX];
    short order[CwGeom<Q2M>::PMAX];   // sorted position -> index in the entry
    int hist[32], cursor[32];
    CwStage<Q2M> st[2];
};

// acc[T0 + i] += w1[i] z, i < Q2M (T0 + i < 8 + Q2M - 1: always a tile row)
template <int T0, int Q2M, int T1E>
__device__ __forceinline__ void cw_rows(float2 (&acc)[T1E], const float *w1, float2 z) {
#pragma unroll
    for (int h = 0; h < Q2M / 4; ++h) {
        const float4 w = reinterpret_cast<const float4 *>(w1)[h];
        acc[T0 + 4 * h] = ffma2(make_float2(w.x, w.x), z, acc[T0 + 4 * h]);
        acc[T0 + 4 * h + 1] = ffma2(make_float2(w.y, w.y), z, acc[T0 + 4 * h + 1]);
        acc[T0 + 4 * h + 2] = ffma2(make_float2(w.z, w.z), z, acc[T0 + 4 * h + 2]);
        acc[T0 + 4 * h + 3] = ffma2(make_float2(w.w, w.w), z, acc[T0 + 4 * h + 3]);
    }
}

template <int WIN, int Q2M, int N2T>
__global__ void __launch_bounds__(32 * CwGeom<Q2M>::NW, 2) k_spread_cw(NGeom g, const int4 *__restrict__ work,
                                                                       const int *__restrict__ work_len,
                                                                       const float4 *__restrict__ pts32,
                                                                       const float2 *__restrict__ ys, float2 *__restrict__ grid) {
    using G = CwGeom<Q2M>;
    constexpr int LG = G::LG, SPW = G::SPW, T1E = G::T1E, PCH = G::PCH;
    static_assert(Q2M % 4 == 0 && Q2M <= 16 && Q2M <= LG && G::NW <= 20, "taps per axis: a multiple of 4, at most one slab's lanes");
    extern __shared__ __align__(16) unsigned char cw_smem[];
    CwSmem<Q2M> &sm = *reinterpret_cast<CwSmem<Q2M> *>(cw_smem);
    if (blockIdx.x >= __ldg(work_len + 1)) return;
    const int4 piece = __ldg(work + blockIdx.x);
    const int sb = piece.x, first = piece.y, np = piece.z;
    const int q = g.q, q2 = 2 * q, S2 = g.S2;
    const int sb1 = sb % g.nsb1, sb2 = (sb / g.nsb1) % g.nsb2, sb0 = sb / (g.nsb1 * g.nsb2);
    const int tid = threadIdx.x, NT = blockDim.x;

    // the entry's records and values, and a counting sort by the first azimuthal tap s = c2 - sb2 S2
    if (tid < 32) sm.hist[tid] = 0;
    __syncthreads();
    for (int i = tid; i < np; i += NT) {
        const float4 pt = pts32[first + i];
        sm.pt[i] = pt;
        sm.y[i] = ys[first + i];
        int c0, c1, c2;
        unpack_cells(pt.w, c0, c1, c2);
        atomicAdd(&sm.hist[c2 - sb2 * S2], 1);
    }
    __syncthreads();
    if (tid < 32) {                               // exclusive scan of the S2 <= 32 counts
        const int v = sm.hist[tid];
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, x, o);
            if (tid >= o) x += t;
        }
        sm.cursor[tid] = x - v;
    }
    __syncthreads();
    for (int i = tid; i < np; i += NT) {
        int c0, c1, c2;
        unpack_cells(sm.pt[i].w, c0, c1, c2);
        sm.order[atomicAdd(&sm.cursor[c2 - sb2 * S2], 1)] = (short)i;
    }
    __syncthreads();

    // window values of a chunk of sorted points: one (point, axis) unit per thread, the warps
    // taken edge first (0, NW - 1, 1, NW - 2, ...) since the warps of the outer slabs reach the
    // fewest points in the sweep below (a chunk's 3 x 64 units leave the middle warps out)
    const float par0 = g.parf[0], par1 = g.parf[1], par2 = g.parf[2];
    const float nrm0 = g.normf[0], nrm1 = g.normf[1], nrm2 = g.normf[2];
    const int nwarps = NT >> 5, wq = tid >> 5;
    const int srank = (wq < (nwarps + 1) / 2 ? 2 * wq : 2 * (nwarps - 1 - wq) + 1) * 32 + (tid & 31);
    auto stage = [&](int ch, CwStage<Q2M> &b) {
        const int n = min(PCH, np - ch * PCH);
        for (int unit = srank; unit < 3 * n; unit += NT) {
            const int p = unit / 3, ax = unit - 3 * p;
            const int i = sm.order[ch * PCH + p];
            const float4 pt = sm.pt[i];
            const float f = ax == 0 ? pt.x : (ax == 1 ? pt.y : pt.z);
            const float par = ax == 0 ? par0 : (ax == 1 ? par1 : par2), nrm = ax == 0 ? nrm0 : (ax == 1 ? nrm1 : nrm2);
            float2 y = make_float2(0.f, 0.f);
            if (ax == 0) {
                y = sm.y[i];
                int c0, c1, c2;
                unpack_cells(pt.w, c0, c1, c2);
                b.meta[p] = (c0 - sb0 * 8) | ((c1 - sb1 * 8) << 8) | ((c2 - sb2 * S2) << 16);
            }
            float *dst = ax == 1 ? b.w1[p] : b.w2[p];
#pragma unroll 4
            for (int j = 0; j < Q2M; ++j) {
                // tap j sits at grid index c - q + 1 + j: x = (u - c) + q - 1 - j
                const float v = window_pair32<WIN>(f + (float)(q - 1 - j), (float)q, par, nrm).x;
                const float w = j < q2 ? v : 0.f;
                if (ax == 0) b.yw0[p][j] = make_float2(y.x * w, y.y * w);
                else dst[j] = w;
            }
        }
    };

    const int warp = tid >> 5, lane = tid & 31, slot = lane & (LG - 1);
    const int ta = warp * SPW + lane / LG;        // this lane's tile slab
    float2 acc[T1E];
#pragma unroll
    for (int tb = 0; tb < T1E; ++tb) acc[tb] = make_float2(0.f, 0.f);
    // grid coordinates of this lane's slab and of tile row 0 (axis 1 windowed: rows stored in order)
    const int r0 = ta < G::SLABS ? row_checked(sb0 * 8 - q + 1 + ta, g.first[0], g.rows[0], g.N[0]) : -1;
    const int n2 = N2T ? N2T : g.N[2], tile_w = S2 + q2 - 1, rows1 = g.rows[1];
    const int r1 = sb1 * 8 - q + 1 - g.first[1];
    // add column col of the lane's registers to the grid and clear them (constant row stride when
    // N2T is set, so that the 2q + 7 atomic adds share one address register)
    // tile rows stored on axis 1, as a bit mask (T1E <= 23)
    const unsigned rows_ok = (r0 < 0) ? 0u : (((1u << min(T1E, max(rows1 - r1, 0))) - 1u) & ~((1u << min(T1E, max(-r1, 0))) - 1u));
    auto flush = [&](int col) {
        const unsigned ok = col < tile_w ? rows_ok : 0u;
        float2 *gp = grid + ((int64_t)max(r0, 0) * rows1 + r1) * n2 + wrap_index(sb2 * S2 - q + 1 + col, n2);
#pragma unroll
        for (int tb = 0; tb < T1E; ++tb) {
            const float2 v = acc[tb];
            acc[tb] = make_float2(0.f, 0.f);
            if (((ok >> tb) & 1u) && (v.x != 0.f || v.y != 0.f)) atomicAdd(gp + tb * n2, v);
        }
    };

    const int nch = (np + PCH - 1) / PCH;
    stage(0, sm.st[0]);
    __syncthreads();
    int cur = 0;                                  // window start (tile column), the same in every warp
    int col = slot;                               // this lane's tile column: cur + ((slot - cur) mod LG)
    for (int ch = 0; ch < nch; ++ch) {
        if (ch + 1 < nch) stage(ch + 1, sm.st[(ch + 1) & 1]);
        const CwStage<Q2M> &b = sm.st[ch & 1];
        const int n = min(PCH, np - ch * PCH);
#pragma unroll 2
        for (int p = 0; p < n; ++p) {
            const int meta = b.meta[p];
            const int ta0 = meta & 255, tb0 = (meta >> 8) & 255, s = meta >> 16;
            if (s + q2 - LG > cur) {              // move the window: columns below s + 2q - LG are complete
                const int nc = s + q2 - LG;
                if (col < nc) flush(col);
                cur = nc;
                col = cur + ((slot - cur) & (LG - 1));
            }
            if (warp * SPW + SPW - 1 < ta0 || warp * SPW > ta0 + q2 - 1) continue;   // no slab of this warp
            const int j0 = ta - ta0, j2 = col - s;
            const float2 yw = (unsigned)j0 < (unsigned)q2 ? b.yw0[p][j0] : make_float2(0.f, 0.f);
            const float a2 = (unsigned)j2 < (unsigned)q2 ? b.w2[p][j2] : 0.f;
            const float2 z = make_float2(yw.x * a2, yw.y * a2);
            const float *w1 = b.w1[p];
            switch (tb0) {
                case 0: cw_rows<0, Q2M, T1E>(acc, w1, z); break;
                case 1: cw_rows<1, Q2M, T1E>(acc, w1, z); break;
                case 2: cw_rows<2, Q2M, T1E>(acc, w1, z); break;
                case 3: cw_rows<3, Q2M, T1E>(acc, w1, z); break;
                case 4: cw_rows<4, Q2M, T1E>(acc, w1, z); break;
                case 5: cw_rows<5, Q2M, T1E>(acc, w1, z); break;
                case 6: cw_rows<6, Q2M, T1E>(acc, w1, z); break;
                default: cw_rows<7, Q2M, T1E>(acc, w1, z); break;
            }
        }
        __syncthreads();
    }
    flush(col);
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

template <int WIN, int Q2M>
cudaError_t spread_rs_t(sgl_plan *p, const NGeom &g, const double2 *vals) {
    if (g.C0 != 8 || g.C1 != 8 || 2 * p->q > Q2M || g.S2 > 33 - 2 * p->q) return cudaErrorInvalidConfiguration;
    k_gather_sorted<<<nufft_blocks(p->M, 1), 256, 0, p->stream>>>(p->M, p->b.perm, vals, p->b.ys32);
    cudaError_t e = cudaMemsetAsync(p->b.sched, 0, sizeof(int), p->stream);
    if (e != cudaSuccess) return e;
    const int threads = 32 * (8 + 2 * p->q - 1);
    k_spread_rs<WIN, Q2M><<<p->num_sms * rs_ctas_per_sm<Q2M>(), threads, 0, p->stream>>>(g, p->b.work[1], p->b.work_len, p->b.pts32, p->b.ys32,
                                                               (float2 *)p->b.bufA, p->b.sched);
    p->launches += 2;
    return cudaGetLastError();
}

template <int WIN, int Q2M>
cudaError_t spread_cw_t(sgl_plan *p, const NGeom &g, const double2 *vals) {
    if (g.C0 != 8 || g.C1 != 8 || 2 * p->q > Q2M || g.S2 > 32 || p->ax[1].rows == p->ax[1].N) return cudaErrorInvalidConfiguration;
    k_gather_sorted<<<nufft_blocks(p->M, 1), 256, 0, p->stream>>>(p->M, p->b.perm, vals, p->b.ys32);
    const int n2 = p->ax[2].N;
    auto kern = n2 == 128 ? k_spread_cw<WIN, Q2M, 128>
                          : (n2 == 256 ? k_spread_cw<WIN, Q2M, 256> : (n2 == 512 ? k_spread_cw<WIN, Q2M, 512> : k_spread_cw<WIN, Q2M, 0>));
    const int smem = (int)sizeof(CwSmem<Q2M>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = work_list_cap(p->M, p->bins.nsuper, spread_chunk(p->prec));   // entries past work_len[1] return
    kern<<<(unsigned)blocks, 32 * CwGeom<Q2M>::NW, smem, p->stream>>>(g, p->b.work[1], p->b.work_len, p->b.pts32, p->b.ys32,
                                                                      (float2 *)p->b.bufA);
    p->launches += 2;
    return cudaGetLastError();
}

template <typename T, int WIN>
cudaError_t spread_t(sgl_plan *p, const double2 *vals) {
    NGeom g = make_geom(p);
    if constexpr (sizeof(T) == 4) {
        // the sliding-window kernel wherever axis 1 is windowed (measured at B = 64, 10^6 points:
        // 1.49 -> 1.30 ms at q = 8, 1.26 -> 1.01 at q = 6, 0.80 -> 0.58 at q = 4); the
        // register-tile kernel for the small grids whose axis 1 is periodic
        if (g.C0 == 8 && g.C1 == 8 && g.S2 <= 32 && p->ax[1].rows < p->ax[1].N) {
            if (p->q <= 4) return spread_cw_t<WIN, 8>(p, g, vals);
            if (p->q <= 6) return spread_cw_t<WIN, 12>(p, g, vals);
            if (p->q <= 8) return spread_cw_t<WIN, 16>(p, g, vals);
        }
        if (p->q <= 4) return spread_rs_t<WIN, 8>(p, g, vals);
        if (p->q <= 6) return spread_rs_t<WIN, 12>(p, g, vals);
        if (p->q <= 8) return spread_rs_t<WIN, 16>(p, g, vals);
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
