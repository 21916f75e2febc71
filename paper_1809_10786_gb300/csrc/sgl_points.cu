// sgl_points.cu -- point preprocessing for the NFSGLFT (Sect. 6 and 7 of the paper):
//   rho = max_i |x_i| (Sect. 7, choice of rho), the transformed points
//   xtilde_i = [arccos gamma(r_i), theta_i, phi_i] with gamma(r) = (2r - rho)/rho
//   (Sect. 6, eq. of the transformed points), their oversampled-grid coordinates
//   u_d = N_d xtilde_d / (2 pi), and a counting sort of the points by spatial bin.
#include "sgl_internal.cuh"

namespace sgl {
namespace {

constexpr int kThreads = 256;

// rho^2 = max |x|^2 over the finite points; with `copy` non-NULL the points are also copied there
__global__ void k_max_radius(const double *__restrict__ xyz, int64_t M,
                             unsigned long long *__restrict__ r2max, int *__restrict__ flags,
                             double *__restrict__ copy) {
    double best = 0.0;
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        if (copy) { copy[3 * i] = x; copy[3 * i + 1] = y; copy[3 * i + 2] = z; }
        if (!(isfinite(x) && isfinite(y) && isfinite(z))) { bad = true; continue; }
        best = fmax(best, x * x + y * y + z * z);
    }
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    __shared__ double wmax[kThreads / 32];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = best;
    if (bad) atomicOr(flags, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, wmax[w]);
        // non-negative doubles order like their bit patterns
        atomicMax(r2max, (unsigned long long)__double_as_longlong(m));
    }
}

struct PointGeom {
    int N[3];
    int S2, C0, C1;     // azimuthal chunk, columns per super-bin
    int nsb1, nsb2;     // super-bins along axes 1 and 2
    int cmax0, cmax1;   // largest cell index on axes 0 and 1 (N/2)
};

__device__ __forceinline__ double rho_of(const unsigned long long *r2max) {
    double rho = sqrt(__longlong_as_double((long long)*r2max)) * (1.0 + 0x1p-20);
    return rho > 0.0 ? rho : 1.0;
}

// atan2(a, b) in binary64 (a published method: argument reduction by a table of angles plus a
// Taylor series).  A binary32 first guess g (on the operands scaled by a power of two, so neither
// overflows nor underflows in binary32) picks th_k = k pi / kRotK nearest to it; with c = cos th_k,
// s = sin th_k from the table, tan(theta - th_k) = (a c - b s) / (b c + a s), and
// theta = th_k + atan(t), |t| <= tan(pi / 2 kRotK + 1e-6) < 8e-4, by the series t - t^3/3 + t^5/5 -
// t^7/7 (the next term is below 1e-27).  atan2(0, 0) = 0.
__device__ __forceinline__ double atan2_tab(double a, double b, const double2 *__restrict__ rot) {
    const double m = fmax(fabs(a), fabs(b));
    if (!(m > 0.0)) return 0.0;
    const int e = max(min((int)((__double_as_longlong(m) >> 52) & 0x7ff) - 1023, 1000), -1000);   // m = 1.f 2^e
    const double sc = __longlong_as_double((long long)(1023 - e) << 52);                         // 2^-e (exact)
    const float g = atan2f((float)(a * sc), (float)(b * sc));
    const int k = __float2int_rn(g * ((float)kRotK / 3.14159265f));
    const double2 cs = __ldg(rot + (k + kRotK));
    const double num = fma(a, cs.x, -b * cs.y);                // r sin(theta - th_k)
    const double den = fma(b, cs.x, a * cs.y);                 // r cos(theta - th_k) > 0
    const double t = num / den, t2 = t * t;
    const double at = fma(t * t2, fma(t2, fma(t2, -1.0 / 7.0, 1.0 / 5.0), -1.0 / 3.0), t);
    return fma((double)k, kPi / kRotK, at);
}

// grid coordinates u_d = N_d t_d / (2 pi) of one point.  t0 = arccos(gamma), gamma = (2r - rho)/rho,
// is atan2(sqrt(1 - gamma^2), gamma) with the common factor 2/rho left out:
// atan2(2 sqrt(r (rho - r)), 2r - rho) (r <= rho: rho carries the 2^-20 margin).
__device__ __forceinline__ void grid_coords(double x, double y, double z, double rho, const PointGeom &g,
                                            const double2 *__restrict__ rot, double &u0, double &u1, double &u2) {
    const double rxy2 = fma(x, x, y * y);
    const double rxy = sqrt(rxy2), r = sqrt(fma(z, z, rxy2));
    const double t0 = atan2_tab(2.0 * sqrt(fmax(r * (rho - r), 0.0)), 2.0 * r - rho, rot);
    const double t1 = atan2_tab(rxy, z, rot);                  // [0, pi]
    double t2 = atan2_tab(y, x, rot);                          // [-pi, pi]
    if (t2 < 0.0) t2 += 2.0 * kPi;
    const double inv2pi = 1.0 / (2.0 * kPi);
    u0 = g.N[0] * t0 * inv2pi;
    u1 = g.N[1] * t1 * inv2pi;
    u2 = g.N[2] * t2 * inv2pi;
    if (u2 >= g.N[2]) u2 -= g.N[2];
    if (u2 < 0.0) u2 = 0.0;
}

// bin key: super-bin (axis 0, azimuthal chunk, axis 1) first, then the column inside it, so the
// points of one column are contiguous and the columns of one super-bin are contiguous
__device__ __forceinline__ int bin_of_coords(double u0, double u1, double u2, const PointGeom &g) {
    const int c0 = min(max((int)floor(u0), 0), g.cmax0);
    const int c1 = min(max((int)floor(u1), 0), g.cmax1);
    const int c2 = min(max((int)floor(u2), 0), g.N[2] - 1);
    const int sb = ((c0 / g.C0) * g.nsb2 + c2 / g.S2) * g.nsb1 + c1 / g.C1;
    return (sb * g.C0 + c0 % g.C0) * g.C1 + c1 % g.C1;
}

__global__ void k_transform_points(const double *__restrict__ xyz, int64_t M, const unsigned long long *__restrict__ r2max,
                                   PointGeom g, const double2 *__restrict__ rot, double *__restrict__ u_tmp, int *__restrict__ bin_of,
                                   int *__restrict__ rank_of, int *__restrict__ bin_count) {
    const double rho = rho_of(r2max);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        if (!(isfinite(x) && isfinite(y) && isfinite(z))) { x = 0.0; y = 0.0; z = 0.0; }
        double u0, u1, u2;
        grid_coords(x, y, z, rho, g, rot, u0, u1, u2);
        u_tmp[3 * i] = u0; u_tmp[3 * i + 1] = u1; u_tmp[3 * i + 2] = u2;
        const int b = bin_of_coords(u0, u1, u2, g);
        bin_of[i] = b;
        rank_of[i] = atomicAdd(&bin_count[b], 1);
    }
}

// exclusive scan, three phases: per-block totals, scan of totals, final offsets
constexpr int kScanItems = 8;
constexpr int kScanBlock = kThreads * kScanItems;

__global__ void k_scan_block_totals(const int *__restrict__ cnt, int64_t n, int *__restrict__ totals) {
    __shared__ int ws[kThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    int s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kThreads + threadIdx.x;
        if (i < n) s += cnt[i];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += ws[w];
        totals[blockIdx.x] = t;
    }
}

// single block: exclusive scan of nblk totals in place (nblk small)
__global__ void k_scan_totals(int *__restrict__ totals, int nblk) {
    __shared__ int buf[kThreads];
    int carry = 0;
    for (int start = 0; start < nblk; start += kThreads) {
        int i = start + threadIdx.x;
        int v = (i < nblk) ? totals[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < kThreads; o <<= 1) {
            int t = (threadIdx.x >= o) ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nblk) totals[i] = carry + buf[threadIdx.x] - v;
        __syncthreads();
        carry += buf[kThreads - 1];
        __syncthreads();
    }
}

__global__ void k_scan_final(const int *__restrict__ cnt, int64_t n, const int *__restrict__ totals, int *__restrict__ off) {
    __shared__ int buf[kScanBlock];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    for (int k = 0; k < kScanItems; ++k) {
        int j = k * kThreads + threadIdx.x;
        buf[j] = (base + j < n) ? cnt[base + j] : 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {      // serial scan inside the block keeps this simple; n/kScanBlock blocks run in parallel
        int acc = totals[blockIdx.x];
        for (int j = 0; j < kScanBlock; ++j) { int v = buf[j]; buf[j] = acc; acc += v; }
    }
    __syncthreads();
    for (int k = 0; k < kScanItems; ++k) {
        int j = k * kThreads + threadIdx.x;
        if (base + j < n) off[base + j] = buf[j];
    }
}

__global__ void k_scatter_points(int64_t M, const double *__restrict__ u_tmp, const int *__restrict__ bin_of,
                                 const int *__restrict__ rank_of, const int *__restrict__ off, PointGeom g,
                                 double *__restrict__ u_sorted, float4 *__restrict__ pts32, int *__restrict__ perm) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const int pos = off[bin_of[i]] + rank_of[i];
        const double u0 = u_tmp[3 * i], u1 = u_tmp[3 * i + 1], u2 = u_tmp[3 * i + 2];
        u_sorted[3 * pos] = u0;
        u_sorted[3 * pos + 1] = u1;
        u_sorted[3 * pos + 2] = u2;
        // cells as in the bin key; fractional parts relative to them (exact in binary64, rounded once)
        const int c0 = min(max((int)floor(u0), 0), g.cmax0);
        const int c1 = min(max((int)floor(u1), 0), g.cmax1);
        const int c2 = min(max((int)floor(u2), 0), g.N[2] - 1);
        pts32[pos] = make_float4((float)(u0 - c0), (float)(u1 - c1), (float)(u2 - c2), __int_as_float(c0 | (c1 << 10) | (c2 << 20)));
        perm[pos] = (int)i;
    }
}

// Work lists (one thread per super-bin): counts of full pieces and of remainders, laid out as
// [full 0][rem 0][full 1][rem 1], nsuper each, so that one exclusive scan of the whole array
// orders every list's full pieces before its remainders.
__global__ void k_piece_count(const int *__restrict__ bin_off, int64_t nsuper, int bins_per_super, int64_t M, int P0,
                              int P1, int *__restrict__ cnt) {
    for (int64_t sb = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sb < nsuper; sb += (int64_t)gridDim.x * blockDim.x) {
        const int f = bin_off[sb * bins_per_super];
        const int l = (sb + 1 < nsuper) ? bin_off[(sb + 1) * bins_per_super] : (int)M;
        const int n = l - f;
        cnt[sb] = n / P0;
        cnt[nsuper + sb] = (n % P0) ? 1 : 0;
        cnt[2 * nsuper + sb] = n / P1;
        cnt[3 * nsuper + sb] = (n % P1) ? 1 : 0;
    }
}

__global__ void k_piece_fill(const int *__restrict__ bin_off, int64_t nsuper, int bins_per_super, int64_t M, int P0, int P1,
                             const int *__restrict__ cnt, const int *__restrict__ off, int4 *__restrict__ list0,
                             int4 *__restrict__ list1, int *__restrict__ len) {
    const int len0 = off[2 * nsuper];                 // entries of list 0 (they precede list 1 in the scan)
    for (int64_t sb = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sb < nsuper; sb += (int64_t)gridDim.x * blockDim.x) {
        const int f = bin_off[sb * bins_per_super];
        const int l = (sb + 1 < nsuper) ? bin_off[(sb + 1) * bins_per_super] : (int)M;
        for (int k = 0; k < 2; ++k) {
            const int P = k ? P1 : P0;
            int4 *list = k ? list1 : list0;
            const int base = k ? len0 : 0;
            const int nfull = cnt[2 * k * nsuper + sb];
            const int o = off[2 * k * nsuper + sb] - base;
            for (int j = 0; j < nfull; ++j) list[o + j] = make_int4((int)sb, f + j * P, P, 0);
            if (cnt[(2 * k + 1) * nsuper + sb]) {
                const int r = off[(2 * k + 1) * nsuper + sb] - base;
                list[r] = make_int4((int)sb, f + nfull * P, l - f - nfull * P, 0);
            }
        }
        if (sb == 0) {
            len[0] = len0;
            len[1] = off[4 * nsuper - 1] + cnt[4 * nsuper - 1] - len0;
        }
    }
}

void scan(const int *cnt, int64_t n, int *tmp, int *off, cudaStream_t s) {
    const int nblk = (int)((n + kScanBlock - 1) / kScanBlock);
    k_scan_block_totals<<<nblk, kThreads, 0, s>>>(cnt, n, tmp);
    k_scan_totals<<<1, kThreads, 0, s>>>(tmp, nblk);
    k_scan_final<<<nblk, kThreads, 0, s>>>(cnt, n, tmp, off);
}

int grid_blocks(int64_t work, int threads) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (int)b;
}

}  // namespace

cudaError_t launch_points_rho(sgl_plan *p, const double *xyz, int64_t M, double *copy) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(p->b.r2max, 0, sizeof(unsigned long long), p->stream)) != cudaSuccess) return e;
    if (M > 0) {
        k_max_radius<<<grid_blocks(M, kThreads), kThreads, 0, p->stream>>>(xyz, M, p->b.r2max, p->b.dev_flags, copy);
        p->launches += 1;
    }
    return cudaGetLastError();
}

cudaError_t launch_points_bins(sgl_plan *p, const double *xyz, int64_t M, cudaStream_t s) {
    Buffers &b = p->b;
    cudaError_t e;
    if ((e = cudaMemsetAsync(b.bin_count, 0, sizeof(int) * p->nbins, s)) != cudaSuccess) return e;
    PointGeom g;
    for (int d = 0; d < 3; ++d) g.N[d] = p->ax[d].N;
    g.S2 = p->bins.S2;
    g.C0 = p->bins.C0;
    g.C1 = p->bins.C1;
    g.nsb1 = p->bins.nsb[1];
    g.nsb2 = p->bins.nsb[2];
    g.cmax0 = p->ax[0].N / 2;
    g.cmax1 = p->ax[1].N / 2;
    if (M > 0) {
        k_transform_points<<<grid_blocks(M, kThreads), kThreads, 0, s>>>(xyz, M, b.r2max, g, b.rot, b.u_tmp, b.bin_of, b.rank_of, b.bin_count);
        scan(b.bin_count, p->nbins, b.scan_tmp, b.bin_off, s);
        k_scatter_points<<<grid_blocks(M, kThreads), kThreads, 0, s>>>(M, b.u_tmp, b.bin_of, b.rank_of, b.bin_off, g, b.u_sorted,
                                                                       b.pts32, b.perm);
        const int64_t ns = p->bins.nsuper;
        const int bps = p->bins.C0 * p->bins.C1, P1 = spread_chunk(p->prec);
        k_piece_count<<<grid_blocks(ns, kThreads), kThreads, 0, s>>>(b.bin_off, ns, bps, M, kTcPass, P1, b.piece_cnt);
        scan(b.piece_cnt, 4 * ns, b.scan_tmp, b.piece_off, s);
        k_piece_fill<<<grid_blocks(ns, kThreads), kThreads, 0, s>>>(b.bin_off, ns, bps, M, kTcPass, P1, b.piece_cnt, b.piece_off,
                                                                    b.work[0], b.work[1], b.work_len);
        p->launches += 10;
    } else if ((e = cudaMemsetAsync(b.work_len, 0, 2 * sizeof(int), s)) != cudaSuccess) {
        return e;
    }
    return cudaGetLastError();
}

cudaError_t launch_max_radius_raw(cudaStream_t s, const double *xyz, int64_t M, unsigned long long *r2max, int *flags) {
    if (M > 0) k_max_radius<<<grid_blocks(M, kThreads), kThreads, 0, s>>>(xyz, M, r2max, flags, nullptr);
    return cudaGetLastError();
}

}  // namespace sgl
