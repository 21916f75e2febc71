// sgl_points.cu -- point preprocessing for the NFSGLFT (Sect. 6 and 7 of the paper):
//   rho = max_i |x_i| (Sect. 7, choice of rho), the transformed points
//   xtilde_i = [arccos gamma(r_i), theta_i, phi_i] with gamma(r) = (2r - rho)/rho
//   (Sect. 6, eq. of the transformed points), their oversampled-grid coordinates
//   u_d = N_d xtilde_d / (2 pi), and a counting sort of the points by spatial bin.
#include "sgl_dfl.cuh"
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
    float2 scale[3];    // N_d / (2 pi) as a double-float (h, l)
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

// ---- the same angles in double-float arithmetic (FP32-mixed plans): every operation on the
// FP32 pipe, relative rounding about 1e-13, far below the binary32 offsets the kernels read.

// finiteness from the exponent field (integer operations only)
__device__ __forceinline__ bool finite_bits(double x) {
    return ((((unsigned long long)__double_as_longlong(x)) >> 52) & 0x7ff) != 0x7ff;
}

// unbiased exponent field of a double (-1023 for zero and subnormals)
__device__ __forceinline__ int exponent_of(double x) {
    return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff) - 1023;
}

// atan2(a, b) in double-float: the table step of atan2_tab with (cos, sin) of k pi / kRotK as
// double-float pairs; atan(t) = t - t^3/3 (the next term is below 7e-17).  atan2(0, 0) = 0.
__device__ __forceinline__ dfl atan2_df(dfl a, dfl b, const float4 *__restrict__ rotf) {
    if (a.h == 0.f && b.h == 0.f) return dfl(0.f, 0.f);
    const float g = atan2f(a.h, b.h);
    const int k = __float2int_rn(g * ((float)kRotK / 3.14159265f));
    const float4 cs = __ldg(rotf + (k + kRotK));             // (cos h, cos l, sin h, sin l)
    const dfl c(cs.x, cs.y), sn(cs.z, cs.w);
    const dfl num = a * c - b * sn;
    const dfl den = b * c + a * sn;
    const dfl t = df_div(num, den);
    const float t3 = __fmul_rn(__fmul_rn(t.h, t.h), t.h) * (-1.f / 3.f);
    constexpr dfl step(kPi / kRotK);                          // pi / kRotK
    const float kf = (float)k;                                // |k| <= kRotK: exact
    const float p = __fmul_rn(kf, step.h);
    const dfl th = fast_two_sum(p, fmaf(kf, step.l, fmaf(kf, step.h, -p)));
    return th + (t + dfl(t3));
}

// cell c = floor(u) (clamped to [0, cmax]) and the binary32 offset u - c of a double-float u
__device__ __forceinline__ int cell_df(dfl u, int cmax, float &frac) {
    float c = floorf(u.h);
    if (u.h == c && u.l < 0.f) c -= 1.f;
    const int ci = min(max((int)c, 0), cmax);
    frac = __fadd_rn(__fsub_rn(u.h, (float)ci), u.l);
    return ci;
}

// bin key: super-bin (axis 0, azimuthal chunk, axis 1) first, then the column inside it, so the
// points of one column are contiguous and the columns of one super-bin are contiguous
__device__ __forceinline__ int bin_of_cells(int c0, int c1, int c2, const PointGeom &g) {
    const int sb = ((c0 / g.C0) * g.nsb2 + c2 / g.S2) * g.nsb1 + c1 / g.C1;
    return (sb * g.C0 + c0 % g.C0) * g.C1 + c1 % g.C1;
}

__device__ __forceinline__ float4 record(float f0, float f1, float f2, int c0, int c1, int c2) {
    return make_float4(f0, f1, f2, __int_as_float(c0 | (c1 << 10) | (c2 << 20)));
}

// Transform, cells, binary32 record and bin key of each point in input order, and its rank in
// its bin (atomic counter).  DF: double-float angles; u_tmp (binary64 coordinates) written when
// non-NULL.
template <bool DF>
__global__ void __launch_bounds__(256) k_transform_points(const double *__restrict__ xyz, int64_t M,
                                                          const unsigned long long *__restrict__ r2max, PointGeom g,
                                                          const double2 *__restrict__ rot, const float4 *__restrict__ rotf,
                                                          double *__restrict__ u_tmp, float4 *__restrict__ rec_tmp,
                                                          int *__restrict__ bin_of, int *__restrict__ rank_of,
                                                          int *__restrict__ bin_count) {
    // rho (binary64 plans) or rho 2^-Erho as a double-float (rho = sqrt(max r^2)(1 + 2^-20))
    double rho = 1.0;
    dfl rho_s(1.f, 0.f);
    int Erho = 0;
    if constexpr (DF) {
        const double r2 = __longlong_as_double((long long)*r2max);
        if (r2 > 0.0) {
            const int E2 = exponent_of(r2) & ~1;                  // even: sqrt(r2 2^-E2) = sqrt(r2) 2^-E2/2
            const dfl s = df_sqrt(df_split_bits(r2, E2));           // in [1, 2)
            rho_s = s + df_mul(s, 0x1p-20f);
            Erho = E2 / 2;
        }
    } else {
        rho = rho_of(r2max);
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        if (!(finite_bits(x) && finite_bits(y) && finite_bits(z))) { x = 0.0; y = 0.0; z = 0.0; }
        int c0, c1, c2;
        float f0, f1, f2;
        if constexpr (DF) {
            const int E = max(max(exponent_of(x), exponent_of(y)), exponent_of(z));
            const dfl xs = df_split_bits(x, E), ys = df_split_bits(y, E), zs = df_split_bits(z, E);
            const dfl rxy2 = xs * xs + ys * ys;
            const dfl rxy = df_sqrt(rxy2), r = df_sqrt(rxy2 + zs * zs);      // times 2^-E
            // t0 on the common scale 2^-Erho (E <= Erho: rho >= r >= every coordinate)
            const int d = E - Erho;
            const dfl rr = d >= -100 ? df_scale2(r, d) : dfl(0.f, 0.f);
            const dfl t0 = atan2_df(df_mul(df_sqrt(rr * (rho_s - rr)), 2.f), df_mul(rr, 2.f) - rho_s, rotf);
            const dfl t1 = atan2_df(rxy, zs, rotf);
            dfl t2 = atan2_df(ys, xs, rotf);
            constexpr dfl two_pi(2.0 * kPi);
            if (t2.h < 0.f) t2 = t2 + two_pi;
            const dfl u0 = t0 * dfl(g.scale[0].x, g.scale[0].y);
            const dfl u1 = t1 * dfl(g.scale[1].x, g.scale[1].y);
            dfl u2 = t2 * dfl(g.scale[2].x, g.scale[2].y);
            const float n2 = (float)g.N[2];
            if (u2.h > n2 || (u2.h == n2 && u2.l >= 0.f)) u2 = u2 - dfl(n2);
            if (u2.h < 0.f) u2 = dfl(0.f, 0.f);
            c0 = cell_df(u0, g.cmax0, f0);
            c1 = cell_df(u1, g.cmax1, f1);
            c2 = cell_df(u2, g.N[2] - 1, f2);
            if (u_tmp) {
                u_tmp[3 * i] = df_to_double(u0); u_tmp[3 * i + 1] = df_to_double(u1); u_tmp[3 * i + 2] = df_to_double(u2);
            }
        } else {
            double u0, u1, u2;
            grid_coords(x, y, z, rho, g, rot, u0, u1, u2);
            u_tmp[3 * i] = u0; u_tmp[3 * i + 1] = u1; u_tmp[3 * i + 2] = u2;
            // cells as in the bin key; offsets relative to them (exact in binary64, rounded once)
            c0 = min(max((int)floor(u0), 0), g.cmax0);
            c1 = min(max((int)floor(u1), 0), g.cmax1);
            c2 = min(max((int)floor(u2), 0), g.N[2] - 1);
            f0 = (float)(u0 - c0); f1 = (float)(u1 - c1); f2 = (float)(u2 - c2);
        }
        rec_tmp[i] = record(f0, f1, f2, c0, c1, c2);
        const int b = bin_of_cells(c0, c1, c2, g);
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

// offsets of one block of kScanBlock counts: each thread scans its kScanItems consecutive counts,
// the threads' totals are scanned by warp shuffles and the warps' totals by warp 0
__global__ void __launch_bounds__(kThreads) k_scan_final(const int *__restrict__ cnt, int64_t n, const int *__restrict__ totals,
                                                         int *__restrict__ off) {
    __shared__ __align__(16) int buf[kScanBlock];
    __shared__ int wsum[kThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    for (int k = 0; k < kScanItems; ++k) {
        const int j = k * kThreads + threadIdx.x;
        buf[j] = (base + j < n) ? cnt[base + j] : 0;
    }
    __syncthreads();
    int v[kScanItems];
    const int4 *b4 = reinterpret_cast<const int4 *>(buf + kScanItems * threadIdx.x);
    static_assert(kScanItems == 8, "two int4 per thread");
    const int4 lo = b4[0], hi = b4[1];
    v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w; v[4] = hi.x; v[5] = hi.y; v[6] = hi.z; v[7] = hi.w;
    int t = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) { const int c = v[k]; v[k] = t; t += c; }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = t;                                        // inclusive scan of the threads' totals in the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = lane < kThreads / 32 ? wsum[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < kThreads / 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += u;
        }
        if (lane < kThreads / 32) wsum[lane] = wi - w;  // exclusive
    }
    __syncthreads();
    const int add = totals[blockIdx.x] + wsum[warp] + inc - t;
    int4 *o4 = reinterpret_cast<int4 *>(buf + kScanItems * threadIdx.x);
    o4[0] = make_int4(v[0] + add, v[1] + add, v[2] + add, v[3] + add);
    o4[1] = make_int4(v[4] + add, v[5] + add, v[6] + add, v[7] + add);
    __syncthreads();
    for (int k = 0; k < kScanItems; ++k) {
        const int j = k * kThreads + threadIdx.x;
        if (base + j < n) off[base + j] = buf[j];
    }
}

// points in bin order: record, permutation and (when u_tmp is non-NULL) binary64 coordinates
__global__ void __launch_bounds__(256) k_scatter_points(int64_t M, const float4 *__restrict__ rec_tmp, const double *__restrict__ u_tmp,
                                                        const int *__restrict__ bin_of, const int *__restrict__ rank_of,
                                                        const int *__restrict__ off, double *__restrict__ u_sorted,
                                                        float4 *__restrict__ pts32, int *__restrict__ perm) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
        const int pos = off[bin_of[i]] + rank_of[i];
        pts32[pos] = rec_tmp[i];
        perm[pos] = (int)i;
        if (u_tmp) {
            u_sorted[3 * pos] = u_tmp[3 * i];
            u_sorted[3 * pos + 1] = u_tmp[3 * i + 1];
            u_sorted[3 * pos + 2] = u_tmp[3 * i + 2];
        }
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

int grid_blocks(int64_t work, int threads, int64_t cap = 152 * 32) {
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

}  // namespace

cudaError_t launch_points_rho(sgl_plan *p, const double *xyz, int64_t M, double *copy) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(p->b.r2max, 0, sizeof(unsigned long long), p->stream)) != cudaSuccess) return e;
    if (M > 0) {
        // a few CTAs per SM: one atomicMax per CTA on the same word
        k_max_radius<<<grid_blocks(M, kThreads, 8 * (int64_t)p->num_sms), kThreads, 0, p->stream>>>(xyz, M, p->b.r2max,
                                                                                                    p->b.dev_flags, copy);
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
    for (int d = 0; d < 3; ++d) {
        const dfl sc(p->ax[d].N / (2.0 * kPi));
        g.scale[d] = make_float2(sc.h, sc.l);
    }
    if (M > 0) {
        // FP32-mixed plans: double-float angles; binary64 coordinates only for the generic
        // spreading kernel (cutoffs above 8); binary64 plans: binary64 throughout
        const bool df = p->prec == SGL_FP32_MIXED;
        double *u_tmp = (!df || p->q > 8) ? b.u_tmp : nullptr;
        const int blocks = grid_blocks(M, kThreads);
        if (df)
            k_transform_points<true><<<blocks, kThreads, 0, s>>>(xyz, M, b.r2max, g, b.rot, b.rotf, u_tmp, b.rec_tmp, b.bin_of,
                                                                 b.rank_of, b.bin_count);
        else
            k_transform_points<false><<<blocks, kThreads, 0, s>>>(xyz, M, b.r2max, g, b.rot, b.rotf, u_tmp, b.rec_tmp, b.bin_of,
                                                                  b.rank_of, b.bin_count);
        scan(b.bin_count, p->nbins, b.scan_tmp, b.bin_off, s);
        k_scatter_points<<<blocks, kThreads, 0, s>>>(M, b.rec_tmp, u_tmp, b.bin_of, b.rank_of, b.bin_off, b.u_sorted, b.pts32,
                                                     b.perm);
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
    if (M > 0) k_max_radius<<<grid_blocks(M, kThreads, 8 * 152), kThreads, 0, s>>>(xyz, M, r2max, flags, nullptr);
    return cudaGetLastError();
}

}  // namespace sgl
