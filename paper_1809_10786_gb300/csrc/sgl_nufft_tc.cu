// sgl_nufft_tc.cu -- windowed interpolation (NFFT step 3, Sect. 2) and its window-derivative
// form (the point gradient) on the 5th-generation tensor cores, FP32-mixed plans.
//
// For one super-bin (C0 x C1 cell columns x S2 azimuthal cells) and one chunk of up to 128
// of its points, the sum over the taps factors slab by slab.  For the tile slab ta (one grid
// row on axis 0) let G_ta[tb][c] be the grid values on the T1 = C1 + 2q - 1 tile rows of axis
// 1 and the 32 azimuthal lanes c of the super-bin.  Then
//
//     D_ta[p][tb] = sum_c  w2_p[c] G_ta[tb][c]                (a 128 x 48 x 32 product)
//     s_p         = sum_ta w0_p[ta] sum_tb w1_p[tb] D_ta[p][tb]
//
// with w_d the point's window weights on the tile (zero off its 2q taps).  The product runs
// as tcgen05.mma kind::tf32 with an FP32 accumulator in tensor memory; both operands are
// split into a TF32 head and a TF32 remainder (x = hi + lo), and hi*hi + hi*lo + lo*hi keeps
// the product at FP32 accuracy.  The gradient adds a second product with the derivative
// weights w2' and contracts D_ta with w0', w1' as well.
//
// Data: the forward FFT's grid is re-laid out once per call into four FP32 planes
// (Re hi, Im hi, Re lo, Im lo) with a wrapped halo on the azimuthal axis, so that every
// G_ta tile is one TMA box (32 lanes x T1 rows, 128-byte swizzle) per plane.
//
// CTA = one super-bin, 6 warps: warp 0 issues the TMA loads into a ring of NS stages, warp 1
// owns tensor memory and issues the MMAs, warps 2-5 (one thread per point, the thread's TMEM
// lane = its point) write the w2 operand and reduce D_ta from TMEM (two accumulator buffers,
// so the MMAs of slab ta+1 overlap the reduction of slab ta).  Every mbarrier wait is bounded
// (about a second); on expiry the CTA sets bit 1 of the plan's device flags, drains what it
// has in flight and returns.
#include "sgl_nufft_common.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

namespace sgl {
namespace {

constexpr int kC0 = 8, kC1 = 8;       // cell columns per super-bin (FP32 plans)
constexpr int kLanes = 32;            // azimuthal lanes = MMA K
constexpr int kPM = 128;              // points per chunk = MMA M
constexpr int kNB = 48;               // MMA N: rows 0..T1-1 Re, rows 24..24+T1-1 Im
constexpr int kImRow = 24;
constexpr int kT1Max = 23;            // C1 + 2q - 1 for q <= 8
constexpr int kNS = 3;                // TMA stages
constexpr int kTileA = kPM * 128;     // bytes of one A operand (128 rows x 32 FP32)
constexpr int kTileB = kNB * 128;     // bytes of one B operand (48 rows x 32 FP32)
constexpr int kThreads = 192;
constexpr long long kWaitCycles = 1ll << 31;   // ~1 s at 2 GHz

// instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major, M = 128, N = 48
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kNB >> 3) << 17) | ((uint32_t)(kPM >> 4) << 24);

template <bool GRAD>
struct TcSmem {
    alignas(1024) unsigned char a[GRAD ? 4 : 2][kTileA];     // w2 hi, lo (+ w2' hi, lo)
    alignas(1024) unsigned char b[kNS][2][kTileB];            // per stage: grid tile hi, lo
    uint64_t full[kNS], empty[kNS], tfull[2], tempty[2], afull, done;
    uint32_t tmem_base;
    int abort;
};

struct TcArgs {
    const int *bin_off;
    int64_t M, nsuper;
    const float4 *pts;
    const int *perm;
    double2 *vals;                          // interpolation output
    const unsigned long long *r2max;        // gradient: rho
    const double2 *gout;
    double *gxyz;
    int *dev_flags;
    int T1;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory operand descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
           ((uint64_t)2 << 61);
}

// byte offset of element (row, k) in a K-major 128-byte-swizzled tile of 32 FP32 per row
__device__ __forceinline__ uint32_t sw128_off(int row, int k4) { return (uint32_t)(row * 128 + ((k4 ^ (row & 7)) << 4)); }

__device__ __forceinline__ float tf32_head(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
    return ok != 0;
}

// wait for the phase of the given parity to complete; false after about a second
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    if (mbar_try(mbar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(mbar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(mbar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(mbar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, uint32_t mbar, int x, int y, int z, int w) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], [%2];"
        :: "r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(mbar), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(dtmem), "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar) : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
                   "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// write 32 weights (one operand row) as TF32 head and remainder, 128-byte swizzled
__device__ __forceinline__ void store_split_row(unsigned char *hi, unsigned char *lo, int row, const float *w) {
#pragma unroll
    for (int k4 = 0; k4 < 8; ++k4) {
        float4 h, l;
        h.x = tf32_head(w[4 * k4]);     l.x = tf32_head(w[4 * k4] - h.x);
        h.y = tf32_head(w[4 * k4 + 1]); l.y = tf32_head(w[4 * k4 + 1] - h.y);
        h.z = tf32_head(w[4 * k4 + 2]); l.z = tf32_head(w[4 * k4 + 2] - h.z);
        h.w = tf32_head(w[4 * k4 + 3]); l.w = tf32_head(w[4 * k4 + 3] - h.w);
        const uint32_t o = sw128_off(row, k4);
        *reinterpret_cast<float4 *>(hi + o) = h;
        *reinterpret_cast<float4 *>(lo + o) = l;
    }
}

template <int WIN, bool GRAD>
__global__ void __launch_bounds__(kThreads, GRAD ? 2 : 3)
k_nufft_tc(const __grid_constant__ CUtensorMap tmap, NGeom g, TcArgs args) {
    using S = TcSmem<GRAD>;
    constexpr uint32_t kBufCols = GRAD ? 128 : 64;     // TMEM columns per accumulator buffer
    constexpr uint32_t kAllocCols = 2 * kBufCols;
    extern __shared__ unsigned char smem_raw[];
    S &sm = *reinterpret_cast<S *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);

    const int64_t sb = blockIdx.x;
    if (sb >= args.nsuper) return;
    const int first = args.bin_off[sb * kC0 * kC1];
    const int last = (sb + 1 < args.nsuper) ? args.bin_off[(sb + 1) * kC0 * kC1] : (int)args.M;
    const int np = last - first;
    if (np <= 0) return;
    const int sb1 = (int)(sb % g.nsb1), sb2 = (int)((sb / g.nsb1) % g.nsb2), sb0 = (int)(sb / ((int64_t)g.nsb1 * g.nsb2));
    const int q = g.q, q2 = 2 * q;
    const int T0 = kC0 + q2 - 1, T1 = args.T1;
    const int nchunks = (np + kPM - 1) / kPM;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // ---- setup: barriers (thread 0), tensor memory (warp 1)
    if (threadIdx.x == 0) {
        for (int i = 0; i < kNS; ++i) { mbar_init(smem_addr(&sm.full[i]), 1); mbar_init(smem_addr(&sm.empty[i]), 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(smem_addr(&sm.tfull[i]), 1); mbar_init(smem_addr(&sm.tempty[i]), 4); }
        mbar_init(smem_addr(&sm.afull), 4);
        mbar_init(smem_addr(&sm.done), 1);
        sm.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // grid tiles: rows the TMA boxes do not cover (T1 <= row < 24, 24 + T1 <= row) stay zero
    for (int i = threadIdx.x; i < (int)(sizeof(sm.b) / 16); i += kThreads)
        reinterpret_cast<float4 *>(&sm.b[0][0][0])[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_addr(&sm.tmem_base)),
                     "r"(kAllocCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    volatile int *abort_flag = &sm.abort;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            const int x = sb2 * g.S2;                 // halo-shifted azimuthal coordinate of lane 0
            const int y = sb1 * kC1 + 1;              // stored row of tile row 0 on axis 1 (first = -q)
            const int z0 = sb0 * kC0 + 1;             // stored row of slab 0 on axis 0
            const uint32_t tx = 4u * (uint32_t)T1 * 128u;
            int s = 0;
            for (int ch = 0; ch < nchunks && !*abort_flag; ++ch)
                for (int ta = 0; ta < T0; ++ta, ++s) {
                    const int st = s % kNS;
                    if (s >= kNS && !mbar_wait(smem_addr(&sm.empty[st]), ((s / kNS) + 1) & 1)) {
                        *abort_flag = 1;
                        break;
                    }
                    if (*abort_flag) break;
                    const uint32_t fb = smem_addr(&sm.full[st]);
                    mbar_expect_tx(fb, tx);
                    const uint32_t hi = smem_addr(sm.b[st][0]), lo = smem_addr(sm.b[st][1]);
                    tma_load_4d(hi, &tmap, fb, x, y, z0 + ta, 0);
                    tma_load_4d(hi + kImRow * 128, &tmap, fb, x, y, z0 + ta, 1);
                    tma_load_4d(lo, &tmap, fb, x, y, z0 + ta, 2);
                    tma_load_4d(lo + kImRow * 128, &tmap, fb, x, y, z0 + ta, 3);
                }
            // drain: the last loads issued into each stage have landed before the CTA may exit
            for (int k = (s > kNS ? s - kNS : 0); k < s; ++k) mbar_wait(smem_addr(&sm.full[k % kNS]), (k / kNS) & 1);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            int s = 0;
            bool ok = true;
            for (int ch = 0; ch < nchunks && ok; ++ch) {
                ok = mbar_wait(smem_addr(&sm.afull), ch & 1) && !*abort_flag;
                tc_fence_after();
                for (int ta = 0; ta < T0 && ok; ++ta, ++s) {
                    const int st = s % kNS, buf = s & 1;
                    ok = mbar_wait(smem_addr(&sm.full[st]), (s / kNS) & 1);
                    if (ok && s >= 2) ok = mbar_wait(smem_addr(&sm.tempty[buf]), ((s >> 1) + 1) & 1);
                    if (!ok || *abort_flag) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t d = tmem + buf * kBufCols;
                    const uint32_t ahi = smem_addr(sm.a[0]), alo = smem_addr(sm.a[1]);
                    const uint32_t bhi = smem_addr(sm.b[st][0]), blo = smem_addr(sm.b[st][1]);
#pragma unroll
                    for (int ks = 0; ks < kLanes / 8; ++ks) {
                        const uint32_t ko = ks * 32;          // 8 TF32 of K per instruction
                        mma_tf32(d, sw128_desc(ahi + ko), sw128_desc(bhi + ko), ks > 0);
                        mma_tf32(d, sw128_desc(ahi + ko), sw128_desc(blo + ko), 1);
                        mma_tf32(d, sw128_desc(alo + ko), sw128_desc(bhi + ko), 1);
                    }
                    if constexpr (GRAD) {
                        const uint32_t dhi = smem_addr(sm.a[2]), dlo = smem_addr(sm.a[3]);
#pragma unroll
                        for (int ks = 0; ks < kLanes / 8; ++ks) {
                            const uint32_t ko = ks * 32;
                            mma_tf32(d + 64, sw128_desc(dhi + ko), sw128_desc(bhi + ko), ks > 0);
                            mma_tf32(d + 64, sw128_desc(dhi + ko), sw128_desc(blo + ko), 1);
                            mma_tf32(d + 64, sw128_desc(dlo + ko), sw128_desc(bhi + ko), 1);
                        }
                    }
                    mma_commit(smem_addr(&sm.empty[st]));
                    mma_commit(smem_addr(&sm.tfull[buf]));
                }
            }
            if (!ok) *abort_flag = 1;
            // every MMA issued above has completed before tensor memory is released
            mma_commit(smem_addr(&sm.done));
            mbar_wait(smem_addr(&sm.done), 0);
        }
    } else {
        // ---------------- point threads: operand rows and the reduction of D_ta
        const int quad = warp & 3;                   // TMEM lanes 32 quad .. 32 quad + 31
        const int p = quad * 32 + lane;              // MMA row = point within the chunk
        const float qf = (float)q;
        const float par0 = (float)g.par[0], par1 = (float)g.par[1], par2 = (float)g.par[2];
        const float nrm0 = (float)g.norm[0], nrm1 = (float)g.norm[1], nrm2 = (float)g.norm[2];
        const int cbase = sb2 * g.S2 - tc_halo(q);   // grid index of lane 0
        float rho = 0.f;
        if constexpr (GRAD) rho = rho_from_r2max(args.r2max);
        int s = 0;
        bool ok = true;
        for (int ch = 0; ch < nchunks && ok; ++ch) {
            const int idx = ch * kPM + p;
            const bool live = idx < np;
            const int64_t i = first + (live ? idx : 0);
            const float4 pt = args.pts[i];
            int c0, c1, c2;
            unpack_cells(pt.w, c0, c1, c2);
            const int d0 = c0 - sb0 * kC0, d1 = c1 - sb1 * kC1;
            // axis 2: lane k holds grid index cbase + k; tap rel = k - (c2 - q + 1 - cbase)
            {
                const int k0 = c2 - q + 1 - cbase;
                float w[kLanes];
#pragma unroll
                for (int k = 0; k < kLanes; ++k) {
                    const int rel = k - k0;
                    w[k] = (live && rel >= 0 && rel < q2) ? window<WIN, float>(pt.z + (float)(q - 1 - rel), qf, par2, nrm2) : 0.f;
                }
                store_split_row(sm.a[0], sm.a[1], p, w);
                if constexpr (GRAD) {
#pragma unroll
                    for (int k = 0; k < kLanes; ++k) {
                        const int rel = k - k0;
                        w[k] = (live && rel >= 0 && rel < q2) ? window_deriv<WIN, float>(pt.z + (float)(q - 1 - rel), qf, par2, nrm2)
                                                              : 0.f;
                    }
                    store_split_row(sm.a[2], sm.a[3], p, w);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&sm.afull));
            // axis 1: weights on the tile rows (zero off the point's taps)
            float w1[kT1Max], e1[GRAD ? kT1Max : 1];
#pragma unroll
            for (int tb = 0; tb < kT1Max; ++tb) {
                const int rel = tb - d1;
                const bool on = live && rel >= 0 && rel < q2;
                w1[tb] = on ? window<WIN, float>(pt.y + (float)(q - 1 - rel), qf, par1, nrm1) : 0.f;
                if constexpr (GRAD) e1[tb] = on ? window_deriv<WIN, float>(pt.y + (float)(q - 1 - rel), qf, par1, nrm1) : 0.f;
            }
            float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f, cx = 0.f, cy = 0.f;
            for (int ta = 0; ta < T0; ++ta, ++s) {
                const int buf = s & 1;
                ok = __all_sync(0xffffffffu, mbar_wait(smem_addr(&sm.tfull[buf]), (s >> 1) & 1) && !*abort_flag);
                if (!ok) break;
                tc_fence_after();
                const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + buf * kBufCols;
                float D[kNB];
                tmem_ld16(taddr, D);
                tmem_ld16(taddr + 16, D + 16);
                tmem_ld16(taddr + 32, D + 32);
                float E[GRAD ? kNB : 1];
                if constexpr (GRAD) {
                    tmem_ld16(taddr + 64, E);
                    tmem_ld16(taddr + 80, E + 16);
                    tmem_ld16(taddr + 96, E + 32);
                }
                tmem_wait_ld();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_addr(&sm.tempty[buf]));
                const int j = ta - d0;
                if (j < 0 || j >= q2) continue;
                const float xo = pt.x + (float)(q - 1 - j);
                const float w0 = window<WIN, float>(xo, qf, par0, nrm0);
                float rx = 0.f, ry = 0.f;
#pragma unroll
                for (int tb = 0; tb < kT1Max; ++tb) {
                    rx = fmaf(w1[tb], D[tb], rx);
                    ry = fmaf(w1[tb], D[kImRow + tb], ry);
                }
                if constexpr (GRAD) {
                    const float e0 = window_deriv<WIN, float>(xo, qf, par0, nrm0);
                    float sx = 0.f, sy = 0.f, tx = 0.f, ty = 0.f;
#pragma unroll
                    for (int tb = 0; tb < kT1Max; ++tb) {
                        sx = fmaf(e1[tb], D[tb], sx);
                        sy = fmaf(e1[tb], D[kImRow + tb], sy);
                        tx = fmaf(w1[tb], E[tb], tx);
                        ty = fmaf(w1[tb], E[kImRow + tb], ty);
                    }
                    ax = fmaf(e0, rx, ax); ay = fmaf(e0, ry, ay);     // ds/du0
                    bx = fmaf(w0, sx, bx); by = fmaf(w0, sy, by);     // ds/du1
                    cx = fmaf(w0, tx, cx); cy = fmaf(w0, ty, cy);     // ds/du2
                } else {
                    ax = fmaf(w0, rx, ax);
                    ay = fmaf(w0, ry, ay);
                }
            }
            if (!ok) break;
            if (live) {
                const int dst = args.perm[i];
                if constexpr (GRAD)
                    grad_chain32(g, rho, c0, c1, c2, pt.x, pt.y, pt.z, ax, ay, bx, by, cx, cy, args.gout[dst],
                                 args.gxyz + 3 * (int64_t)dst);
                else
                    args.vals[dst] = make_double2((double)ax, (double)ay);
            }
        }
        if (!ok) *abort_flag = 1;
    }
    tc_fence_before();
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) atomicOr(args.dev_flags, 2);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kAllocCols));
    }
}

// grid[r0][r1][c] (FP32 complex) -> planes[4][r0][r1][pitch]: Re hi, Im hi, Re lo, Im lo at halo
// column e = c + L (every e in [0, pitch) holds grid column (e - L) mod N2)
__global__ void k_split_planes(const float2 *__restrict__ grid, float *__restrict__ planes, int64_t lines, int N2, int pitch,
                               int L) {
    const int64_t n = lines * pitch;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t line = t / pitch;
        const int e = (int)(t - line * pitch);
        const int c = wrap_index(e - L, N2);
        const float2 v = grid[line * N2 + c];
        const float hx = tf32_head(v.x), hy = tf32_head(v.y);
        planes[t] = hx;
        planes[n + t] = hy;
        planes[2 * n + t] = tf32_head(v.x - hx);
        planes[3 * n + t] = tf32_head(v.y - hy);
    }
}

}  // namespace

// ---------------------------------------------------------------- host side
bool tc_eligible(const sgl_plan *p) {
    return p->prec == SGL_FP32_MIXED && !(p->flags & SGL_FLAG_SIMT) && p->q <= 8 && p->ax[0].windowed && p->ax[1].windowed &&
           p->bins.C0 == kC0 && p->bins.C1 == kC1 && p->bins.S2 % 4 == 0 && p->bins.S2 + tc_halo(p->q) + p->q <= kLanes;
}

// Which operations take the tensor-core kernels.  Measured on GB300 (B = 64, 10^6 points,
// q = 8): interpolation 1.15 ms against 1.53 ms on the CUDA cores, gradient 2.74 against
// 2.65 ms; at q = 4 the CUDA-core kernels are three times faster (their work falls as q^3,
// the slab products' does not).  So by default: interpolation for q >= 7, gradient never.
void tc_choose(sgl_plan *p) {
    const bool force = (p->flags & SGL_FLAG_TC) != 0;
    p->tc_interp = p->tc && (force || p->q >= 7);
    p->tc_grad = p->tc && force;
}

int64_t tc_plane_floats(const sgl_plan *p) {
    return 4 * (int64_t)p->ax[0].rows * p->ax[1].rows * tc_pitch(p->ax[2].N);
}

namespace {
std::mutex g_encode_mu;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
}  // namespace

// tensor map over the planes: dims (pitch, rows1, rows0, 4 planes), box 32 lanes x T1 rows
cudaError_t tc_make_tensor_map(sgl_plan *p) {
    {
        std::lock_guard<std::mutex> lock(g_encode_mu);
        if (!g_encode) {
            void *fn = nullptr;
            cudaDriverEntryPointQueryResult qr;
            cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
            if (e != cudaSuccess) return e;
            if (qr != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        }
    }
    const int pitch = tc_pitch(p->ax[2].N);
    const cuuint64_t dims[4] = {(cuuint64_t)pitch, (cuuint64_t)p->ax[1].rows, (cuuint64_t)p->ax[0].rows, 4};
    const cuuint64_t strides[3] = {(cuuint64_t)pitch * 4, (cuuint64_t)pitch * 4 * p->ax[1].rows,
                                   (cuuint64_t)pitch * 4 * p->ax[1].rows * p->ax[0].rows};
    const cuuint32_t box[4] = {(cuuint32_t)kLanes, (cuuint32_t)(kC1 + 2 * p->q - 1), 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    static_assert(sizeof(CUtensorMap) <= sizeof(p->tc_map), "tensor map storage");
    CUtensorMap *map = reinterpret_cast<CUtensorMap *>(p->tc_map);
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p->b.planes, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

namespace {

cudaError_t split_planes(sgl_plan *p) {
    const int64_t lines = (int64_t)p->ax[0].rows * p->ax[1].rows;
    const int pitch = tc_pitch(p->ax[2].N);
    const int64_t n = lines * pitch;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_split_planes<<<(unsigned)blocks, 256, 0, p->stream>>>((const float2 *)p->b.bufA, p->b.planes, lines, p->ax[2].N, pitch,
                                                           tc_halo(p->q));
    p->launches += 1;
    return cudaGetLastError();
}

template <int WIN, bool GRAD>
cudaError_t run_tc(sgl_plan *p, TcArgs a) {
    cudaError_t e = split_planes(p);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(TcSmem<GRAD>) + 1024;
    auto kern = k_nufft_tc<WIN, GRAD>;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
    const CUtensorMap *map = reinterpret_cast<const CUtensorMap *>(p->tc_map);
    kern<<<(unsigned)p->bins.nsuper, kThreads, smem, p->stream>>>(*map, make_geom(p), a);
    p->launches += 1;
    return cudaGetLastError();
}

TcArgs base_args(const sgl_plan *p) {
    TcArgs a{};
    a.bin_off = p->b.bin_off;
    a.M = p->M;
    a.nsuper = p->bins.nsuper;
    a.pts = p->b.pts32;
    a.perm = p->b.perm;
    a.r2max = p->b.r2max;
    a.dev_flags = p->b.dev_flags;
    a.T1 = kC1 + 2 * p->q - 1;
    return a;
}

}  // namespace

cudaError_t launch_interp_tc(sgl_plan *p, double2 *vals) {
    TcArgs a = base_args(p);
    a.vals = vals;
    return p->window == SGL_WIN_KB ? run_tc<SGL_WIN_KB, false>(p, a) : run_tc<SGL_WIN_GAUSS, false>(p, a);
}

cudaError_t launch_grad_tc(sgl_plan *p, const double2 *gout, double *gxyz) {
    TcArgs a = base_args(p);
    a.gout = gout;
    a.gxyz = gxyz;
    return p->window == SGL_WIN_KB ? run_tc<SGL_WIN_KB, true>(p, a) : run_tc<SGL_WIN_GAUSS, true>(p, a);
}

}  // namespace sgl
