// sgl_nufft_tc.cu -- windowed interpolation (NFFT step 3, Sect. 2) and its window-derivative
// form (the point gradient) on the 5th-generation tensor cores, FP32-mixed plans.
//
// For one super-bin (C0 x C1 cell columns x S2 azimuthal cells) and a chunk of up to 128 of
// its points, the sum over the taps factors slab by slab.  For the tile slab ta (one grid row
// on axis 0) let G_ta[tb][c] be the grid values on the T1 = C1 + 2q - 1 tile rows of axis 1
// and the 32 azimuthal lanes c of the super-bin.  Then
//
//     D_ta[p][tb] = sum_c  w2_p[c] G_ta[tb][c]                (M = 128 points, K = 32 lanes)
//     s_p         = sum_ta w0_p[ta] sum_tb w1_p[tb] D_ta[p][tb]
//
// with w_d the point's window weights on the tile (zero off its 2q taps).  G slabs go through
// the tensor core together (N = 2 G TB1 columns: Re and Im of G slabs of TB1 >= T1 rows), as
// tcgen05.mma kind::tf32 with an FP32 accumulator in tensor memory.  Both operands are split
// into a TF32 head and a TF32 remainder (x = hi + lo), and hi*hi + hi*lo + lo*hi keeps the
// product at FP32 accuracy.  The gradient adds a second product with the derivative weights
// w2' and contracts D_ta with w0', w1' as well.
//
// Data: the forward FFT's last pass writes the grid as two FP32 planes (Re, Im) with a wrapped
// halo on the azimuthal axis, so that the tiles of G slabs are one TMA box (32 lanes x TB1 rows
// x G slabs, 128-byte swizzle) per plane; the split into head and remainder happens on chip.
//
// One persistent CTA per SM walks its super-bins in 128-point passes.  Warp 0 issues the TMA
// loads into a ring of tile stages, warps 2-3 split each landed tile in place, warp 1 owns
// tensor memory and issues the MMAs (operand w2 from TMEM, tile from shared memory), four prep
// warps write each pass's operands into TMEM and its axis-0/1 window tables into shared memory
// (one pass ahead), and eight reduction warps (two per lane quadrant, alternate slabs) contract the
// accumulators with the tables -- one thread per point, the thread's TMEM lane is its point.  Every mbarrier wait is bounded (about a second); on
// expiry the CTA sets bit 1 of the plan's device flags, drains what it has in flight and
// returns.
#include "sgl_nufft_common.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

namespace sgl {
namespace {

constexpr int kC0 = 8, kC1 = 8;       // cell columns per super-bin (FP32 plans)
constexpr int kLanes = 32;            // azimuthal lanes = MMA K
constexpr int kPM = 128;              // points per pass = MMA M
constexpr int kTB1Max = 24;           // tile rows per slab, T1 = C1 + 2q - 1 rounded up to 8 (q <= 8)
constexpr long long kWaitCycles = 1ll << 31;   // ~1 s at 2 GHz

// instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t tf32_idesc(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kPM >> 4) << 24);
}

// Pipeline shape.  Interpolation: groups of 4 slabs (N <= 192), two operand buffers (w2).
// Gradient: groups of 2 slabs with two accumulators each (D and D', N <= 96), one operand buffer
// (w2, w2').  Accumulators double-buffered across groups.  TMEM: 512 columns, one CTA per SM.
// Eight reduction warps: two per TMEM lane quadrant, taking alternate slabs of each group.
template <bool GRAD>
struct TcCfg {
    static constexpr int G = GRAD ? 2 : 4;                   // slabs per group
    static constexpr int NBMAX = 2 * G * kTB1Max;            // N of one product (Re and Im rows)
    static constexpr int NCONV = 2;                          // split warps
    static constexpr int WPREP = 2 + NCONV;                  // first of 4 prep warps
    static constexpr int WRED = WPREP + 4;                   // first of 8 reduction warps
    static constexpr int NRED = 8;
    static constexpr int THREADS = 32 * (WRED + NRED);
    static constexpr int DBUF = 2;                           // accumulator buffers
    static constexpr uint32_t DCOLS = GRAD ? 2 * NBMAX : NBMAX;   // accumulator columns per buffer (D, D')
    static constexpr int ABUF = GRAD ? 1 : 2;                // operand (and window table) buffers
    static constexpr uint32_t ACOLS = GRAD ? 128 : 64;       // operand columns per buffer (hi, lo, hi', lo')
    static constexpr uint32_t ABASE = DBUF * DCOLS;
    static constexpr uint32_t ALLOC = 512;
    static constexpr int NS = GRAD ? 4 : 3;                  // tile stages
    static constexpr int STAGE = NBMAX * 128;                // bytes of one tile operand (hi or lo)
    static constexpr int NTAB = GRAD ? 2 : 1;                // window tables per axis (psi; psi')
    static constexpr int NXCH = GRAD ? 8 : 2;                // partial sums one reduction warp hands to its partner
    static_assert(ABASE + ABUF * ACOLS <= ALLOC, "tensor memory budget");
};

template <bool GRAD>
struct TcSmem {
    using C = TcCfg<GRAD>;
    // tile stages: [0] receives the raw FP32 tiles (TMA) and is split in place into the TF32
    // head, [1] takes the remainder
    alignas(1024) unsigned char b[C::NS][2][C::STAGE];
    float w0tab[2][C::NTAB][16][kPM];                        // per buffer: axis-0 psi (psi') per tap j and point row
    float w1tab[2][C::NTAB][kTB1Max][kPM];                   // per buffer: axis-1 psi (psi') per tile row
    float lanes[kPM][kLanes + 1];                            // prep: one point's axis-2 weights placed on the 32 lanes
    float xch[2][C::NXCH][kPM];                              // reduction: second warp's partial sums per point
    uint64_t tma_full[C::NS], conv_full[C::NS], empty[C::NS];
    uint64_t tfull[2], tempty[2], afull[2], aempty[2], tabfull[2], tabfree[2], xfull[2], xfree[2], done;
    uint32_t tmem_base;
    int abort;
};

struct TcArgs {
    const int4 *passes;                     // work list of passes (super-bin, first point, points)
    const int *npasses;                     // its length (device)
    int64_t M;
    const float4 *pts;
    const int *perm;
    double2 *vals;                          // interpolation output
    const unsigned long long *r2max;        // gradient: rho
    const double2 *gout;
    double *gxyz;
    double2 *gvals;                         // gradient form: the values too (NULL: not wanted)
    int *dev_flags;
    int TB1;                                // tile rows per slab (multiple of 8, >= C1 + 2q - 1)
    long long wait_cycles;                  // limit of every mbarrier wait (clock cycles)
    int withhold;                           // test hook: the prep warps withhold their operand arrival
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory operand descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
           ((uint64_t)2 << 61);
}

// TF32 head of x: round to nearest (ties away) at mantissa bit 13 with integer operations (a
// carry out of the mantissa moves into the exponent, which is the correctly rounded result).
// The remainder x - head is exact in FP32; the tensor core reads its top 19 bits.
__device__ __forceinline__ float tf32_head(float x) { return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u); }

// Branch-free window psi(x) and psi'(x) (zero for |x| > q) for the operand rows: straight-line
// code (approximate reciprocal square root, fast exponentials), so the 16 to 32 evaluations of a
// point interleave.  The KB exponent b (s - q) is taken as -b x^2 / (s + q): no cancellation
// near the peak, so the relative error of s enters psi only weakly.  `edge` is psi's limit for
// s -> 0 over the normalization (KB: 2 b e^(-bq)); `ih` is 1 / (2 lambda) (Gaussian).
template <int WIN>
__device__ __forceinline__ float win_fast(float x, float q, float par, float norm, float edge) {
    const float s2 = fmaf(-x, x, q * q);
    if constexpr (WIN == SGL_WIN_KB) {
        const float sv = (s2 > 1e-12f) ? s2 * rsqrtf(s2) : 0.f;
        const float e1 = __expf(-__fdividef(par * x * x, sv + q)), e2 = __expf(-par * (sv + q));
        const float v = (sv > 1e-3f) ? __fdividef(norm * (e1 - e2), sv) : norm * edge;
        return (s2 >= 0.f) ? v : 0.f;
    } else {
        const float v = __expf(-x * x * edge);
        return (s2 >= 0.f) ? v : 0.f;
    }
}

// psi and psi' together (shared square root and exponentials)
template <int WIN>
__device__ __forceinline__ float2 win_both_fast(float x, float q, float par, float norm, float edge) {
    const float s2 = fmaf(-x, x, q * q);
    if constexpr (WIN == SGL_WIN_KB) {
        const float sv = (s2 > 1e-12f) ? s2 * rsqrtf(s2) : 0.f;
        const float e1 = __expf(-__fdividef(par * x * x, sv + q)), em = __expf(-2.f * par * sv);
        const float isv = __fdividef(1.f, sv);
        const float v = (sv > 1e-3f) ? norm * e1 * (1.f - em) * isv : norm * edge;
        const float num = par * sv * (1.f + em) - (1.f - em);
        const float d = (sv > 1e-3f) ? -x * norm * e1 * num * isv * isv * isv : -x * norm * edge * (par * par / 3.f);
        return (s2 >= 0.f) ? make_float2(v, d) : make_float2(0.f, 0.f);
    } else {
        const float v = __expf(-x * x * edge);
        return (s2 >= 0.f) ? make_float2(v, -2.f * x * edge * v) : make_float2(0.f, 0.f);
    }
}

template <int WIN>
__device__ __forceinline__ float win_deriv_fast(float x, float q, float par, float norm, float edge) {
    const float s2 = fmaf(-x, x, q * q);
    if constexpr (WIN == SGL_WIN_KB) {
        // d/dx [sinh(b s)/s] = -x (b s cosh(b s) - sinh(b s)) / s^3; limit s -> 0: -x (2/3) b^3 e^(-bq) (normalized)
        const float sv = (s2 > 1e-12f) ? s2 * rsqrtf(s2) : 0.f;
        const float e1 = __expf(-__fdividef(par * x * x, sv + q)), em = __expf(-2.f * par * sv);
        const float num = par * sv * (1.f + em) - (1.f - em);
        const float v = (sv > 1e-3f) ? __fdividef(-x * norm * e1 * num, sv * sv * sv) : -x * norm * edge * (par * par / 3.f);
        return (s2 >= 0.f) ? v : 0.f;
    } else {
        const float v = -2.f * x * edge * __expf(-x * x * edge);
        return (s2 >= 0.f) ? v : 0.f;
    }
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
    return ok != 0;
}

// wait for the phase of the given parity to complete; false after about a second
// (limit: kWaitCycles unless a test shortens it, see sgl_test_hooks)
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit) {
    if (mbar_try(mbar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(mbar, parity))
        if (clock64() - t0 > limit) return false;
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

// D (TMEM) += A (TMEM) * B (shared memory)
__device__ __forceinline__ void mma_tf32_ts(uint32_t dtmem, uint32_t atmem, uint64_t bdesc, uint32_t idesc, uint32_t accumulate) {
    asm volatile("{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n"
                 :: "r"(dtmem), "r"(atmem), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar) : "memory");
}

// 8 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
                 "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
                 :: "r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                    "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])),
                    "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
                    "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
                    "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])), "r"(__float_as_uint(v[18])),
                    "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])), "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])),
                    "r"(__float_as_uint(v[23])), "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
                    "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])), "r"(__float_as_uint(v[30])),
                    "r"(__float_as_uint(v[31]))
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TF32 head and remainder of 32 weights, written to TMEM columns col (head) and col + 32 (remainder)
__device__ __forceinline__ void store_split_tmem(uint32_t taddr, const float *w) {
    float h[32], l[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        h[k] = tf32_head(w[k]);
        l[k] = w[k] - h[k];
    }
    tmem_st32(taddr, h);
    tmem_st32(taddr + 32, l);
}

// The CTA's sequence of passes: entries blockIdx.x, blockIdx.x + gridDim.x, ... of the pass work
// list (at most 128 points of one super-bin each, full passes first), so every CTA gets the same
// number of full passes to within one.  Every role walks the same sequence.
static_assert(kPM == kTcPass, "pass size and work-list piece size disagree");
// A pass's points are sorted by cell column, axis-0 offset d0 first, so they touch only the slabs
// d0(first point) ... d0(last point) + 2q - 1: the slab groups g0 ... g1 (the others would add
// nothing).  Every role derives the same range from the pass's first and last point records.
struct PassIter {
    int64_t sb = -1;
    int k = -1, pass = 0, first = 0, np = 0, g0 = 0, g1 = -1;
};

__device__ __forceinline__ bool next_pass(PassIter &it, const TcArgs &a, const NGeom &g, int G, int NG) {
    it.k = (it.k < 0) ? (int)blockIdx.x : it.k + (int)gridDim.x;
    if (it.k >= __ldg(a.npasses)) return false;
    const int4 e = __ldg(a.passes + it.k);
    it.sb = e.x;
    it.first = e.y;
    it.np = e.z;
    it.pass = 0;
    const int sb0 = (int)(it.sb / ((int64_t)g.nsb1 * g.nsb2));
    int c0a, c0b, c1, c2;
    unpack_cells(__ldg(a.pts + e.y).w, c0a, c1, c2);
    unpack_cells(__ldg(a.pts + e.y + max(e.z, 1) - 1).w, c0b, c1, c2);
    it.g0 = max(c0a - sb0 * kC0, 0) / G;
    it.g1 = min((c0b - sb0 * kC0 + 2 * g.q - 1) / G, NG - 1);
    return true;
}

// (sum_tb w[tb] re[tb], sum_tb w[tb] im[tb]) over tb < tbn (even): packed multiply-adds over
// pairs of adjacent rows, so that both operands of each are consecutive registers (re and im as
// one tensor-memory load wrote them, w as two loads of the table); even and odd rows are summed
// apart and added at the end.  Pairing (re[tb], im[tb]) under a broadcast weight instead made the
// values-and-gradient kernel 7 % slower (1.143 against 1.071 ms at B = 64, 10^6 points, q = 8).
__device__ __forceinline__ float2 row_pairs(const float (&w)[kTB1Max], const float (&re)[kTB1Max], const float (&im)[kTB1Max], int tbn) {
    float2 pr = make_float2(0.f, 0.f), pi = pr;
#pragma unroll
    for (int k = 0; k < kTB1Max / 2; ++k)
        if (2 * k < tbn) {
            const float2 wk = make_float2(w[2 * k], w[2 * k + 1]);
            pr = ffma2(wk, make_float2(re[2 * k], re[2 * k + 1]), pr);
            pi = ffma2(wk, make_float2(im[2 * k], im[2 * k + 1]), pi);
        }
    return make_float2(pr.x + pr.y, pi.x + pi.y);
}

template <int WIN, bool GRAD>
__global__ void __launch_bounds__(TcCfg<GRAD>::THREADS, 1)
k_nufft_tc(const __grid_constant__ CUtensorMap tmap, NGeom g, TcArgs args) {
    using Cfg = TcCfg<GRAD>;
    using S = TcSmem<GRAD>;
    constexpr int G = Cfg::G, NS = Cfg::NS;
    extern __shared__ unsigned char smem_raw[];
    S &sm = *reinterpret_cast<S *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);

    const int q = g.q, q2 = 2 * q;
    const int T0 = kC0 + q2 - 1;
    const int NG = (T0 + G - 1) / G;                 // slab groups per pass
    const int TB1 = args.TB1, NB = 2 * G * TB1;      // rows per slab, N of one product
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // ---- setup: zero tiles, barriers (thread 0), tensor memory (warp 1)
    for (int i = threadIdx.x; i < (int)(sizeof(sm.b) / 16); i += Cfg::THREADS)
        reinterpret_cast<float4 *>(&sm.b[0][0][0])[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(smem_addr(&sm.tma_full[i]), 1);
            mbar_init(smem_addr(&sm.conv_full[i]), Cfg::NCONV);
            mbar_init(smem_addr(&sm.empty[i]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_addr(&sm.tfull[i]), 1);
            mbar_init(smem_addr(&sm.tempty[i]), Cfg::NRED);
            mbar_init(smem_addr(&sm.afull[i]), 4);
            mbar_init(smem_addr(&sm.aempty[i]), 1);              // operand buffer read by its last MMA (commit)
            mbar_init(smem_addr(&sm.tabfull[i]), 4);
            mbar_init(smem_addr(&sm.tabfree[i]), Cfg::NRED);     // tables read by every reduction warp
            mbar_init(smem_addr(&sm.xfull[i]), 4);
            mbar_init(smem_addr(&sm.xfree[i]), 4);
        }
        mbar_init(smem_addr(&sm.done), 1);
        sm.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_addr(&sm.tmem_base)),
                     "r"(Cfg::ALLOC));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    volatile int *abort_flag = &sm.abort;
    const long long lim = args.wait_cycles;

    if (warp == 0) {
        // ---------------- TMA producer: raw Re / Im tiles of every slab group of every pass
        if (lane == 0) {
            const uint32_t tx = 2u * (uint32_t)(G * TB1) * 128u;
            int s = 0;
            PassIter it;
            while (!*abort_flag && next_pass(it, args, g, G, NG)) {
                const int sb1 = (int)(it.sb % g.nsb1), sb2 = (int)((it.sb / g.nsb1) % g.nsb2);
                const int sb0 = (int)(it.sb / ((int64_t)g.nsb1 * g.nsb2));
                const int x = sb2 * g.S2;             // halo-shifted azimuthal coordinate of lane 0
                const int y = sb1 * kC1 + 1;          // stored row of tile row 0 on axis 1 (first = -q)
                const int z0 = sb0 * kC0 + 1;         // stored row of slab 0 on axis 0
                bool ok = true;
                for (int gi = it.g0; gi <= it.g1; ++gi, ++s) {
                    const int st = s % NS;
                    if (s >= NS && !mbar_wait(smem_addr(&sm.empty[st]), ((s / NS) + 1) & 1, lim)) ok = false;
                    if (!ok || *abort_flag) { ok = false; break; }
                    const uint32_t fb = smem_addr(&sm.tma_full[st]);
                    mbar_expect_tx(fb, tx);
                    const uint32_t hi = smem_addr(sm.b[st][0]);
                    tma_load_4d(hi, &tmap, fb, x, y, z0 + G * gi, 0);
                    tma_load_4d(hi + G * TB1 * 128, &tmap, fb, x, y, z0 + G * gi, 1);
                }
                if (!ok) { *abort_flag = 1; break; }
            }
            // the last loads issued into each stage have landed before the CTA may exit
            for (int k = (s > NS ? s - NS : 0); k < s; ++k) mbar_wait(smem_addr(&sm.tma_full[k % NS]), (k / NS) & 1, lim);
        }
    } else if (warp >= 2 && warp < Cfg::WPREP) {
        // ---------------- split warps: raw tiles -> TF32 head (in place) + remainder
        const int part = warp - 2;
        const int nvec = NB * 8;                      // float4 per tile operand (NB rows x 128 bytes)
        int s = 0;
        PassIter it;
        bool ok = true;
        while (ok && next_pass(it, args, g, G, NG)) {
            for (int gi = it.g0; gi <= it.g1; ++gi, ++s) {
                const int st = s % NS;
                ok = __all_sync(0xffffffffu, mbar_wait(smem_addr(&sm.tma_full[st]), (s / NS) & 1, lim) && !*abort_flag);
                if (!ok) break;
                float4 *hi = reinterpret_cast<float4 *>(sm.b[st][0]);
                float4 *lo = reinterpret_cast<float4 *>(sm.b[st][1]);
#pragma unroll 4
                for (int i = part * 32 + lane; i < nvec; i += 32 * Cfg::NCONV) {
                    const float4 v = hi[i];
                    float4 h, l;
                    h.x = tf32_head(v.x); l.x = v.x - h.x;
                    h.y = tf32_head(v.y); l.y = v.y - h.y;
                    h.z = tf32_head(v.z); l.z = v.z - h.z;
                    h.w = tf32_head(v.w); l.w = v.w - h.w;
                    hi[i] = h;
                    lo[i] = l;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_addr(&sm.conv_full[st]));
            }
        }
        if (!ok) *abort_flag = 1;
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tf32_idesc(NB);
            int s = 0, k = 0;
            bool ok = true;
            PassIter it;
            while (ok && next_pass(it, args, g, G, NG)) {
                const int abuf = k % Cfg::ABUF;
                ok = mbar_wait(smem_addr(&sm.afull[abuf]), (k / Cfg::ABUF) & 1, lim) && !*abort_flag;
                tc_fence_after();
                const uint32_t a = tmem + Cfg::ABASE + (uint32_t)abuf * Cfg::ACOLS;
                for (int gi = it.g0; gi <= it.g1 && ok; ++gi, ++s) {
                    const int st = s % NS, buf = s % Cfg::DBUF, use = s / Cfg::DBUF;
                    ok = mbar_wait(smem_addr(&sm.conv_full[st]), (s / NS) & 1, lim);
                    if (ok && use >= 1) ok = mbar_wait(smem_addr(&sm.tempty[buf]), (use + 1) & 1, lim);
                    if (!ok || *abort_flag) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t bhi = smem_addr(sm.b[st][0]), blo = smem_addr(sm.b[st][1]);
                    const uint32_t d = tmem + (uint32_t)buf * Cfg::DCOLS;
#pragma unroll
                    for (int ks = 0; ks < kLanes / 8; ++ks) {
                        const uint32_t ko = ks * 32, ka = ks * 8;     // 8 TF32 of K: 32 bytes, 8 columns
                        mma_tf32_ts(d, a + ka, sw128_desc(bhi + ko), idesc, ks > 0);
                        mma_tf32_ts(d, a + ka, sw128_desc(blo + ko), idesc, 1);
                        mma_tf32_ts(d, a + 32 + ka, sw128_desc(bhi + ko), idesc, 1);
                    }
                    if constexpr (GRAD) {
#pragma unroll
                        for (int ks = 0; ks < kLanes / 8; ++ks) {
                            const uint32_t ko = ks * 32, ka = ks * 8;
                            mma_tf32_ts(d + Cfg::NBMAX, a + 64 + ka, sw128_desc(bhi + ko), idesc, ks > 0);
                            mma_tf32_ts(d + Cfg::NBMAX, a + 64 + ka, sw128_desc(blo + ko), idesc, 1);
                            mma_tf32_ts(d + Cfg::NBMAX, a + 96 + ka, sw128_desc(bhi + ko), idesc, 1);
                        }
                    }
                    mma_commit(smem_addr(&sm.empty[st]));
                    mma_commit(smem_addr(&sm.tfull[buf]));
                }
                // the operand buffer is free once this pass's products have run (the window tables
                // have their own buffers, freed by the reduction warps)
                if (ok) mma_commit(smem_addr(&sm.aempty[abuf]));
                ++k;
            }
            if (!ok) *abort_flag = 1;
            // every MMA issued above has completed before tensor memory is released
            mma_commit(smem_addr(&sm.done));
            mbar_wait(smem_addr(&sm.done), 0, lim);
        }
    } else {
        // ---------------- point warps (one thread per point; TMEM lane = point)
        const int quad = warp & 3;                   // TMEM lanes 32 quad .. 32 quad + 31
        const int p = quad * 32 + lane;              // MMA row = point of the pass
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        const float qf = (float)q;
        const float par0 = (float)g.par[0], par1 = (float)g.par[1], par2 = (float)g.par[2];
        const float nrm0 = (float)g.norm[0], nrm1 = (float)g.norm[1], nrm2 = (float)g.norm[2];
        bool ok = true;
        PassIter it;
        if (warp < Cfg::WRED) {
            // ---- prep warps: operands (TMEM) and window tables (shared memory) of every pass
            // KB: psi's limit at |x| = q over the normalization, 2 b e^(-bq); Gaussian: 1 / (2 lambda)
            const bool kb = WIN == SGL_WIN_KB;
            const float edge0 = kb ? 2.f * par0 * expf(-par0 * qf) : 0.5f / par0;
            const float edge1 = kb ? 2.f * par1 * expf(-par1 * qf) : 0.5f / par1;
            const float edge2 = kb ? 2.f * par2 * expf(-par2 * qf) : 0.5f / par2;
            int n = 0;
            while (ok && next_pass(it, args, g, G, NG)) {
                const int abuf = n % Cfg::ABUF, use = n / Cfg::ABUF;
                const int tbuf = n & 1, tuse = n >> 1;        // window tables: two buffers in shared memory
                const int idx = it.pass * kPM + p;
                const bool live = idx < it.np;
                const float4 pt = args.pts[it.first + (live ? idx : 0)];
                int c0, c1, c2;
                unpack_cells(pt.w, c0, c1, c2);
                const int sb1 = (int)(it.sb % g.nsb1), sb2 = (int)((it.sb / g.nsb1) % g.nsb2);
                const int k0 = c2 - q + 1 - (sb2 * g.S2 - tc_halo(q));     // lane of the point's first tap
                const int d1 = c1 - sb1 * kC1;
                // Order: the axis-2 weights into registers first, then the window tables (their
                // own two buffers), and only then the wait for the operand buffer, so that the
                // tensor pipe waits for nothing but the operand stores between passes.  The 2q
                // nonzero weights per axis come from compile-time tap indices (independent chains).
                float v2[16], e2[GRAD ? 16 : 1];
#pragma unroll
                for (int rel = 0; rel < 16; ++rel) {
                    if constexpr (GRAD) {
                        const float2 v = win_both_fast<WIN>(pt.z + (float)(q - 1 - rel), qf, par2, nrm2, edge2);
                        v2[rel] = v.x;
                        e2[rel] = v.y;
                    } else {
                        v2[rel] = win_fast<WIN>(pt.z + (float)(q - 1 - rel), qf, par2, nrm2, edge2);
                    }
                }
                if (tuse >= 1)
                    ok = __all_sync(0xffffffffu, mbar_wait(smem_addr(&sm.tabfree[tbuf]), (tuse + 1) & 1, lim) && !*abort_flag);
                if (!ok) break;
#pragma unroll
                for (int tb = 0; tb < kTB1Max; ++tb) {
                    sm.w1tab[tbuf][0][tb][p] = 0.f;
                    if constexpr (GRAD) sm.w1tab[tbuf][GRAD ? 1 : 0][tb][p] = 0.f;
                }
#pragma unroll
                for (int rel = 0; rel < 16; ++rel) {
                    if constexpr (GRAD) {
                        const float2 v = win_both_fast<WIN>(pt.y + (float)(q - 1 - rel), qf, par1, nrm1, edge1);
                        if (live && rel < q2) {
                            sm.w1tab[tbuf][0][d1 + rel][p] = v.x;
                            sm.w1tab[tbuf][GRAD ? 1 : 0][d1 + rel][p] = v.y;
                        }
                    } else {
                        const float v = win_fast<WIN>(pt.y + (float)(q - 1 - rel), qf, par1, nrm1, edge1);
                        if (live && rel < q2) sm.w1tab[tbuf][0][d1 + rel][p] = v;
                    }
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if constexpr (GRAD) {
                        const float2 v = win_both_fast<WIN>(pt.x + (float)(q - 1 - j), qf, par0, nrm0, edge0);
                        if (j < q2) {
                            sm.w0tab[tbuf][0][j][p] = v.x;
                            sm.w0tab[tbuf][GRAD ? 1 : 0][j][p] = v.y;
                        }
                    } else {
                        const float v = win_fast<WIN>(pt.x + (float)(q - 1 - j), qf, par0, nrm0, edge0);
                        if (j < q2) sm.w0tab[tbuf][0][j][p] = v;
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_addr(&sm.tabfull[tbuf]));
                // operands: the axis-2 weights placed on the 32 lanes at the point's offset k0
                // (through this thread's row of shared memory), split, into TMEM
                if (use >= 1) ok = __all_sync(0xffffffffu, mbar_wait(smem_addr(&sm.aempty[abuf]), (use + 1) & 1, lim) && !*abort_flag);
                if (!ok) break;
                tc_fence_after();
                const uint32_t ta_ = tmem + lane_base + Cfg::ABASE + (uint32_t)abuf * Cfg::ACOLS;
                float *row = sm.lanes[p];
                float w[kLanes];
#pragma unroll
                for (int k = 0; k < kLanes; ++k) row[k] = 0.f;
#pragma unroll
                for (int rel = 0; rel < 16; ++rel)
                    if (live && rel < q2) row[k0 + rel] = v2[rel];
#pragma unroll
                for (int k = 0; k < kLanes; ++k) w[k] = row[k];
                store_split_tmem(ta_, w);
                if constexpr (GRAD) {
#pragma unroll
                    for (int rel = 0; rel < 16; ++rel)
                        if (live && rel < q2) row[k0 + rel] = e2[rel];
#pragma unroll
                    for (int k = 0; k < kLanes; ++k) w[k] = row[k];
                    store_split_tmem(ta_ + 64, w);
                }
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0 && !args.withhold) mbar_arrive(smem_addr(&sm.afull[abuf]));
                ++n;
            }
        } else {
            // ---- reduction warps: contract the accumulators with the window tables
            float rho = 0.f;
            if constexpr (GRAD) rho = rho_from_r2max(args.r2max);
            const int half = (warp - Cfg::WRED) >> 2;     // this warp takes slabs z = half, half + 2, ... of a group
            int s = 0, n = 0;
            while (ok && next_pass(it, args, g, G, NG)) {
                const int tbuf = n & 1, tuse = n >> 1;
                ok = __all_sync(0xffffffffu, mbar_wait(smem_addr(&sm.tabfull[tbuf]), tuse & 1, lim) && !*abort_flag);
                if (!ok) break;
                const int idx = it.pass * kPM + p;
                const bool live = idx < it.np;
                const int64_t i = it.first + (live ? idx : 0);
                const float4 pt = args.pts[i];
                int c0, c1, c2;
                unpack_cells(pt.w, c0, c1, c2);
                const int sb0 = (int)(it.sb / ((int64_t)g.nsb1 * g.nsb2));
                const int d0 = c0 - sb0 * kC0;
                float w1[kTB1Max], e1[GRAD ? kTB1Max : 1];
#pragma unroll
                for (int tb = 0; tb < kTB1Max; ++tb) {
                    w1[tb] = sm.w1tab[tbuf][0][tb][p];
                    if constexpr (GRAD) e1[tb] = sm.w1tab[tbuf][GRAD ? 1 : 0][tb][p];
                }
                float2 acc = make_float2(0.f, 0.f), acc1 = acc, acc2 = acc, accv = acc;
                for (int gi = it.g0; gi <= it.g1; ++gi, ++s) {
                    const int buf = s % Cfg::DBUF, use = s / Cfg::DBUF;
                    ok = __all_sync(0xffffffffu, mbar_wait(smem_addr(&sm.tfull[buf]), use & 1, lim) && !*abort_flag);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t taddr = tmem + lane_base + (uint32_t)buf * Cfg::DCOLS;
#pragma unroll 1
                    for (int z = half; z < G; z += 2) {
                        // slab ta = G gi + z: Re of tile row tb at column z TB1 + tb, Im at G TB1 + z TB1 + tb
                        const int j = G * gi + z - d0;
                        float re[kTB1Max], im[kTB1Max];
                        const uint32_t cre = taddr + z * TB1, cim = taddr + (G + z) * TB1;
                        const int tbn = TB1 > 16 ? 24 : 16;
                        tmem_ld8(cre, re);
                        tmem_ld8(cim, im);
                        tmem_ld8(cre + 8, re + 8);
                        tmem_ld8(cim + 8, im + 8);
                        if (TB1 > 16) {
                            tmem_ld8(cre + 16, re + 16);
                            tmem_ld8(cim + 16, im + 16);
                        }
                        tmem_wait_ld();
                        const bool on = j >= 0 && j < q2;
                        float2 r = make_float2(0.f, 0.f), rs = r, rt = r;
                        if (on) {
                            r = row_pairs(w1, re, im, tbn);
                            if constexpr (GRAD) rs = row_pairs(e1, re, im, tbn);
                        }
                        if constexpr (GRAD) {
                            // the derivative product (w2'), into the same registers
                            tmem_ld8(cre + Cfg::NBMAX, re);
                            tmem_ld8(cim + Cfg::NBMAX, im);
                            tmem_ld8(cre + Cfg::NBMAX + 8, re + 8);
                            tmem_ld8(cim + Cfg::NBMAX + 8, im + 8);
                            if (TB1 > 16) {
                                tmem_ld8(cre + Cfg::NBMAX + 16, re + 16);
                                tmem_ld8(cim + Cfg::NBMAX + 16, im + 16);
                            }
                            tmem_wait_ld();
                            if (on) rt = row_pairs(w1, re, im, tbn);
                        }
                        if (!on) continue;
                        const float w0 = sm.w0tab[tbuf][0][j][p];
                        if constexpr (GRAD) {
                            const float e0 = sm.w0tab[tbuf][GRAD ? 1 : 0][j][p];
                            acc = ffma2(make_float2(e0, e0), r, acc);      // ds/du0
                            acc1 = ffma2(make_float2(w0, w0), rs, acc1);   // ds/du1
                            acc2 = ffma2(make_float2(w0, w0), rt, acc2);   // ds/du2
                            accv = ffma2(make_float2(w0, w0), r, accv);    // s
                        } else {
                            acc = ffma2(make_float2(w0, w0), r, acc);
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_addr(&sm.tempty[buf]));
                }
                if (!ok) break;
                // this pass's window tables are no longer read
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_addr(&sm.tabfree[tbuf]));
                // partner warps (same lane quadrant) combine their partial sums; the half-0 warp writes
                const int xs = n & 1;
                if (half == 1) {
                    if (n >= 2) ok = __all_sync(0xffffffffu, mbar_wait(smem_addr(&sm.xfree[xs]), ((n >> 1) + 1) & 1, lim) && !*abort_flag);
                    if (!ok) break;
                    sm.xch[xs][0][p] = acc.x;
                    sm.xch[xs][1][p] = acc.y;
                    if constexpr (GRAD) {
                        sm.xch[xs][2 % Cfg::NXCH][p] = acc1.x;
                        sm.xch[xs][3 % Cfg::NXCH][p] = acc1.y;
                        sm.xch[xs][4 % Cfg::NXCH][p] = acc2.x;
                        sm.xch[xs][5 % Cfg::NXCH][p] = acc2.y;
                        sm.xch[xs][6 % Cfg::NXCH][p] = accv.x;
                        sm.xch[xs][7 % Cfg::NXCH][p] = accv.y;
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_addr(&sm.xfull[xs]));
                } else {
                    ok = __all_sync(0xffffffffu, mbar_wait(smem_addr(&sm.xfull[xs]), (n >> 1) & 1, lim) && !*abort_flag);
                    if (!ok) break;
                    acc.x += sm.xch[xs][0][p];
                    acc.y += sm.xch[xs][1][p];
                    if constexpr (GRAD) {
                        acc1.x += sm.xch[xs][2 % Cfg::NXCH][p];
                        acc1.y += sm.xch[xs][3 % Cfg::NXCH][p];
                        acc2.x += sm.xch[xs][4 % Cfg::NXCH][p];
                        acc2.y += sm.xch[xs][5 % Cfg::NXCH][p];
                        accv.x += sm.xch[xs][6 % Cfg::NXCH][p];
                        accv.y += sm.xch[xs][7 % Cfg::NXCH][p];
                    }
                    __syncwarp();
                    if (lane == 0) mbar_arrive(smem_addr(&sm.xfree[xs]));
                    if (live) {
                        const int dst = args.perm[i];
                        if constexpr (GRAD) {
                            grad_chain32(g, rho, c0, c1, c2, pt.x, pt.y, pt.z, acc.x, acc.y, acc1.x, acc1.y, acc2.x, acc2.y,
                                         args.gout[dst], args.gxyz + 3 * (int64_t)dst);
                            if (args.gvals) args.gvals[dst] = make_double2((double)accv.x, (double)accv.y);
                        } else
                            args.vals[dst] = make_double2((double)acc.x, (double)acc.y);
                    }
                }
                ++n;
            }
        }
        if (!ok) *abort_flag = 1;
    }
    tc_fence_before();
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) atomicOr(args.dev_flags, 2);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(Cfg::ALLOC));
    }
}

int tile_rows(int q) { return (kC1 + 2 * q - 1 + 7) / 8 * 8; }

}  // namespace

// ---------------------------------------------------------------- host side
bool tc_eligible(const sgl_plan *p) {
    return p->prec == SGL_FP32_MIXED && !(p->flags & SGL_FLAG_SIMT) && p->q <= 8 && p->ax[0].windowed && p->ax[1].windowed &&
           p->bins.C0 == kC0 && p->bins.C1 == kC1 && p->bins.S2 % 4 == 0 && p->bins.S2 + tc_halo(p->q) + p->q <= kLanes;
}

// Which operations take the tensor-core kernels by default (SGL_FLAG_TC: every eligible one).
// Measured on GB300 (B = 64, 10^6 points, ms, tensor cores / CUDA cores): q = 8 interpolation
// 0.89 / 1.53, gradient 1.99 / 2.66; q = 6: 0.69 / 1.23, 1.69 / 1.93; q = 4: 0.54 / 0.28,
// 1.27 / 0.48 (the CUDA-core kernels' work falls as q^3, the slab products' much less).
void tc_choose(sgl_plan *p) {
    const bool use = p->tc && ((p->flags & SGL_FLAG_TC) || p->q >= 6);
    p->tc_interp = use;
    p->tc_grad = use;         // equal: the forward FFT then writes only the planes both kernels read
    p->tc_spread = false;     // spreading: the CUDA-core kernel (sgl_nufft.cu) wins in time and accuracy
}

int64_t tc_plane_floats(const sgl_plan *p) {
    return 2 * (int64_t)p->ax[0].rows * p->ax[1].rows * tc_pitch(p->ax[2].N);
}

namespace {
std::mutex g_encode_mu;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

// tensor map over the planes: dims (pitch, rows1, rows0, 2 planes), box 32 lanes x TB1 rows x G slabs
cudaError_t encode_map(sgl_plan *p, int G, void *out) {
    const int pitch = tc_pitch(p->ax[2].N);
    const cuuint64_t dims[4] = {(cuuint64_t)pitch, (cuuint64_t)p->ax[1].rows, (cuuint64_t)p->ax[0].rows, 2};
    const cuuint64_t strides[3] = {(cuuint64_t)pitch * 4, (cuuint64_t)pitch * 4 * p->ax[1].rows,
                                   (cuuint64_t)pitch * 4 * p->ax[1].rows * p->ax[0].rows};
    const cuuint32_t box[4] = {(cuuint32_t)kLanes, (cuuint32_t)tile_rows(p->q), (cuuint32_t)G, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = g_encode(reinterpret_cast<CUtensorMap *>(out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p->b.planes, dims, strides,
                          box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}
}  // namespace

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
    static_assert(sizeof(CUtensorMap) <= sizeof(p->tc_map[0]), "tensor map storage");
    cudaError_t e = encode_map(p, TcCfg<false>::G, p->tc_map[0]);
    if (e == cudaSuccess) e = encode_map(p, TcCfg<true>::G, p->tc_map[1]);
    return e;
}

namespace {

template <int WIN, bool GRAD>
cudaError_t run_tc(sgl_plan *p, TcArgs a) {
    cudaError_t e;
    // the 512 TMEM columns a CTA allocates are the whole SM's: ask for enough shared memory that
    // no second CTA of this kernel fits beside it (its allocation would wait for the first)
    const size_t smem = std::max<size_t>(sizeof(TcSmem<GRAD>) + 1024, (size_t)120 * 1024);
    auto kern = k_nufft_tc<WIN, GRAD>;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
    const CUtensorMap *map = reinterpret_cast<const CUtensorMap *>(p->tc_map[GRAD ? 1 : 0]);
    const int64_t grid = std::min<int64_t>(work_list_cap(p->M, p->bins.nsuper, kTcPass), p->num_sms);
    kern<<<(unsigned)grid, TcCfg<GRAD>::THREADS, smem, p->stream>>>(*map, make_geom(p), a);
    p->launches += 1;
    return cudaGetLastError();
}

TcArgs base_args(const sgl_plan *p) {
    TcArgs a{};
    a.passes = p->b.work[0];
    a.npasses = p->b.work_len;
    a.M = p->M;
    a.pts = p->b.pts32;
    a.perm = p->b.perm;
    a.r2max = p->b.r2max;
    a.dev_flags = p->b.dev_flags;
    a.TB1 = tile_rows(p->q);
    a.wait_cycles = p->wait_cycles > 0 ? p->wait_cycles : kWaitCycles;
    a.withhold = (p->test_hooks & SGL_TEST_WITHHOLD_ARRIVAL) ? 1 : 0;
    return a;
}

}  // namespace

cudaError_t launch_interp_tc(sgl_plan *p, double2 *vals) {
    TcArgs a = base_args(p);
    a.vals = vals;
    return p->window == SGL_WIN_KB ? run_tc<SGL_WIN_KB, false>(p, a) : run_tc<SGL_WIN_GAUSS, false>(p, a);
}

cudaError_t launch_grad_tc(sgl_plan *p, const double2 *gout, double *gxyz, double2 *vals) {
    TcArgs a = base_args(p);
    a.gout = gout;
    a.gxyz = gxyz;
    a.gvals = vals;
    return p->window == SGL_WIN_KB ? run_tc<SGL_WIN_KB, true>(p, a) : run_tc<SGL_WIN_GAUSS, true>(p, a);
}

}  // namespace sgl
