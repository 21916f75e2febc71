// sgl_fft.cu -- the oversampled 3-D FFT of the NFFT (Sect. 2: alpha = (sigma n)^{-d} F^H beta),
// as three batched 1-D passes over tiles of lines staged in shared memory.
//
// The transform is pruned on both sides: the input eta is nonzero only on
// |k0| <= 2B-2, |k1| <= B-1, |k2| <= B-1 (degrees stated in Sect. 6), and the
// interpolation only reads grid rows within q of the range the points can reach
// (t0, theta in [0, pi]: rows [-q, N/2+q] on the first two axes).  Each pass
// places its L_in input elements at positions (e + in_first) mod N of a length-N
// line (zeros elsewhere), runs an in-place mixed-radix decimation-in-frequency
// FFT (radices 8, 4, 2, 3, 5; output in digit-reversed slots), and writes the
// L_out output positions (e + out_first) mod N.  The (sigma n)^{-d} scale and the
// window deconvolution 1/phitilde_k are folded into per-element and per-line factors.
//
// FP32-mixed plans run their two radial-axis passes (pass A of the forward transform, pass A'
// of the adjoint) in double-float arithmetic and the four angular passes in binary32.  The
// radial DFT mixes every radius: its rounding error lands on all rows l0 alike, also at radii
// r near rho where no point lies and the radial conversion matrices K_l (polynomials of degree
// up to 2B - 2 in r) are largest, so the adjoint's K_l^T amplifies it (measured at B = 64, 10^6
// points: a binary32 radial pass alone made the adjoint coefficients 2.4e-5 wrong relative to
// their maximum; binary32 angular passes, whose errors stay on the rows of their own radius, and
// binary32 spreading 2e-8 and 6e-8).
#include "sgl_dfl.cuh"
#include "sgl_internal.cuh"

#include <type_traits>

namespace sgl {
namespace {

// Double-float scalars (sgl_dfl.cuh) carry the radial passes of FP32-mixed plans.
// multiplication by a sign s = +1 or -1 (the transform direction)
__device__ __forceinline__ dfl operator*(int s, dfl a) { return s > 0 ? a : -a; }
__device__ __forceinline__ dfl operator*(dfl a, int s) { return s > 0 ? a : -a; }

template <typename T> struct CT;
template <> struct CT<float> { using type = float2; };
template <> struct CT<double> { using type = double2; };
template <> struct CT<dfl> { using type = dfl2; };
template <typename T> using C2 = typename CT<T>::type;

// a scalar of the pass arithmetic stored as the output type's scalar, and widened to binary64
__device__ __forceinline__ float narrow_f(float v) { return v; }
__device__ __forceinline__ float narrow_f(dfl v) { return __fadd_rn(v.h, v.l); }
__device__ __forceinline__ double widen(float v) { return (double)v; }
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ double widen(dfl v) { return (double)v.h + (double)v.l; }
template <typename S, typename V> __device__ __forceinline__ S narrow(V v) {
    if constexpr (sizeof(S) == 4) return narrow_f(v);
    else return widen(v);
}

template <typename T> __device__ __forceinline__ C2<T> mk(T x, T y) { C2<T> r; r.x = x; r.y = y; return r; }
template <typename T> __device__ __forceinline__ C2<T> add(C2<T> a, C2<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ C2<T> sub(C2<T> a, C2<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ C2<T> mul(C2<T> a, C2<T> b) { return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
// multiply by s*i (s = +-1)
template <typename T> __device__ __forceinline__ C2<T> mul_si(C2<T> a, int s) { return s > 0 ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x); }

// in-place r-point DFT  y_u = sum_t x_t e^{s 2 pi i t u / r}
template <typename T>
__device__ __forceinline__ void dft2(C2<T> *x) { C2<T> a = x[0], b = x[1]; x[0] = add<T>(a, b); x[1] = sub<T>(a, b); }

template <typename T>
__device__ __forceinline__ void dft4(C2<T> *x, int s) {
    C2<T> a = add<T>(x[0], x[2]), b = sub<T>(x[0], x[2]);
    C2<T> c = add<T>(x[1], x[3]), d = mul_si<T>(sub<T>(x[1], x[3]), s);
    x[0] = add<T>(a, c); x[2] = sub<T>(a, c); x[1] = add<T>(b, d); x[3] = sub<T>(b, d);
}

template <typename T>
__device__ __forceinline__ void dft8(C2<T> *x, int s) {
    C2<T> e[4] = {x[0], x[2], x[4], x[6]}, o[4] = {x[1], x[3], x[5], x[7]};
    dft4<T>(e, s);
    dft4<T>(o, s);
    constexpr T h = T(0.70710678118654752440);
    // W8^u = e^{s 2 pi i u / 8}
    C2<T> w1 = mk<T>(h, s * h), w3 = mk<T>(-h, s * h);
    C2<T> t0 = o[0], t1 = mul<T>(o[1], w1), t2 = mul_si<T>(o[2], s), t3 = mul<T>(o[3], w3);
    x[0] = add<T>(e[0], t0); x[4] = sub<T>(e[0], t0);
    x[1] = add<T>(e[1], t1); x[5] = sub<T>(e[1], t1);
    x[2] = add<T>(e[2], t2); x[6] = sub<T>(e[2], t2);
    x[3] = add<T>(e[3], t3); x[7] = sub<T>(e[3], t3);
}

template <typename T>
__device__ __forceinline__ void dft3(C2<T> *x, int s) {
    constexpr T c = T(-0.5), d0 = T(0.86602540378443864676);
    const T d = d0 * s;                                        // W3 = c + i d
    C2<T> a = add<T>(x[1], x[2]), b = sub<T>(x[1], x[2]);
    C2<T> y0 = add<T>(x[0], a);
    C2<T> m = mk<T>(x[0].x + c * a.x, x[0].y + c * a.y);
    C2<T> n = mk<T>(-d * b.y, d * b.x);                        // i d (x1 - x2)
    x[0] = y0; x[1] = add<T>(m, n); x[2] = sub<T>(m, n);
}

template <typename T>
__device__ __forceinline__ void dft5(C2<T> *x, int s) {
    constexpr T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);
    constexpr T s1p = T(0.95105651629515357212), s2p = T(0.58778525229247312917);
    const T s1 = s1p * s, s2 = s2p * s;
    C2<T> a1 = add<T>(x[1], x[4]), b1 = sub<T>(x[1], x[4]);
    C2<T> a2 = add<T>(x[2], x[3]), b2 = sub<T>(x[2], x[3]);
    C2<T> y0 = add<T>(x[0], add<T>(a1, a2));
    C2<T> m1 = mk<T>(x[0].x + c1 * a1.x + c2 * a2.x, x[0].y + c1 * a1.y + c2 * a2.y);
    C2<T> m2 = mk<T>(x[0].x + c2 * a1.x + c1 * a2.x, x[0].y + c2 * a1.y + c1 * a2.y);
    // i (s1 b1 + s2 b2) and i (s2 b1 - s1 b2)
    C2<T> n1 = mk<T>(-(s1 * b1.y + s2 * b2.y), s1 * b1.x + s2 * b2.x);
    C2<T> n2 = mk<T>(-(s2 * b1.y - s1 * b2.y), s2 * b1.x - s1 * b2.x);
    x[0] = y0; x[1] = add<T>(m1, n1); x[4] = sub<T>(m1, n1); x[2] = add<T>(m2, n2); x[3] = sub<T>(m2, n2);
}

enum { LOAD_STRIDED = 0, LOAD_ZETA = 1 };

struct ZetaSrc {
    const double2 *zeta;   // [K0+1][K1+1][2K1+1]
    int K0, K1;
};

template <typename C> __device__ __forceinline__ double2 to_d2(C v) { return make_double2((double)v.x, (double)v.y); }

template <typename T, int R>
__device__ __forceinline__ void dft_r(C2<T> *x, int s) {
    if constexpr (R == 2) dft2<T>(x);
    else if constexpr (R == 3) dft3<T>(x, s);
    else if constexpr (R == 4) dft4<T>(x, s);
    else if constexpr (R == 5) dft5<T>(x, s);
    else dft8<T>(x, s);
}

// q / d and q % d for d > 0; a shift and a mask when d is a power of two
__device__ __forceinline__ void divmod(int q, int d, int &quo, int &rem) {
    if ((d & (d - 1)) == 0) {
        const int sh = __ffs(d) - 1;
        quo = q >> sh;
        rem = q & (d - 1);
    } else {
        quo = q / d;
        rem = q - quo * d;
    }
}

// One decimation-in-frequency pass of radix R over every line of the tile (in place):
// sub-problem length L, span S = L / R; butterfly (g, nn) combines positions g L + nn + t S.
template <typename T, int R>
__device__ __forceinline__ void dif_stage(C2<T> *buf, int LS, int TB, int N, int L, int sign, const C2<T> *__restrict__ tw) {
    const int S = L / R;
    const int per_line = N / R;
    const int stride_tw = N / L;
    for (int w = threadIdx.x; w < TB * per_line; w += blockDim.x) {
        int bl, j, g, nn;
        divmod(w, per_line, bl, j);
        divmod(j, S, g, nn);
        C2<T> *base = buf + bl * LS + g * L + nn;
        C2<T> x[R];
#pragma unroll
        for (int t = 0; t < R; ++t) x[t] = base[t * S];
        dft_r<T, R>(x, sign);
        base[0] = x[0];
        const int tstep = nn * stride_tw;         // nn * u * stride_tw < N: no reduction needed
#pragma unroll
        for (int u = 1; u < R; ++u) {
            C2<T> wv = tw[tstep * u];
            if (sign < 0) wv.y = -wv.y;
            base[u * S] = mul<T>(x[u], wv);
        }
    }
}

__device__ __forceinline__ int wrapN(int e, int N) {
    if (e < 0) e += N;
    if (e >= N) e -= N;
    return e;
}

template <typename T, typename InC, typename OutC, int MODE>
__global__ void __launch_bounds__(256) k_fft_pass(FftPass ps, int TB, int lgTB, const InC *__restrict__ in, OutC *__restrict__ out,
                                                  ZetaSrc zs, int scale_on_output) {
    extern __shared__ unsigned char smem_raw[];
    C2<T> *buf = reinterpret_cast<C2<T> *>(smem_raw);
    const int N = ps.N;
    const int LS = N + 1;                          // padded line stride in shared memory
    const int64_t tiles_inner = (ps.nb_inner + TB - 1) / TB;
    const int64_t outer = blockIdx.x / tiles_inner;
    const int64_t inner0 = (blockIdx.x % tiles_inner) * TB;
    const int nlines = (int)min((int64_t)TB, ps.nb_inner - inner0);
    const int tid = threadIdx.x, NT = blockDim.x;

    // ---- load: position pos of a line holds input element e = pos - in_first (mod N), zero if e >= L_in.
    // Items j = tid + NT r of the TB x N tile (element-contiguous inputs: line j / N, position j % N;
    // strided inputs: line j % TB, position j / TB, so that a warp reads consecutive lines), loaded
    // in batches of kBatch independent loads before they go to shared memory.
    const bool in_elem_fast = (MODE == LOAD_STRIDED) && (ps.in_se == 1);
    const int total = TB * N;
    constexpr int kBatch = 8;
    for (int j0 = 0; j0 < total; j0 += NT * kBatch) {
        C2<T> v[kBatch];
        int dst[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int j = j0 + tid + NT * u;
            int bl, pos;
            if (in_elem_fast) { bl = j / N; pos = j - bl * N; }
            else { bl = j & (TB - 1); pos = j >> lgTB; }
            dst[u] = (j < total) ? bl * LS + pos : -1;
            const int e = wrapN(pos - ps.in_first, N);
            v[u] = mk<T>(T(0), T(0));
            if (j < total && bl < nlines && e < ps.L_in) {
                const int64_t inner = inner0 + bl;
                double2 d;
                if (MODE == LOAD_ZETA) {
                    // line = (k1, m) over (2K1+1)^2, element = k0 + K0; eta mirrored from zeta
                    const int W = 2 * zs.K1 + 1;
                    const int mi = (int)(inner % W);
                    const int k1 = (int)(inner / W) - zs.K1;
                    const int k0 = e - zs.K0;
                    d = zs.zeta[((int64_t)abs(k0) * (zs.K1 + 1) + abs(k1)) * W + mi];
                    if (k1 < 0 && ((mi - zs.K1) & 1)) { d.x = -d.x; d.y = -d.y; }
                } else if (scale_on_output || (!ps.elem_scale && !ps.line_scale)) {
                    // no factor on the input: straight conversion to the pass arithmetic
                    const InC x = in[outer * ps.in_so + inner * ps.in_si + (int64_t)e * ps.in_se];
                    v[u] = mk<T>(T(x.x), T(x.y));
                    continue;
                } else {
                    d = to_d2(in[outer * ps.in_so + inner * ps.in_si + (int64_t)e * ps.in_se]);
                }
                if (!scale_on_output) {
                    double f = 1.0;
                    if (ps.elem_scale) f *= ps.elem_scale[e];
                    if (ps.line_scale) f *= ps.line_scale[outer * ps.nb_inner + inner];
                    d.x *= f; d.y *= f;
                }
                v[u] = mk<T>(T(d.x), T(d.y));
            }
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
            if (dst[u] >= 0) buf[dst[u]] = v[u];
    }
    __syncthreads();

    // ---- in-place decimation-in-frequency passes
    const C2<T> *tw = reinterpret_cast<const C2<T> *>(ps.tw);
    int L = N;
    for (int st = 0; st < ps.nrad; ++st) {
        switch (ps.rad[st]) {
            case 2: dif_stage<T, 2>(buf, LS, TB, N, L, ps.sign, tw); L /= 2; break;
            case 3: dif_stage<T, 3>(buf, LS, TB, N, L, ps.sign, tw); L /= 3; break;
            case 4: dif_stage<T, 4>(buf, LS, TB, N, L, ps.sign, tw); L /= 4; break;
            case 5: dif_stage<T, 5>(buf, LS, TB, N, L, ps.sign, tw); L /= 5; break;
            default: dif_stage<T, 8>(buf, LS, TB, N, L, ps.sign, tw); L /= 8; break;
        }
        __syncthreads();
    }

    // ---- split-plane output with a wrapped halo (one line after the other, consecutive columns)
    if constexpr (std::is_same<OutC, float2>::value) {
        if (ps.planes) {
            for (int bl = 0; bl < nlines; ++bl) {
                float *row = ps.planes + (inner0 + bl) * ps.pitch;
                for (int k = tid; k < ps.pitch; k += NT) {
                    int e = (k - ps.halo) % N;       // the halo can span more than one period of short lines
                    if (e < 0) e += N;
                    const C2<T> v = buf[bl * LS + __ldg(ps.rev + e)];
                    row[k] = narrow<float>(v.x);
                    row[ps.plane_n + k] = narrow<float>(v.y);
                }
            }
            return;
        }
    }

    // ---- store the output window (digit-reversed slots), optional scale on output
    const bool out_elem_fast = (ps.out_se == 1);
    const int bl_fast = tid & (TB - 1), pos_step = NT >> lgTB;
    for (int it = 0; it < (out_elem_fast ? TB : 1); ++it) {
        for (int k = out_elem_fast ? tid : (tid >> lgTB); k < ps.L_out; k += out_elem_fast ? NT : pos_step) {
            const int bl = out_elem_fast ? it : bl_fast;
            if (bl >= nlines) continue;
            const int e = k;
            const int64_t inner = inner0 + bl;
            const int pos = wrapN(e + ps.out_first, N);
            const C2<T> v = buf[bl * LS + __ldg(ps.rev + pos)];
            using S = decltype(OutC::x);
            OutC o;
            if (!(scale_on_output && (ps.elem_scale || ps.line_scale))) {
                o.x = narrow<S>(v.x);
                o.y = narrow<S>(v.y);
                out[outer * ps.out_so + inner * ps.out_si + (int64_t)e * ps.out_se] = o;
                continue;
            }
            double f = 1.0;
            if (ps.elem_scale) f *= ps.elem_scale[e];
            if (ps.line_scale) f *= ps.line_scale[outer * ps.nb_inner + inner];
            o.x = (S)(widen(v.x) * f);
            o.y = (S)(widen(v.y) * f);
            out[outer * ps.out_so + inner * ps.out_si + (int64_t)e * ps.out_se] = o;
        }
    }
}

// lines per tile: a power of two in [8, 64] with about 4096 elements per tile
int lines_per_tile(int N, int &lg) {
    lg = 3;
    while (lg < 6 && (1 << (lg + 1)) * N <= 4096) ++lg;
    return 1 << lg;
}

template <typename T, typename InC, typename OutC, int MODE>
cudaError_t run_pass(sgl_plan *p, FftPass ps, const void *in, void *out, ZetaSrc zs, int scale_on_output) {
    int lgTB = 0;
    const int TB = lines_per_tile(ps.N, lgTB);
    const size_t smem = (size_t)TB * (ps.N + 1) * sizeof(C2<T>);
    auto kern = k_fft_pass<T, InC, OutC, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = ps.nb_outer * ((ps.nb_inner + TB - 1) / TB);
    if (tiles <= 0) return cudaSuccess;
    kern<<<(unsigned)tiles, 256, smem, p->stream>>>(ps, TB, lgTB, (const InC *)in, (OutC *)out, zs, scale_on_output);
    p->launches += 1;
    return cudaGetLastError();
}

FftPass base_pass(const Axis &a, int sign, bool fp32) {
    FftPass ps{};
    ps.N = a.N;
    ps.nrad = a.nrad;
    for (int i = 0; i < a.nrad; ++i) ps.rad[i] = a.rad[i];
    ps.sign = sign;
    ps.tw = fp32 ? (const void *)a.tw_f : (const void *)a.tw_d;
    ps.rev = a.rev;
    return ps;
}

template <typename T>
cudaError_t forward_passes(sgl_plan *p) {
    const Axis &A0 = p->ax[0], &A1 = p->ax[1], &A2 = p->ax[2];
    constexpr bool f32 = std::is_same<T, float>::value;
    const int64_t W = 2 * p->K1 + 1;
    ZetaSrc zs{p->b.zeta, p->K0, p->K1};
    cudaError_t e;
    // pass A (axis 0): zeta (mirrored, deconvolved) -> X0[l0 row][k1][m]
    FftPass a = base_pass(A0, +1, f32);
    a.L_in = 2 * p->K0 + 1; a.in_first = -p->K0;
    a.L_out = A0.rows; a.out_first = A0.first;
    a.nb_outer = 1; a.nb_inner = W * W;
    a.out_so = 0; a.out_si = 1; a.out_se = W * W;
    a.elem_scale = A0.deconv; a.line_scale = p->b.linescale;
    if constexpr (f32) {
        a.tw = A0.tw_df;                          // radial pass in double-float (file comment)
        if ((e = run_pass<dfl, double2, C2<T>, LOAD_ZETA>(p, a, nullptr, p->b.bufA, zs, 0)) != cudaSuccess) return e;
    } else if ((e = run_pass<T, double2, C2<T>, LOAD_ZETA>(p, a, nullptr, p->b.bufA, zs, 0)) != cudaSuccess) {
        return e;
    }
    // pass B (axis 1): X0 -> X1[l0][l1 row][m]
    FftPass b = base_pass(A1, +1, f32);
    b.L_in = (int)W; b.in_first = -p->K1;
    b.L_out = A1.rows; b.out_first = A1.first;
    b.nb_outer = A0.rows; b.nb_inner = W;
    b.in_so = W * W; b.in_si = 1; b.in_se = W;
    b.out_so = (int64_t)A1.rows * W; b.out_si = 1; b.out_se = W;
    if ((e = run_pass<T, C2<T>, C2<T>, LOAD_STRIDED>(p, b, p->b.bufA, p->b.bufB, zs, 0)) != cudaSuccess) return e;
    // pass C (axis 2): X1 -> grid[l0][l1][l2], full lines
    FftPass c = base_pass(A2, +1, f32);
    c.L_in = (int)W; c.in_first = -p->K1;
    c.L_out = A2.N; c.out_first = 0;
    c.nb_outer = 1; c.nb_inner = (int64_t)A0.rows * A1.rows;
    c.in_so = 0; c.in_si = W; c.in_se = 1;
    c.out_so = 0; c.out_si = A2.N; c.out_se = 1;
    if (f32 && p->tc_interp) {                    // the tensor-core interpolation reads the planes only
        c.planes = p->b.planes;
        c.pitch = tc_pitch(A2.N);
        c.halo = tc_halo(p->q);
        c.plane_n = c.nb_inner * c.pitch;
    }
    return run_pass<T, C2<T>, C2<T>, LOAD_STRIDED>(p, c, p->b.bufB, p->b.bufA, zs, 0);
}

template <typename T>
cudaError_t adjoint_passes(sgl_plan *p) {
    const Axis &A0 = p->ax[0], &A1 = p->ax[1], &A2 = p->ax[2];
    constexpr bool f32 = std::is_same<T, float>::value;
    const int64_t W = 2 * p->K1 + 1;
    ZetaSrc zs{p->b.zeta, p->K0, p->K1};
    cudaError_t e;
    // pass C' (axis 2): grid -> Y1[l0][l1][m]
    FftPass c = base_pass(A2, -1, f32);
    c.L_in = A2.N; c.in_first = 0;
    c.L_out = (int)W; c.out_first = -p->K1;
    c.nb_outer = 1; c.nb_inner = (int64_t)A0.rows * A1.rows;
    c.in_so = 0; c.in_si = A2.N; c.in_se = 1;
    c.out_so = 0; c.out_si = W; c.out_se = 1;
    if ((e = run_pass<T, C2<T>, C2<T>, LOAD_STRIDED>(p, c, p->b.bufA, p->b.bufB, zs, 1)) != cudaSuccess) return e;
    // pass B' (axis 1): Y1 -> Y0[l0][k1][m]
    FftPass b = base_pass(A1, -1, f32);
    b.L_in = A1.rows; b.in_first = A1.first;
    b.L_out = (int)W; b.out_first = -p->K1;
    b.nb_outer = A0.rows; b.nb_inner = W;
    b.in_so = (int64_t)A1.rows * W; b.in_si = 1; b.in_se = W;
    b.out_so = W * W; b.out_si = 1; b.out_se = W;
    if ((e = run_pass<T, C2<T>, C2<T>, LOAD_STRIDED>(p, b, p->b.bufB, p->b.bufA, zs, 1)) != cudaSuccess) return e;
    // pass A' (axis 0): Y0 -> eta'[k0][k1][m] (FP64), deconvolved
    FftPass a = base_pass(A0, -1, f32);
    a.L_in = A0.rows; a.in_first = A0.first;
    a.L_out = 2 * p->K0 + 1; a.out_first = -p->K0;
    a.nb_outer = 1; a.nb_inner = W * W;
    a.in_so = 0; a.in_si = 1; a.in_se = W * W;
    a.out_so = 0; a.out_si = 1; a.out_se = W * W;
    a.elem_scale = A0.deconv; a.line_scale = p->b.linescale;
    if constexpr (f32) {
        a.tw = A0.tw_df;                          // radial pass in double-float (file comment)
        return run_pass<dfl, C2<T>, double2, LOAD_STRIDED>(p, a, p->b.bufA, p->b.bufB, zs, 1);
    }
    return run_pass<T, C2<T>, double2, LOAD_STRIDED>(p, a, p->b.bufA, p->b.bufB, zs, 1);
}

}  // namespace

cudaError_t launch_fft_forward(sgl_plan *p) {
    return p->prec == SGL_FP32_MIXED ? forward_passes<float>(p) : forward_passes<double>(p);
}

cudaError_t launch_fft_adjoint(sgl_plan *p) {
    return p->prec == SGL_FP32_MIXED ? adjoint_passes<float>(p) : adjoint_passes<double>(p);
}

}  // namespace sgl
