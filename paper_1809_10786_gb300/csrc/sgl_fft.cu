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
// binary32 spreading 2e-8 and 6e-8).  The forward's radial pass needs it too: its rounding error
// is set by the largest rows and lands on the outer radii as well, where the values are small and
// the gradient's chain rule divides by sin t0 (measured: in binary32 the values' error rose from
// 1.9e-7 to 1.0e-6 and the point gradient's from 4.4e-7 to 5.4e-5).
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

// 16 = 4 x 4: DFT-4 over n2 for each n1, twiddles W16^(n1 k2), DFT-4 over n1 for each k2; output
// index k2 + 4 k1
template <typename T>
__device__ __forceinline__ void dft16(C2<T> *x, int s) {
    constexpr T c1 = T(0.92387953251128675613), s1 = T(0.38268343236508977173), h = T(0.70710678118654752440);
    C2<T> y[4][4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
        C2<T> a[4] = {x[n1], x[n1 + 4], x[n1 + 8], x[n1 + 12]};
        dft4<T>(a, s);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) y[n1][k2] = a[k2];
    }
    // W16^j = e^{s 2 pi i j / 16}, j = n1 k2 in {1, 2, 3, 4, 6, 9}
    y[1][1] = mul<T>(y[1][1], mk<T>(c1, s * s1));
    y[1][2] = mul<T>(y[1][2], mk<T>(h, s * h));
    y[1][3] = mul<T>(y[1][3], mk<T>(s1, s * c1));
    y[2][1] = mul<T>(y[2][1], mk<T>(h, s * h));
    y[2][2] = mul_si<T>(y[2][2], s);
    y[2][3] = mul<T>(y[2][3], mk<T>(-h, s * h));
    y[3][1] = mul<T>(y[3][1], mk<T>(s1, s * c1));
    y[3][2] = mul<T>(y[3][2], mk<T>(-h, s * h));
    y[3][3] = mul<T>(y[3][3], mk<T>(-c1, -s * s1));
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
        C2<T> b[4] = {y[0][k2], y[1][k2], y[2][k2], y[3][k2]};
        dft4<T>(b, s);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) x[k2 + 4 * k1] = b[k1];
    }
}

enum { LOAD_STRIDED = 0, LOAD_ZETA = 1 };

struct ZetaSrc {
    const double2 *zeta;   // [K0+1][K1+1][2K1+1]
    int K0, K1;
    int half;              // lines (kappa1 >= 0, m) only: inner = kappa1 (2K1+1) + m + K1
};

template <typename C> __device__ __forceinline__ double2 to_d2(C v) { return make_double2((double)v.x, (double)v.y); }

template <typename T, int R>
__device__ __forceinline__ void dft_r(C2<T> *x, int s) {
    if constexpr (R == 2) dft2<T>(x);
    else if constexpr (R == 3) dft3<T>(x, s);
    else if constexpr (R == 4) dft4<T>(x, s);
    else if constexpr (R == 5) dft5<T>(x, s);
    else if constexpr (R == 8) dft8<T>(x, s);
    else dft16<T>(x, s);
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
                    const int k1 = (int)(inner / W) - (zs.half ? 0 : zs.K1);
                    const int k0 = e - zs.K0;
                    d = zs.zeta[((int64_t)abs(k0) * (zs.K1 + 1) + abs(k1)) * W + mi];
                    if (k1 < 0 && ((mi - zs.K1) & 1)) { d.x = -d.x; d.y = -d.y; }
                } else {
                    // element e at |e - mir_c| (plain lines: mir_c = 0), with the polar parity below mir_c
                    const int k = e - ps.mir_c;
                    const int64_t at = outer * ps.in_so + inner * ps.in_si + (int64_t)abs(k) * ps.in_se;
                    const bool neg = k < 0 && ((inner - ps.mir_c) & 1);
                    if (scale_on_output || (!ps.elem_scale && !ps.line_scale)) {
                        // no factor on the input: straight conversion to the pass arithmetic
                        const InC x = in[at];
                        v[u] = neg ? mk<T>(-T(x.x), -T(x.y)) : mk<T>(T(x.x), T(x.y));
                        continue;
                    }
                    d = to_d2(in[at]);
                    if (neg) { d.x = -d.x; d.y = -d.y; }
                }
                if (!scale_on_output) {
                    double f = 1.0;
                    if (ps.elem_scale) f *= ps.elem_scale[e];
                    if (ps.line_scale) f *= ps.line_scale[outer * ps.nb_inner + inner + ps.ls_off];
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
                float *row = ps.planes + (outer * ps.plane_so + inner0 + bl + ps.plane_off) * ps.pitch;
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
            if (ps.line_scale) f *= ps.line_scale[outer * ps.nb_inner + inner + ps.ls_off];
            o.x = (S)(widen(v.x) * f);
            o.y = (S)(widen(v.y) * f);
            out[outer * ps.out_so + inner * ps.out_si + (int64_t)e * ps.out_se] = o;
        }
    }
}

// ---------------------------------------------------------------- register Stockham passes
// Power-of-two lengths N = R1 R2 (R3): each thread holds E = max radix elements of one line and
// TPL = N / E threads share a line (TB = 256 / TPL lines per CTA).  Stage j (radix R, L = product
// of the earlier radices, M = N / L, Q = M / R) takes butterflies b = (c, n1) = (b mod L, b / L):
// z_k = W_M^(n1 k) sum_{n2 < R} y_c[n1 + Q n2] W_R^(n2 k), which is y_{c + L k}[n1] of the next
// stage (Stockham autosort: input and output in natural order).  The first stage reads its
// elements straight from global memory, the last one writes them there; between stages the line
// goes through shared memory once (index i stored at i + i / E: no bank conflicts on the stride-E
// writes).  Thread t takes butterflies t + TPL i of every stage.
template <int N, int R1, int R2, int R3>
struct RegFft {
    static constexpr int E = R1 > R2 ? (R1 > R3 ? R1 : R3) : (R2 > R3 ? R2 : R3);
    static constexpr int TPL = N / E;
    static constexpr int TB = 256 / TPL;
    static constexpr int LS = (N + N / E) | 1;          // odd line stride (64-bit words) in shared memory
    static_assert(R1 * R2 * R3 == N && E % R1 == 0 && E % R2 == 0 && E % R3 == 0 && TPL <= 256, "radices");
};

__device__ __forceinline__ int pad_e(int i, int E) { return i + i / E; }

// load: FFT position pos of a line holds input element e = (pos - in_first) mod N (zero if e >= L_in)
template <typename T, typename InC, int MODE>
__device__ __forceinline__ C2<T> reg_load(const FftPass &ps, const InC *__restrict__ in, const ZetaSrc &zs, int64_t outer,
                                          int64_t inner, bool valid, int e, int scale_on_output, int E) {
    if (!valid || e >= ps.L_in) return mk<T>(T(0), T(0));
    C2<T> v;
    if constexpr (MODE == LOAD_ZETA) {
        const int W = 2 * zs.K1 + 1;
        const int mi = (int)(inner % W);
        const int k1 = (int)(inner / W) - (zs.half ? 0 : zs.K1);
        const int k0 = e - zs.K0;
        double2 d = zs.zeta[((int64_t)abs(k0) * (zs.K1 + 1) + abs(k1)) * W + mi];
        if (k1 < 0 && ((mi - zs.K1) & 1)) { d.x = -d.x; d.y = -d.y; }
        if constexpr (std::is_same<T, dfl>::value) { v.x = df_split_bits(d.x, E); v.y = df_split_bits(d.y, E); }
        else { v.x = T(d.x); v.y = T(d.y); }
    } else {
        // element e at |e - mir_c| (plain lines: mir_c = 0), with the polar parity below mir_c
        const int k = e - ps.mir_c;
        InC x = in[outer * ps.in_so + inner * ps.in_si + (int64_t)abs(k) * ps.in_se];
        if (k < 0 && ((inner - ps.mir_c) & 1)) { x.x = -x.x; x.y = -x.y; }
        if constexpr (std::is_same<T, dfl>::value && sizeof(x.x) == 8) { v.x = df_split_bits(x.x, E); v.y = df_split_bits(x.y, E); }
        else { v.x = T(x.x); v.y = T(x.y); }
    }
    if (!scale_on_output && (ps.elem_scale || ps.line_scale)) {
        if constexpr (std::is_same<T, dfl>::value) {
            dfl f(1.f, 0.f);
            if (ps.elem_scale_df) f = dfl(ps.elem_scale_df[e].x, ps.elem_scale_df[e].y);
            if (ps.line_scale_df) {
                const float2 l = ps.line_scale_df[outer * ps.nb_inner + inner + ps.ls_off];
                f = f * dfl(l.x, l.y);
            }
            v.x = v.x * f; v.y = v.y * f;
        } else {
            double f = 1.0;
            if (ps.elem_scale) f *= ps.elem_scale[e];
            if (ps.line_scale) f *= ps.line_scale[outer * ps.nb_inner + inner + ps.ls_off];
            v.x = T(widen(v.x) * f); v.y = T(widen(v.y) * f);
        }
    }
    return v;
}

// store output element e (position (e + out_first) mod N), optional scale on output
template <typename T, typename OutC>
__device__ __forceinline__ void reg_store(const FftPass &ps, OutC *__restrict__ out, int64_t outer, int64_t inner, int e, C2<T> v,
                                          int scale_on_output, int E) {
    using S = decltype(OutC::x);
    OutC o;
    if (scale_on_output && (ps.elem_scale || ps.line_scale)) {
        if constexpr (std::is_same<T, dfl>::value) {
            dfl f(1.f, 0.f);
            if (ps.elem_scale_df) f = dfl(ps.elem_scale_df[e].x, ps.elem_scale_df[e].y);
            if (ps.line_scale_df) {
                const float2 l = ps.line_scale_df[outer * ps.nb_inner + inner + ps.ls_off];
                f = f * dfl(l.x, l.y);
            }
            v.x = v.x * f; v.y = v.y * f;
        } else {
            double f = 1.0;
            if (ps.elem_scale) f *= ps.elem_scale[e];
            if (ps.line_scale) f *= ps.line_scale[outer * ps.nb_inner + inner + ps.ls_off];
            o.x = (S)(widen(v.x) * f);
            o.y = (S)(widen(v.y) * f);
            out[outer * ps.out_so + inner * ps.out_si + (int64_t)e * ps.out_se] = o;
            return;
        }
    }
    if constexpr (std::is_same<T, dfl>::value && sizeof(S) == 8) {
        o.x = df_to_double_scaled(v.x, E);
        o.y = df_to_double_scaled(v.y, E);
    } else {
        o.x = narrow<S>(v.x);
        o.y = narrow<S>(v.y);
    }
    out[outer * ps.out_so + inner * ps.out_si + (int64_t)e * ps.out_se] = o;
}

// one stage on the registers: E / R butterflies of radix R, then the twiddles W_M^(n1 k)
template <typename T, int N, int E, int TPL, int R, int L>
__device__ __forceinline__ void reg_stage(C2<T> *v, int t, int sign, const C2<T> *__restrict__ tw) {
#pragma unroll
    for (int i = 0; i < E / R; ++i) {
        dft_r<T, R>(v + i * R, sign);
        if constexpr (L * R < N) {                                 // not the last stage (there n1 = 0)
            const int n1 = (t + TPL * i) / L;
#pragma unroll
            for (int k = 1; k < R; ++k) {
                C2<T> w = tw[L * n1 * k];                          // W_M^(n1 k) = W_N^(L n1 k), L n1 k < N
                if (sign < 0) w.y = -w.y;
                v[i * R + k] = mul<T>(v[i * R + k], w);
            }
        }
    }
}

// stage outputs -> shared memory (new layout c + L' n, L' = L R) -> the next stage's inputs
template <typename T, int N, int E, int TPL, int R, int L, int RN>
__device__ __forceinline__ void reg_exchange(C2<T> *v, C2<T> *line, int t) {
#pragma unroll
    for (int i = 0; i < E / R; ++i) {
        const int b = t + TPL * i, c = b % L, n1 = b / L;
#pragma unroll
        for (int k = 0; k < R; ++k) line[pad_e(c + L * k + L * R * n1, E)] = v[i * R + k];
    }
    __syncthreads();
    constexpr int L2 = L * R, Q2 = N / L2 / RN;
#pragma unroll
    for (int i = 0; i < E / RN; ++i) {
        const int b = t + TPL * i, c = b % L2, n1 = b / L2;
#pragma unroll
        for (int n2 = 0; n2 < RN; ++n2) v[i * RN + n2] = line[pad_e(c + L2 * (n1 + Q2 * n2), E)];
    }
    __syncthreads();
}

template <typename T, typename InC, typename OutC, int MODE, int N, int R1, int R2, int R3>
__global__ void __launch_bounds__(256) k_fft_reg(FftPass ps, const InC *__restrict__ in, OutC *__restrict__ out, ZetaSrc zs,
                                                 int scale_on_output, int line_fast) {
    using G = RegFft<N, R1, R2, R3>;
    constexpr int E = G::E, TPL = G::TPL, TB = G::TB;
    extern __shared__ unsigned char smem_raw[];
    C2<T> *sbuf = reinterpret_cast<C2<T> *>(smem_raw);       // [TB][LS]
    const int64_t tiles_inner = (ps.nb_inner + TB - 1) / TB;
    const int64_t outer = blockIdx.x / tiles_inner;
    const int64_t inner0 = (blockIdx.x % tiles_inner) * TB;
    const int tid = threadIdx.x;
    const int bl = line_fast ? tid % TB : tid / TPL;
    const int t = line_fast ? tid / TB : tid % TPL;
    const int64_t inner = inner0 + bl;
    const bool valid = inner < ps.nb_inner;
    C2<T> *line = sbuf + bl * G::LS;
    const C2<T> *tw = reinterpret_cast<const C2<T> *>(ps.tw);
    const int SE = df_scale_exponent(ps.scale_bits);              // 0 unless binary64 data in double-float

    // stage 1 inputs: butterfly b = n1 (L = 1) reads positions n1 + (N / R1) n2
    C2<T> v[E];
#pragma unroll
    for (int i = 0; i < E / R1; ++i) {
        const int n1 = t + TPL * i;
#pragma unroll
        for (int n2 = 0; n2 < R1; ++n2) {
            int e = n1 + (N / R1) * n2 - ps.in_first;
            e = e >= N ? e - N : (e < 0 ? e + N : e);
            v[i * R1 + n2] = reg_load<T, InC, MODE>(ps, in, zs, outer, inner, valid, e, scale_on_output, SE);
        }
    }
    reg_stage<T, N, E, TPL, R1, 1>(v, t, ps.sign, tw);
    reg_exchange<T, N, E, TPL, R1, 1, R2>(v, line, t);
    reg_stage<T, N, E, TPL, R2, R1>(v, t, ps.sign, tw);
    constexpr int RL = R3 > 1 ? R3 : R2, LL = N / RL;              // last stage: radix, L
    if constexpr (R3 > 1) {
        reg_exchange<T, N, E, TPL, R2, R1, R3>(v, line, t);
        reg_stage<T, N, E, TPL, R3, R1 * R2>(v, t, ps.sign, tw);
    }

    // last stage outputs: butterfly b = c (n1 = 0) holds positions c + LL k
    if constexpr (std::is_same<OutC, float2>::value) {
        if (ps.planes) {                                           // split planes with a wrapped halo
            if (!valid) return;
            float *row = ps.planes + (outer * ps.plane_so + inner + ps.plane_off) * ps.pitch;
#pragma unroll
            for (int i = 0; i < E / RL; ++i) {
#pragma unroll
                for (int k = 0; k < RL; ++k) {
                    const int pos = t + TPL * i + LL * k;
                    const float re = narrow<float>(v[i * RL + k].x), im = narrow<float>(v[i * RL + k].y);
                    int col = pos + ps.halo;                       // < pitch: pitch >= N + 32, halo <= 8
                    row[col] = re; row[ps.plane_n + col] = im;
                    col = pos + ps.halo + N;
                    if (col < ps.pitch) { row[col] = re; row[ps.plane_n + col] = im; }
                    col = pos + ps.halo - N;
                    if (col >= 0) { row[col] = re; row[ps.plane_n + col] = im; }
                }
            }
            return;
        }
    }
    if (!valid) return;
#pragma unroll
    for (int i = 0; i < E / RL; ++i) {
#pragma unroll
        for (int k = 0; k < RL; ++k) {
            const int pos = t + TPL * i + LL * k;
            int e = pos - ps.out_first;
            e = e >= N ? e - N : (e < 0 ? e + N : e);
            if (e < ps.L_out) reg_store<T, OutC>(ps, out, outer, inner, e, v[i * RL + k], scale_on_output, SE);
        }
    }
}

// ---------------------------------------------------------------- symmetry-reduced grid
// eta is even in kappa0 and has the parity of m in kappa1 (Sect. 6), so the oversampled grid of the
// NFFT is even in l0 and alpha(l0, -l1, l2) = alpha(l0, l1, l2 + N2/2).  Plans whose axes 0 and 1
// are windowed transform half of the lines: pass A
// the radial lines kappa1 >= 0 (pass B reads kappa1 < 0 back through the parity), passes B and C the
// grid lines (l0, l1) in [0, N0/2] x [0, N1/2].  The q halo rows on each side of the two windowed axes
// are then copies of the rows they mirror: row -l (1 <= l <= q) and row N - l (N/2 - q <= l < N/2)
// hold line l, shifted by N2/2 on axis 1.  The adjoint first adds every halo row onto the row it
// mirrors, transforms the same half, folds kappa1 < 0 onto kappa1 >= 0 (parity) before pass A', and
// folds kappa0 < 0 onto kappa0 >= 0 after it (sgl_convert.cu).  Both FFT kernels (register and
// generic) read the mirrored lines and write the plane rows of the reduced layout.
struct HaloGeom {
    int q, N0h, N1h, R1, N2;    // q, N0/2, N1/2, rows kept on axis 1, azimuthal length (even)
};

// storage row (first row -q) -> the grid line l in [0, N/2] it holds, and whether it is a mirror
__device__ __forceinline__ int halo_source(int r, int q, int Nh) {
    const int l = r - q;
    return l < 0 ? -l : (l > Nh ? 2 * Nh - l : l);
}

// the halo rows, enumerated: axis-0 halo rows (2q) x all rows of axis 1, then the rows of axis 0
// inside [0, N0/2] x the axis-1 halo rows (2q)
__device__ __forceinline__ void halo_row(int64_t idx, const HaloGeom &h, int &a, int &b) {
    const int q2 = 2 * h.q;
    if (idx < (int64_t)q2 * h.R1) {
        const int ai = (int)(idx / h.R1);
        b = (int)(idx - (int64_t)ai * h.R1);
        a = ai < h.q ? ai : h.N0h + h.q + 1 + (ai - h.q);
    } else {
        const int64_t j = idx - (int64_t)q2 * h.R1;
        a = h.q + (int)(j / q2);
        const int bi = (int)(j % q2);
        b = bi < h.q ? bi : h.N1h + h.q + 1 + (bi - h.q);
    }
}
inline int64_t halo_rows(const HaloGeom &h) { return (int64_t)2 * h.q * h.R1 + (int64_t)(h.N0h + 1) * 2 * h.q; }

// forward: every halo row (blockIdx.x) copied from the row it mirrors
template <typename C>
__global__ void __launch_bounds__(256) k_halo_mirror(HaloGeom h, C *__restrict__ grid) {
    int a, b;
    halo_row(blockIdx.x, h, a, b);
    const int l0 = halo_source(a, h.q, h.N0h), l1 = halo_source(b, h.q, h.N1h);
    const int sh = (b - h.q < 0 || b - h.q > h.N1h) ? h.N2 / 2 : 0;
    const C *src = grid + ((int64_t)(l0 + h.q) * h.R1 + l1 + h.q) * h.N2;
    C *dst = grid + ((int64_t)a * h.R1 + b) * h.N2;
    for (int c = threadIdx.x; c < h.N2; c += blockDim.x) dst[c] = src[c + sh < h.N2 ? c + sh : c + sh - h.N2];
}

// the same on the tensor-core planes (Re, Im; column k holds position (k - halo) mod N2)
__global__ void __launch_bounds__(256) k_halo_mirror_planes(HaloGeom h, float *__restrict__ planes, int64_t plane_n, int pitch,
                                                            int halo) {
    int a, b;
    halo_row(blockIdx.x, h, a, b);
    const int l0 = halo_source(a, h.q, h.N0h), l1 = halo_source(b, h.q, h.N1h);
    const int sh = (b - h.q < 0 || b - h.q > h.N1h) ? h.N2 / 2 : 0;
    const float *src = planes + ((int64_t)(l0 + h.q) * h.R1 + l1 + h.q) * pitch;
    float *dst = planes + ((int64_t)a * h.R1 + b) * pitch;
    for (int k = threadIdx.x; k < pitch; k += blockDim.x) {
        const int pos = (k - halo + sh + h.N2) % h.N2;         // k - halo >= -halo > -N2
        dst[k] = src[pos + halo];
        dst[plane_n + k] = src[plane_n + pos + halo];
    }
}

// adjoint of the mirrors: every halo row (blockIdx.x) added onto the row it mirrors.  Each row
// with mirrors gathers them itself (one block per line (l0, l1) that has any), so no two blocks
// write one row.
__device__ __forceinline__ int halo_mirror_row(int l, int q, int Nh) {
    if (l >= 1 && l <= q) return q - l;
    if (l >= Nh - q && l < Nh) return 2 * Nh - l + q;
    return -1;
}
template <typename C>
__global__ void __launch_bounds__(256) k_halo_fold(HaloGeom h, C *__restrict__ grid) {
    // lines with an axis-0 mirror (2q values of l0) x all l1, then the other l0 x the 2q l1 with a mirror
    const int q2 = 2 * h.q, H1 = h.N1h + 1;
    const int64_t idx = blockIdx.x;
    int l0, l1;
    if (idx < (int64_t)q2 * H1) {
        const int li = (int)(idx / H1);
        l1 = (int)(idx - (int64_t)li * H1);
        l0 = li < h.q ? 1 + li : h.N0h - h.q + (li - h.q);
    } else {
        const int64_t j = idx - (int64_t)q2 * H1;
        const int li = (int)(j / q2), bi = (int)(j % q2);
        l0 = li == 0 ? 0 : (li <= h.N0h - q2 - 1 ? h.q + li : h.N0h);
        l1 = bi < h.q ? 1 + bi : h.N1h - h.q + (bi - h.q);
    }
    const int m0 = halo_mirror_row(l0, h.q, h.N0h), m1 = halo_mirror_row(l1, h.q, h.N1h);
    const int64_t r0 = l0 + h.q, r1 = l1 + h.q;
    C *dst = grid + (r0 * h.R1 + r1) * h.N2;
    const C *s0 = m0 >= 0 ? grid + ((int64_t)m0 * h.R1 + r1) * h.N2 : nullptr;
    const C *s1 = m1 >= 0 ? grid + (r0 * h.R1 + m1) * h.N2 : nullptr;
    const C *s01 = (m0 >= 0 && m1 >= 0) ? grid + ((int64_t)m0 * h.R1 + m1) * h.N2 : nullptr;
    for (int c = threadIdx.x; c < h.N2; c += blockDim.x) {
        const int cs = c + h.N2 / 2 < h.N2 ? c + h.N2 / 2 : c - h.N2 / 2;
        C v = dst[c];
        if (s0) { const C w = s0[c]; v.x += w.x; v.y += w.y; }
        if (s1) { const C w = s1[cs]; v.x += w.x; v.y += w.y; }
        if (s01) { const C w = s01[cs]; v.x += w.x; v.y += w.y; }
        dst[c] = v;
    }
}
inline int64_t halo_fold_rows(const HaloGeom &h) { return (int64_t)2 * h.q * (h.N1h + 1) + (int64_t)(h.N0h + 1 - 2 * h.q) * 2 * h.q; }

// adjoint of the polar parity: Yh[l0][k][m] = Y[l0][K1 + k][m] + (-1)^m Y[l0][K1 - k][m] (k > 0)
template <typename C>
__global__ void __launch_bounds__(256) k_fold_kappa1(int64_t H0, int K1, const C *__restrict__ Y, C *__restrict__ Yh) {
    const int W = 2 * K1 + 1;
    const int64_t total = H0 * (K1 + 1) * W;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int mi = (int)(i % W);
    const int k = (int)((i / W) % (K1 + 1));
    const int64_t l0 = i / ((int64_t)W * (K1 + 1));
    const C *row = Y + l0 * W * W;
    C v = row[(K1 + k) * W + mi];
    if (k > 0) {
        const C w = row[(K1 - k) * W + mi];
        const bool neg = (mi - K1) & 1;
        v.x += neg ? -w.x : w.x;
        v.y += neg ? -w.y : w.y;
    }
    Yh[i] = v;
}

// lines per tile: a power of two in [8, 64] with about 4096 elements per tile
int lines_per_tile(int N, int &lg) {
    lg = 3;
    while (lg < 6 && (1 << (lg + 1)) * N <= 4096) ++lg;
    return 1 << lg;
}

template <typename T, typename InC, typename OutC, int MODE, int N, int R1, int R2, int R3>
cudaError_t run_reg(sgl_plan *p, const FftPass &ps, const void *in, void *out, ZetaSrc zs, int scale_on_output) {
    using G = RegFft<N, R1, R2, R3>;
    const size_t smem = (size_t)G::TB * G::LS * sizeof(C2<T>);
    auto kern = k_fft_reg<T, InC, OutC, MODE, N, R1, R2, R3>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t tiles = ps.nb_outer * ((ps.nb_inner + G::TB - 1) / G::TB);
    if (tiles <= 0) return cudaSuccess;
    // threads of a line adjacent when its elements are adjacent in memory, else lines adjacent
    const int line_fast = (MODE == LOAD_ZETA || ps.in_se != 1) ? 1 : 0;
    kern<<<(unsigned)tiles, 256, smem, p->stream>>>(ps, (const InC *)in, (OutC *)out, zs, scale_on_output, line_fast);
    p->launches += 1;
    return cudaGetLastError();
}

template <typename T, typename InC, typename OutC, int MODE>
cudaError_t run_pass(sgl_plan *p, FftPass ps, const void *in, void *out, ZetaSrc zs, int scale_on_output) {
    if (!(p->flags & SGL_FLAG_GENERIC_FFT)) {
        switch (ps.N) {
            case 64: return run_reg<T, InC, OutC, MODE, 64, 8, 8, 1>(p, ps, in, out, zs, scale_on_output);
            case 128: return run_reg<T, InC, OutC, MODE, 128, 16, 8, 1>(p, ps, in, out, zs, scale_on_output);
            case 256: return run_reg<T, InC, OutC, MODE, 256, 16, 16, 1>(p, ps, in, out, zs, scale_on_output);
            case 512: return run_reg<T, InC, OutC, MODE, 512, 8, 8, 8>(p, ps, in, out, zs, scale_on_output);
            case 1024: return run_reg<T, InC, OutC, MODE, 1024, 16, 8, 8>(p, ps, in, out, zs, scale_on_output);
            default: break;
        }
    }
    if constexpr (std::is_same<T, dfl>::value && std::is_same<InC, double2>::value && std::is_same<OutC, double2>::value) {
        // binary64 data of other lengths: the generic kernel in binary64 (it keeps the full range)
        ps.tw = ps.tw64;
        ps.scale_bits = nullptr;
        return run_pass<double, InC, OutC, MODE>(p, ps, in, out, zs, scale_on_output);
    } else {
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
}

FftPass base_pass(const Axis &a, int sign, bool fp32) {
    FftPass ps{};
    ps.N = a.N;
    ps.nrad = a.nrad;
    for (int i = 0; i < a.nrad; ++i) ps.rad[i] = a.rad[i];
    ps.sign = sign;
    ps.tw = fp32 ? (const void *)a.tw_f : (const void *)a.tw_d;
    ps.tw64 = a.tw_d;
    ps.rev = a.rev;
    return ps;
}

// the twiddle table of an axis in the pass arithmetic AR
template <typename AR> const void *twiddles(const Axis &a) {
    if constexpr (std::is_same<AR, dfl>::value) return a.tw_df;
    else if constexpr (std::is_same<AR, float>::value) return a.tw_f;
    else return a.tw_d;
}

// Storage T (float2 / double2 work buffers) and the arithmetic of the passes: FP32-mixed plans run
// the radial passes in double-float (RA = dfl) and the angular ones in binary32 (AA = float); FP64
// plans run all three in double-float (RA = AA = dfl, the default) or in binary64
// (SGL_FLAG_NATIVE_FP64).
template <typename T, typename RA, typename AA>
cudaError_t forward_passes(sgl_plan *p) {
    const Axis &A0 = p->ax[0], &A1 = p->ax[1], &A2 = p->ax[2];
    constexpr bool f32 = std::is_same<T, float>::value;
    const int64_t W = 2 * p->K1 + 1;
    ZetaSrc zs{p->b.zeta, p->K0, p->K1};
    cudaError_t e;
    // binary64 data in double-float passes: one power-of-two scale for all three, from max |zeta|
    constexpr bool scaled = !f32 && std::is_same<RA, dfl>::value;
    const unsigned long long *sb = scaled ? p->b.df_max + 2 : nullptr;
    if (scaled &&
        (e = launch_max_abs(p, (const double *)p->b.zeta, 2 * (int64_t)(p->K0 + 1) * (p->K1 + 1) * W, p->b.df_max + 2)) != cudaSuccess)
        return e;
    // symmetry-reduced grid: half of the lines on axes 0 and 1, then the halo rows by mirroring
    const bool half = p->half_grid;
    const int H0 = A0.N / 2 + 1, H1 = A1.N / 2 + 1;
    const int64_t K1p = p->K1 + 1, k1_lines = half ? K1p : W;   // kappa1 lines of pass A
    const int64_t interior = ((int64_t)p->q * A1.rows + p->q) * A2.N;   // grid offset of line (0, 0)
    zs.half = half ? 1 : 0;
    // pass A (axis 0): zeta (mirrored, deconvolved) -> X0[l0 row][k1][m]
    FftPass a = base_pass(A0, +1, f32);
    a.scale_bits = sb;
    a.tw = twiddles<RA>(A0);
    a.L_in = 2 * p->K0 + 1; a.in_first = -p->K0;
    a.L_out = half ? H0 : A0.rows; a.out_first = half ? 0 : A0.first;
    a.nb_outer = 1; a.nb_inner = k1_lines * W;
    a.out_so = 0; a.out_si = 1; a.out_se = k1_lines * W;
    a.elem_scale = A0.deconv; a.line_scale = p->b.linescale;
    a.elem_scale_df = A0.deconv_df; a.line_scale_df = p->b.linescale_df;
    a.ls_off = half ? p->K1 * W : 0;
    if ((e = run_pass<RA, double2, C2<T>, LOAD_ZETA>(p, a, nullptr, p->b.bufA, zs, 0)) != cudaSuccess) return e;
    // pass B (axis 1): X0 -> X1[l0][l1 row][m] (reduced: kappa1 < 0 read through the polar parity)
    FftPass b = base_pass(A1, +1, f32);
    b.tw = twiddles<AA>(A1);
    b.scale_bits = sb;
    b.L_in = (int)W; b.in_first = -p->K1;
    b.L_out = half ? H1 : A1.rows; b.out_first = half ? 0 : A1.first;
    b.nb_outer = half ? H0 : A0.rows; b.nb_inner = W;
    b.in_so = k1_lines * W; b.in_si = 1; b.in_se = W;
    b.out_so = (int64_t)b.L_out * W; b.out_si = 1; b.out_se = W;
    b.mir_c = half ? p->K1 : 0;
    if ((e = run_pass<AA, C2<T>, C2<T>, LOAD_STRIDED>(p, b, p->b.bufA, p->b.bufB, zs, 0)) != cudaSuccess) return e;
    // pass C (axis 2): X1 -> grid[l0][l1][l2], full lines (reduced: the lines of [0, N0/2] x [0, N1/2])
    FftPass c = base_pass(A2, +1, f32);
    c.tw = twiddles<AA>(A2);
    c.scale_bits = sb;
    c.L_in = (int)W; c.in_first = -p->K1;
    c.L_out = A2.N; c.out_first = 0;
    if (half) {
        c.nb_outer = H0; c.nb_inner = H1;
        c.in_so = (int64_t)H1 * W; c.in_si = W; c.in_se = 1;
        c.out_so = (int64_t)A1.rows * A2.N; c.out_si = A2.N; c.out_se = 1;
    } else {
        c.nb_outer = 1; c.nb_inner = (int64_t)A0.rows * A1.rows;
        c.in_so = 0; c.in_si = W; c.in_se = 1;
        c.out_so = 0; c.out_si = A2.N; c.out_se = 1;
    }
    const bool planes = f32 && p->tc_interp;      // the tensor-core interpolation reads the planes only
    if (planes) {
        c.planes = p->b.planes;
        c.pitch = tc_pitch(A2.N);
        c.halo = tc_halo(p->q);
        c.plane_n = (int64_t)A0.rows * A1.rows * c.pitch;
        if (half) { c.plane_so = A1.rows; c.plane_off = (int64_t)p->q * A1.rows + p->q; }
    }
    if ((e = run_pass<AA, C2<T>, C2<T>, LOAD_STRIDED>(p, c, p->b.bufB, (C2<T> *)p->b.bufA + (half ? interior : 0), zs, 0)) !=
        cudaSuccess)
        return e;
    if (!half) return cudaSuccess;
    const HaloGeom h{p->q, A0.N / 2, A1.N / 2, A1.rows, A2.N};
    if (planes) k_halo_mirror_planes<<<(unsigned)halo_rows(h), 128, 0, p->stream>>>(h, c.planes, c.plane_n, c.pitch, c.halo);
    else k_halo_mirror<C2<T>><<<(unsigned)halo_rows(h), 128, 0, p->stream>>>(h, (C2<T> *)p->b.bufA);
    p->launches += 1;
    return cudaGetLastError();
}

template <typename T, typename RA, typename AA>
cudaError_t adjoint_passes(sgl_plan *p) {
    const Axis &A0 = p->ax[0], &A1 = p->ax[1], &A2 = p->ax[2];
    constexpr bool f32 = std::is_same<T, float>::value;
    const int64_t W = 2 * p->K1 + 1;
    ZetaSrc zs{p->b.zeta, p->K0, p->K1};
    cudaError_t e;
    // binary64 data in double-float passes: one power-of-two scale for all three, from max |grid|
    constexpr bool scaled = !f32 && std::is_same<RA, dfl>::value;
    const unsigned long long *sb = scaled ? p->b.df_max + 2 : nullptr;
    // symmetry-reduced grid: the halo rows folded onto the rows they mirror, half of the lines on
    // axes 1 and 0, kappa1 < 0 folded onto kappa1 >= 0 between them; eta'[k0][k1 >= 0][m] in bufA
    const bool half = p->half_grid;
    const int H0 = A0.N / 2 + 1, H1 = A1.N / 2 + 1;
    const int64_t K1p = p->K1 + 1, k1_lines = half ? K1p : W;
    const int64_t interior = ((int64_t)p->q * A1.rows + p->q) * A2.N;
    if (half) {
        const HaloGeom h{p->q, A0.N / 2, A1.N / 2, A1.rows, A2.N};
        k_halo_fold<C2<T>><<<(unsigned)halo_fold_rows(h), 128, 0, p->stream>>>(h, (C2<T> *)p->b.bufA);
        p->launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (scaled && (e = launch_max_abs(p, (const double *)p->b.bufA, 2 * (int64_t)A0.rows * A1.rows * A2.N, p->b.df_max + 2)) !=
                      cudaSuccess)
        return e;
    // pass C' (axis 2): grid -> Y1[l0][l1][m]
    FftPass c = base_pass(A2, -1, f32);
    c.tw = twiddles<AA>(A2);
    c.scale_bits = sb;
    c.L_in = A2.N; c.in_first = 0;
    c.L_out = (int)W; c.out_first = -p->K1;
    if (half) {
        c.nb_outer = H0; c.nb_inner = H1;
        c.in_so = (int64_t)A1.rows * A2.N; c.in_si = A2.N; c.in_se = 1;
        c.out_so = (int64_t)H1 * W; c.out_si = W; c.out_se = 1;
    } else {
        c.nb_outer = 1; c.nb_inner = (int64_t)A0.rows * A1.rows;
        c.in_so = 0; c.in_si = A2.N; c.in_se = 1;
        c.out_so = 0; c.out_si = W; c.out_se = 1;
    }
    if ((e = run_pass<AA, C2<T>, C2<T>, LOAD_STRIDED>(p, c, (const C2<T> *)p->b.bufA + (half ? interior : 0), p->b.bufB, zs, 1)) !=
        cudaSuccess)
        return e;
    // pass B' (axis 1): Y1 -> Y0[l0][k1][m]
    FftPass b = base_pass(A1, -1, f32);
    b.tw = twiddles<AA>(A1);
    b.scale_bits = sb;
    b.L_in = half ? H1 : A1.rows; b.in_first = half ? 0 : A1.first;
    b.L_out = (int)W; b.out_first = -p->K1;
    b.nb_outer = half ? H0 : A0.rows; b.nb_inner = W;
    b.in_so = (int64_t)b.L_in * W; b.in_si = 1; b.in_se = W;
    b.out_so = W * W; b.out_si = 1; b.out_se = W;
    if ((e = run_pass<AA, C2<T>, C2<T>, LOAD_STRIDED>(p, b, p->b.bufB, p->b.bufA, zs, 1)) != cudaSuccess) return e;
    const void *y0 = p->b.bufA;
    if (half) {                                   // Y0 -> Y0h[l0][k1 >= 0][m] (bufB)
        const int64_t n = (int64_t)H0 * K1p * W;
        k_fold_kappa1<C2<T>><<<(unsigned)((n + 255) / 256), 256, 0, p->stream>>>(H0, p->K1, (const C2<T> *)p->b.bufA,
                                                                                   (C2<T> *)p->b.bufB);
        p->launches += 1;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        y0 = p->b.bufB;
    }
    // pass A' (axis 0): Y0 -> eta'[k0][k1][m] (FP64), deconvolved (bufB; reduced: k1 >= 0, bufA)
    FftPass a = base_pass(A0, -1, f32);
    a.tw = twiddles<RA>(A0);
    a.scale_bits = sb;
    a.L_in = half ? H0 : A0.rows; a.in_first = half ? 0 : A0.first;
    a.L_out = 2 * p->K0 + 1; a.out_first = -p->K0;
    a.nb_outer = 1; a.nb_inner = k1_lines * W;
    a.in_so = 0; a.in_si = 1; a.in_se = k1_lines * W;
    a.out_so = 0; a.out_si = 1; a.out_se = k1_lines * W;
    a.elem_scale = A0.deconv; a.line_scale = p->b.linescale;
    a.elem_scale_df = A0.deconv_df; a.line_scale_df = p->b.linescale_df;
    a.ls_off = half ? p->K1 * W : 0;
    return run_pass<RA, C2<T>, double2, LOAD_STRIDED>(p, a, y0, half ? p->b.bufA : p->b.bufB, zs, 1);
}

}  // namespace

cudaError_t launch_fft_forward(sgl_plan *p) {
    if (p->prec == SGL_FP32_MIXED) return forward_passes<float, dfl, float>(p);
    if (p->flags & SGL_FLAG_NATIVE_FP64) return forward_passes<double, double, double>(p);
    return forward_passes<double, dfl, dfl>(p);
}

cudaError_t launch_fft_adjoint(sgl_plan *p) {
    if (p->prec == SGL_FP32_MIXED) return adjoint_passes<float, dfl, float>(p);
    if (p->flags & SGL_FLAG_NATIVE_FP64) return adjoint_passes<double, double, double>(p);
    return adjoint_passes<double, dfl, dfl>(p);
}

}  // namespace sgl
