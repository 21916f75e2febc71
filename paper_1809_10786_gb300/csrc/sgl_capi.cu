// sgl_capi.cu -- the C-ABI of include/sgl.h: argument checks, plan set-up (FP64 host
// precompute of the polar conversion matrices, window Fourier factors and FFT tables),
// workspace ownership and the order of the kernel launches.
#include "sgl_internal.cuh"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

namespace sgl {

static thread_local std::string g_last_error;

// Event pairs recorded around each stage; read (and recycled) by sgl_profile.
struct Profiler {
    struct Pair { cudaEvent_t a, b; int stage; };
    std::vector<Pair> open, pool;
    cudaEvent_t take() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back().a;
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    ~Profiler() {
        for (auto &p : open) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
        for (auto &p : pool) cudaEventDestroy(p.a);
    }
};

// RAII scope: records a start event on construction and an end event on destruction, on the
// plan's stream or on the stream the stage runs on.
struct StageScope {
    sgl_plan *p;
    int stage;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    StageScope(sgl_plan *pl, int st) : StageScope(pl, st, pl->stream) {}
    StageScope(sgl_plan *pl, int st, cudaStream_t str) : p(pl), stage(st), s(str) {
        if (p->prof) { a = p->prof->take(); cudaEventRecord(a, s); }
    }
    ~StageScope() {
        if (p->prof && a) {
            cudaEvent_t b = p->prof->take();
            cudaEventRecord(b, s);
            p->prof->open.push_back({a, b, stage});
        }
    }
};

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone;
}

// Orders the plan's stream after the binning forked by the last sgl_set_points.  Inside a stream
// capture the wait becomes an external-event node of the graph (the binning ran outside it).
cudaError_t join_points(sgl_plan *p) {
    if (!p->bins_pending) return cudaSuccess;
    const bool cap = capturing(p->stream);
    cudaError_t e = cudaStreamWaitEvent(p->stream, p->ev_bins, cap ? cudaEventWaitExternal : 0);
    if (e == cudaSuccess && !cap) p->bins_pending = false;   // a captured wait orders only the graph
    return e;
}

void release_side(sgl_plan *p) {
    if (p->side) cudaStreamSynchronize(p->side);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_bins) cudaEventDestroy(p->ev_bins);
    if (p->side) cudaStreamDestroy(p->side);
    p->side = nullptr;
    p->ev_fork = p->ev_bins = nullptr;
    p->bins_pending = false;
}

sgl_status set_error(sgl_status code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

// Allocation-failure injection (sgl_test_fail_alloc): the number of further device allocations
// that succeed before one fails; negative: off.
static std::atomic<long long> g_fail_alloc_after{-1};

cudaError_t device_malloc(void **p, size_t bytes) {
    *p = nullptr;
    long long left = g_fail_alloc_after.load();
    while (left >= 0) {
        if (g_fail_alloc_after.compare_exchange_weak(left, left - 1)) {
            if (left == 0) return cudaErrorMemoryAllocation;      // the injected failure (one-shot)
            break;
        }
    }
    return cudaMalloc(p, bytes);
}

namespace {

sgl_status ok() {
    g_last_error.clear();
    return SGL_OK;
}

bool is_235_smooth(int n) {
    for (int f : {2, 3, 5})
        while (n % f == 0) n /= f;
    return n == 1;
}

int next_fft_size(double target) {
    int n = (int)std::ceil(target - 1e-9);
    if (n % 2) ++n;
    while (!is_235_smooth(n)) n += 2;
    return n;
}

void factor(int N, int *rad, int &nrad) {
    nrad = 0;
    while (N % 8 == 0) { rad[nrad++] = 8; N /= 8; }
    while (N % 4 == 0) { rad[nrad++] = 4; N /= 4; }
    while (N % 2 == 0) { rad[nrad++] = 2; N /= 2; }
    while (N % 3 == 0) { rad[nrad++] = 3; N /= 3; }
    while (N % 5 == 0) { rad[nrad++] = 5; N /= 5; }
}

// modified Bessel function I_0 by its power series (all terms positive)
double bessel_i0(double z) {
    const double x = 0.25 * z * z;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 500; ++k) {
        term *= x / ((double)k * k);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

// Fourier transform int psi(x) e^{-i w x} dx of the peak-normalized window (x in grid cells).
// Kaiser-Bessel: psi = [sinh(b s)/s] / [sinh(b q)/q], s = sqrt(q^2 - x^2); the pair
//   int sinh(b sqrt(q^2-x^2)) / sqrt(q^2-x^2) e^{-i w x} dx = pi I_0(q sqrt(b^2 - w^2))  (|w| <= b)
// Gaussian: psi = exp(-x^2 / (2 lambda)),  transform sqrt(2 pi lambda) exp(-lambda w^2 / 2)
// (Lemma on the Gaussian's Fourier transform, Sect. 2, after the change of variables).
double window_hat(int window, double w, double q, double par) {
    if (window == SGL_WIN_KB) {
        const double b = par;
        const double arg = std::sqrt(std::max(b * b - w * w, 0.0));
        // q / sinh(b q) = 2 q e^{-b q} / (1 - e^{-2 b q})
        const double scale = 2.0 * q * std::exp(-b * q) / (-std::expm1(-2.0 * b * q));
        return kPi * bessel_i0(q * arg) * scale;
    }
    return std::sqrt(2.0 * kPi * par) * std::exp(-0.5 * par * w * w);
}

// psi(x) of the kernels on the host, peak-normalized (psi(0) = 1), zero for |x| > q:
// KB [sinh(b s)/s] / [sinh(b q)/q], s = sqrt(q^2 - x^2); Gauss exp(-x^2 / (2 lambda))
double window_value_host(int window, double x, double q, double par) {
    if (std::fabs(x) > q) return 0.0;
    if (window == SGL_WIN_KB) {
        const double s = std::sqrt(q * q - x * x);
        const double ratio = (s > 1e-12) ? -std::expm1(-2.0 * par * s) / s : 2.0 * par;
        return std::exp(par * (s - q)) * ratio * q / (-std::expm1(-2.0 * par * q));
    }
    return std::exp(-x * x / (2.0 * par));
}

// largest error of the 1-D windowed interpolation of a single frequency |k| <= K on a grid of N
// points (n frequencies before oversampling), over the fractional positions (i + 1/2) / 128
double axis_error(int window, int N, int n, int K, int q) {
    const double sig = (double)N / n;
    const double par = (window == SGL_WIN_KB) ? kPi * (2.0 - 1.0 / sig) : sig * q / ((2.0 * sig - 1.0) * kPi);
    constexpr int kFrac = 128;
    double emax = 0.0;
    std::vector<double> psi((size_t)kFrac * 2 * q);
    for (int i = 0; i < kFrac; ++i)
        for (int j = 0; j < 2 * q; ++j) psi[(size_t)i * 2 * q + j] = window_value_host(window, (i + 0.5) / kFrac + q - 1 - j, q, par);
    for (int k = -K; k <= K; ++k) {
        const double w = 2.0 * kPi * k / N;
        const double ph = window_hat(window, w, (double)q, par);
        for (int i = 0; i < kFrac; ++i) {
            double re = 0.0, im = 0.0;
            for (int j = 0; j < 2 * q; ++j) {
                const double x = (i + 0.5) / kFrac + q - 1 - j, v = psi[(size_t)i * 2 * q + j];
                re += v * std::cos(w * x);
                im -= v * std::sin(w * x);
            }
            emax = std::max(emax, std::hypot(1.0 - re / ph, im / ph));
        }
    }
    return emax;
}

// psi (D = 0) and psi' (D = 1) of the kernels, peak-normalized, in extended precision (|x| <= q):
// KB psi = norm e^{b(s-q)} (1 - e^{-2bs}) / s, norm = q / (1 - e^{-2bq}), s = sqrt(q^2 - x^2),
//    psi' = -x 2 norm e^{-bq} (b s cosh(bs) - sinh(bs)) / s^3;  Gauss psi = e^{-x^2 / 2 lambda}, psi' = -x psi / lambda
long double window_ld(int window, int D, long double x, long double q, long double par) {
    if (window == SGL_WIN_KB) {
        const long double b = par, s = sqrtl(std::max(q * q - x * x, (long double)0));
        const long double norm = q / (-expm1l(-2 * b * q));
        if (D == 0) return s > 0 ? norm * expl(b * (s - q)) * (-expm1l(-2 * b * s)) / s : norm * expl(-b * q) * 2 * b;
        if (s <= 0) return -x * 2 * norm * expl(-b * q) * b * b * b / 3;
        return -x * 2 * norm * expl(-b * q) * (b * s * coshl(b * s) - sinhl(b * s)) / (s * s * s);
    }
    const long double v = expl(-x * x / (2 * par));
    return D == 0 ? v : -x * v / par;
}

// The table of one axis (psi and psi', layout at kWinNI): Chebyshev interpolation of degree
// kWinDeg on each piece, rewritten as a polynomial in the offset t = x - midpoint.  Tables depend
// only on (window, q, shape parameter) and are cached: plans of a batch share most of them.
std::vector<double> axis_window_table(int window, int q, double par) {
    constexpr int n = kWinDeg + 1;
    static std::mutex mu;
    static std::map<std::tuple<int, int, double>, std::vector<double>> cache;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(std::make_tuple(window, q, par));
        if (it != cache.end()) return it->second;
    }
    const long double pi = 3.14159265358979323846264338327950288L;
    // cos(pi k (j + 1/2) / n) (the Chebyshev nodes and the transform) and the monomial
    // coefficients of T_k(s): T_0 = 1, T_1 = s, T_{k+1} = 2 s T_k - T_{k-1}
    long double cs[n][n], T[n][n];
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j) cs[k][j] = cosl(pi * k * (j + 0.5L) / n);
    for (int k = 0; k < n; ++k)
        for (int c = 0; c < n; ++c) T[k][c] = 0;
    T[0][0] = 1;
    T[1][1] = 1;
    for (int k = 1; k + 1 < n; ++k)
        for (int c = 0; c < n; ++c) T[k + 1][c] = (c > 0 ? 2 * T[k][c - 1] : 0) - T[k - 1][c];
    std::vector<double> tab((size_t)2 * kWinNI * n);
    const long double h = (long double)q / kWinNI, half = h / 2;
    for (int D = 0; D < 2; ++D)
        for (int i = 0; i < kWinNI; ++i) {
            const long double mid = (i + 0.5L) * h;
            long double f[n], a[n];
            for (int j = 0; j < n; ++j) f[j] = window_ld(window, D, mid + half * cs[1][j], q, par);
            for (int k = 0; k < n; ++k) {
                long double acc = 0;
                for (int j = 0; j < n; ++j) acc += f[j] * cs[k][j];
                a[k] = acc * 2 / n;
            }
            a[0] /= 2;
            long double sc = 1;                     // s = t / half: the coefficient of t^c is m_c / half^c
            for (int c = 0; c < n; ++c, sc /= half) {
                long double m = 0;
                for (int k = c; k < n; ++k) m += a[k] * T[k][c];
                tab[((size_t)D * kWinNI + i) * n + c] = (double)(m * sc);
            }
        }
    std::lock_guard<std::mutex> lk(mu);
    cache.emplace(std::make_tuple(window, q, par), tab);
    return tab;
}

void window_tables(const sgl_plan *p, std::vector<double> &tab) {
    tab.assign(kWinTab, 0.0);
    for (int d = 0; d < 3; ++d) {
        const std::vector<double> t = axis_window_table(p->window, p->q, p->ax[d].wpar);
        std::copy(t.begin(), t.end(), tab.begin() + (size_t)d * t.size());
    }
}

// sum |eta_k| over n complex values into *acc (block sums, then one atomic add per block)
__global__ void __launch_bounds__(256) k_abs_sum(const double2 *__restrict__ x, int64_t n, double *__restrict__ acc) {
    __shared__ double ws[8];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += hypot(x[i].x, x[i].y);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) s += ws[w];
        atomicAdd(acc, s);
    }
}

double error_bound_of(int window, const int N[3], const int n[3], const int K[3], int q) {
    double b = 1.0;
    for (int d = 0; d < 3; ++d) b *= 1.0 + axis_error(window, N[d], n[d], K[d], q);
    return b - 1.0;
}

// Normalized associated Legendre values Pbar_lm(x) = Q_lm P_lm(x) for 0 <= m <= l < B
// (Condon-Shortley phase included), out[l * B + m], by the standard stable recurrences
//   Pbar_mm = -sqrt((2m+1)/(2m)) sin Pbar_{m-1,m-1},  Pbar_{m+1,m} = sqrt(2m+3) x Pbar_mm,
//   Pbar_lm = a_lm (x Pbar_{l-1,m} - b_lm Pbar_{l-2,m}),
//   a_lm = sqrt((4l^2-1)/(l^2-m^2)),  b_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)).
void legendre_normalized(int B, double x, double sn, double *out) {
    std::fill(out, out + (size_t)B * B, 0.0);
    double pmm = 1.0 / std::sqrt(4.0 * kPi);
    for (int m = 0; m < B; ++m) {
        if (m > 0) pmm *= -std::sqrt((2.0 * m + 1.0) / (2.0 * m)) * sn;
        out[(size_t)m * B + m] = pmm;
        if (m + 1 < B) out[(size_t)(m + 1) * B + m] = std::sqrt(2.0 * m + 3.0) * x * pmm;
        for (int l = m + 2; l < B; ++l) {
            const double a = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
            const double bb = std::sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
            out[(size_t)l * B + m] = a * (x * out[(size_t)(l - 1) * B + m] - bb * out[(size_t)(l - 2) * B + m]);
        }
    }
}

}  // namespace

// Polar conversion matrices (Sect. 6, spherical subtransform; Thm. on the factorization):
// for m >= 0, kappa1 = 0..K1, l = m..B-1, with w_j = (2j+1) pi / (4B), j < 2B:
//  m even: P[m][k][l] = (1/2B) sum_j cos(k w_j) Pbar_lm(cos w_j)       (DCT, then Chebyshev -> exponential)
//  m odd:  eps_k = (c_k/2B) sum_j cos(k w_j) Pbar_lm(cos w_j) / sin w_j  (c_0 = 1, c_k = 2; V_B weighting)
//          zeta_k = (1/4i) {2eps_0 - eps_2 (k=1); eps_{k-1} - eps_{k+1} (1<k<2B-2); eps_{k-1} (k >= 2B-2)}
//          and P[m][k][l] holds the real factor 4i zeta_k / 4 (the kernels apply the -i).
// The matrices for -m are (-1)^m times those for m.  Also the cosine table cos(m pi / 4B), m < 8B.
// No heap use (the allocation-free entry point builds its tables in static storage).
// Compensated dot-product accumulation (Ogita, Rump and Oishi's Dot2: the product's rounding
// error by a fused multiply-add, the sum's by TwoSum), as accurate as a sum in twice the working
// precision.  The tables took 10 s at B = 128 with extended-precision sums and a cosine per term.
struct Dot2 {
    double s = 0.0, c = 0.0;
    void add(double a, double b) {
        const double p = a * b, e = std::fma(a, b, -p);
        const double t = s + p, z = t - s;
        c += ((s - (t - z)) + (p - z)) + e;
        s = t;
    }
    double value() const { return s + c; }
};

void conversion_tables(int B, double *P, double *costab, double *leg) {
    constexpr int kMaxB2 = 2 * 128;
    const int K1 = B - 1, n2 = 2 * B, per = 8 * B;
    std::fill(P, P + (size_t)B * (K1 + 1) * B, 0.0);
    // cos(m pi / 4B), m < 8B; cos(k w_j) = costab[k (2j + 1) mod 8B] (exact argument reduction)
    for (int m = 0; m < per; ++m)
        costab[m] = (double)cosl((long double)m * 3.14159265358979323846264338327950288L / (4.0L * B));
    double w[kMaxB2], isin[kMaxB2], eps[kMaxB2 + 2];
    for (int j = 0; j < n2; ++j) {
        w[j] = (2.0 * j + 1.0) * kPi / (4.0 * B);
        isin[j] = 1.0 / std::sin(w[j]);
        legendre_normalized(B, std::cos(w[j]), std::sin(w[j]), leg + (size_t)j * B * B);
    }
    double lv[kMaxB2];
    // sum_j cos(k w_j) lv[j]: the table index k (2j + 1) mod 8B stepped by 2k
    auto cos_dot = [&](int k) {
        Dot2 d;
        int idx = k % per;
        const int step = (2 * k) % per;
        for (int j = 0; j < n2; ++j) {
            d.add(costab[idx], lv[j]);
            idx += step;
            if (idx >= per) idx -= per;
        }
        return d.value();
    };
    for (int m = 0; m < B; ++m) {
        for (int l = m; l < B; ++l) {
            for (int j = 0; j < n2; ++j) lv[j] = leg[((size_t)j * B + l) * B + m] * (m % 2 ? isin[j] : 1.0);
            if (m % 2 == 0) {
                for (int k = 0; k <= K1; ++k) P[((size_t)m * (K1 + 1) + k) * B + l] = cos_dot(k) / n2;
            } else {
                std::fill(eps, eps + n2 + 2, 0.0);
                for (int k = 0; k < n2; ++k) eps[k] = cos_dot(k) * (k == 0 ? 1.0 : 2.0) / n2;
                for (int k = 1; k <= K1; ++k) {
                    double v;
                    if (k == 1) v = 2.0 * eps[0] - eps[2];
                    else if (k < n2 - 2) v = eps[k - 1] - eps[k + 1];
                    else v = eps[k - 1];
                    P[((size_t)m * (K1 + 1) + k) * B + l] = v / 4.0;
                }
            }
        }
    }
}

namespace {

// P_m and the cosine table depend on B only: computed once per B per process and reused by every plan
struct ConvTables { std::vector<double> P, costab; };
const ConvTables &cached_conversion_tables(int B) {
    static std::mutex mu;
    static std::map<int, ConvTables> cache;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(B);
    if (it == cache.end()) {
        ConvTables t;
        t.P.resize((size_t)B * B * B);
        t.costab.resize((size_t)8 * B);
        std::vector<double> leg((size_t)2 * B * B * B);
        conversion_tables(B, t.P.data(), t.costab.data(), leg.data());
        it = cache.emplace(B, std::move(t)).first;
    }
    return it->second;
}

struct DevAlloc {
    std::vector<void *> ptrs;
    int64_t bytes = 0;
    template <typename T>
    cudaError_t get(T **p, size_t count) {
        *p = nullptr;
        if (count == 0) count = 1;
        void *q = nullptr;
        cudaError_t e = device_malloc(&q, count * sizeof(T));
        if (e != cudaSuccess) return e;
        ptrs.push_back(q);
        bytes += (int64_t)(count * sizeof(T));
        *p = (T *)q;
        return cudaSuccess;
    }
    void release() {
        for (void *q : ptrs) cudaFree(q);
        ptrs.clear();
    }
};

struct PlanHolder {
    sgl_plan plan;
    DevAlloc alloc;
};

const char *kStageNames[ST_COUNT] = {"points", "radial_matrix", "radial", "polar", "fft_forward", "interp",
                                     "spread", "fft_adjoint", "polar_adjoint", "radial_adjoint", "grad_interp",
                                     "trig_export"};

PlanHolder *holder_of(sgl_plan *p) { return reinterpret_cast<PlanHolder *>(p); }

bool aligned8(const void *p) { return ((uintptr_t)p & 7u) == 0; }

sgl_status check_plan(const sgl_plan *p) {
    if (!p) return set_error(SGL_ERR_ARG, "plan is NULL");
    return SGL_OK;
}

sgl_status launch_status(cudaError_t e, const char *what) {
    if (e != cudaSuccess) return set_error(SGL_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    return ok();
}

template <typename T>
cudaError_t upload(T *dst, const std::vector<T> &src, cudaStream_t s) {
    return cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

// binary64 values as double-float pairs (h = v rounded to binary32, l = the rest rounded)
std::vector<float2> df_pairs(const std::vector<double> &v) {
    std::vector<float2> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        const float h = (float)v[i];
        o[i] = make_float2(h, (float)(v[i] - (double)h));
    }
    return o;
}

}  // namespace
}  // namespace sgl

using namespace sgl;

extern "C" {

int64_t sgl_num_coeffs(int B) {
    if (B < 1) return -1;
    return (int64_t)B * (B + 1) * (2 * B + 1) / 6;
}

const char *sgl_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace sgl {

// Plan creation.  shared (optional): FFT work buffers owned by a batch, used instead of the
// plan's own when both are large enough (only the plan's own buffers are freed with it).
sgl_status plan_create_impl(sgl_plan **out, int B, int64_t M_max, int precision, int window, int q, double sigma,
                            unsigned flags, void *cuda_stream, const SharedWork *shared) {
    if (!out) return set_error(SGL_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (B < 1 || B > 128) return set_error(SGL_ERR_ARG, "B must be in [1, 128]");
    if (M_max < 0 || M_max >= ((int64_t)1 << 31)) return set_error(SGL_ERR_ARG, "M_max must be in [0, 2^31)");
    if (precision != SGL_FP64 && precision != SGL_FP32_MIXED) return set_error(SGL_ERR_ARG, "unknown precision");
    if (window != SGL_WIN_KB && window != SGL_WIN_GAUSS) return set_error(SGL_ERR_ARG, "unknown window");
    if (q < 1 || q > kMaxQ) return set_error(SGL_ERR_ARG, "q must be in [1, 16]");
    if (!(sigma >= 1.5 && sigma <= 4.0)) return set_error(SGL_ERR_ARG, "sigma must be in [1.5, 4]");
    if (flags & ~(SGL_FLAG_HOST_IO | SGL_FLAG_PROFILE | SGL_FLAG_SIMT | SGL_FLAG_TC | SGL_FLAG_NATIVE_FP64 | SGL_FLAG_OVERLAP_POINTS |
                  SGL_FLAG_GENERIC_FFT | SGL_FLAG_FULL_GRID))
        return set_error(SGL_ERR_ARG, "unknown flag bits");
    if ((flags & SGL_FLAG_SIMT) && (flags & SGL_FLAG_TC)) return set_error(SGL_ERR_ARG, "SGL_FLAG_SIMT and SGL_FLAG_TC exclude each other");

    PlanHolder *h = new (std::nothrow) PlanHolder();
    if (!h) return set_error(SGL_ERR_ALLOC, "host allocation failed");
    sgl_plan *p = &h->plan;
    std::memset(p, 0, sizeof(sgl_plan));
    cudaGetDevice(&p->device);
    if (cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess || p->num_sms < 1)
        p->num_sms = 1;
    p->stream = (cudaStream_t)cuda_stream;
    p->B = B; p->q = q; p->prec = precision; p->window = window; p->flags = flags; p->sigma = sigma;
    p->M_max = M_max; p->M = 0; p->Nc = sgl_num_coeffs(B);
    p->K0 = 2 * B - 2; p->K1 = B - 1;
    const int nsz[3] = {4 * B, 2 * B, 2 * B};
    const int Ksz[3] = {p->K0, p->K1, p->K1};
    auto fail = [&](sgl_status st, const std::string &m) {
        release_side(p);
        h->alloc.release();
        delete p->prof;
        delete h;
        return set_error(st, m);
    };
    for (int d = 0; d < 3; ++d) {
        Axis &a = p->ax[d];
        a.n = nsz[d];
        a.N = next_fft_size(sigma * nsz[d]);
        a.K = Ksz[d];
        if (a.N > 1024) return fail(SGL_ERR_UNSUPPORTED, "FFT length above 1024");
        if (q >= a.N) return fail(SGL_ERR_ARG, "q must be smaller than every oversampled grid size");
        a.sigma = (double)a.N / a.n;
        a.windowed = (d < 2) && (a.N / 2 + 2 * q + 1 <= a.N);
        a.rows = a.windowed ? a.N / 2 + 2 * q + 1 : a.N;
        a.first = a.windowed ? -q : 0;
        a.wpar = (window == SGL_WIN_KB) ? kPi * (2.0 - 1.0 / a.sigma) : a.sigma * q / ((2.0 * a.sigma - 1.0) * kPi);
        factor(a.N, a.rad, a.nrad);
    }
    {
        // symmetry-reduced FFT passes: axes 0 and 1 windowed (the halo rows then lie inside one
        // period), the azimuthal length even (the half-period shift); every FFT length is even
        p->half_grid = !(flags & SGL_FLAG_FULL_GRID) && p->ax[0].windowed && p->ax[1].windowed && p->ax[2].N % 2 == 0;
    }
    {
        BinGeom &g = p->bins;
        // FP32 plans with q <= 8: a multiple of 4, so that the tensor-core kernels' TMA boxes start
        // 16-byte aligned (lanes from sb2 * S2 - tc_halo(q)); otherwise as wide as one warp allows
        g.S2 = (precision == SGL_FP32_MIXED && q <= 8) ? 4 * ((32 - tc_halo(q) - q) / 4) : 33 - 2 * q;
        // must match the spreading kernels' template sizes; FP64 double-float spreading amortizes
        // its per-cell flush over the larger super-bin, the binary64 kernel's half-warp layout
        // keeps 4 x 2
        const bool native64 = precision == SGL_FP64 && (flags & SGL_FLAG_NATIVE_FP64);
        g.C0 = native64 ? 4 : 8;
        g.C1 = (precision == SGL_FP32_MIXED) ? 8 : (native64 ? 2 : 4);
        g.ncell[0] = p->ax[0].N / 2 + 1;
        g.ncell[1] = p->ax[1].N / 2 + 1;
        g.nsb[0] = (g.ncell[0] + g.C0 - 1) / g.C0;
        g.nsb[1] = (g.ncell[1] + g.C1 - 1) / g.C1;
        g.nsb[2] = (p->ax[2].N + g.S2 - 1) / g.S2;
        g.nsuper = (int64_t)g.nsb[0] * g.nsb[1] * g.nsb[2];
        g.nbins = g.nsuper * g.C0 * g.C1;
        p->nbins = g.nbins;
    }

    // ---- device allocations
    DevAlloc &A = h->alloc;
    Buffers &b = p->b;
    const int K0 = p->K0, K1 = p->K1;
    const int64_t W = 2 * K1 + 1;
    const size_t csz = precision == SGL_FP32_MIXED ? sizeof(float2) : sizeof(double2);
    const Axis &A0 = p->ax[0], &A1 = p->ax[1], &A2 = p->ax[2];
    // bufA also holds the symmetry-reduced adjoint's eta'[2K0+1][K1+1][W] (binary64)
    const size_t nA = std::max<size_t>(std::max<size_t>((size_t)A0.rows * W * W, (size_t)A0.rows * A1.rows * A2.N),
                                       ((size_t)(2 * K0 + 1) * (K1 + 1) * W * sizeof(double2) + csz - 1) / csz);
    const size_t bytesB = std::max<size_t>((size_t)A0.rows * A1.rows * W * csz, (size_t)(2 * K0 + 1) * W * W * sizeof(double2));
    cudaError_t e = cudaSuccess;
#define ALLOC(ptr, n) do { if ((e = A.get(&(ptr), (n))) != cudaSuccess) return fail(SGL_ERR_ALLOC, std::string("cudaMalloc: ") + cudaGetErrorString(e)); } while (0)
    ALLOC(b.P, (size_t)B * (K1 + 1) * B);
    ALLOC(b.costab, (size_t)8 * B);
    ALLOC(b.radv, (size_t)B * B * (B + 1));
    ALLOC(b.Kmat, (size_t)(K0 + 1) * B * (B + 1) / 2);
    ALLOC(b.beta, (size_t)(2 * B - 1) * (K0 + 1) * B);
    ALLOC(b.zeta, (size_t)(K0 + 1) * (K1 + 1) * W);
    ALLOC(b.linescale, (size_t)(W * W));
    ALLOC(b.linescale_df, (size_t)(W * W));
    if (shared && shared->bufA && shared->bufB && shared->bytesA >= nA * csz && shared->bytesB >= bytesB) {
        b.bufA = shared->bufA; b.bufB = shared->bufB;
        b.bufA_bytes = shared->bytesA; b.bufB_bytes = shared->bytesB;
    } else {
        unsigned char *pa = nullptr, *pb = nullptr;
        ALLOC(pa, nA * csz);
        ALLOC(pb, bytesB);
        b.bufA = pa; b.bufB = pb;
        b.bufA_bytes = nA * csz; b.bufB_bytes = bytesB;
    }
    for (int d = 0; d < 3; ++d) {
        Axis &a = p->ax[d];
        ALLOC(a.tw_d, (size_t)a.N);
        ALLOC(a.tw_f, (size_t)a.N);
        ALLOC(a.tw_df, (size_t)a.N);
        ALLOC(a.rev, (size_t)a.N);
        ALLOC(a.deconv, (size_t)(2 * a.K + 1));
        ALLOC(a.deconv_df, (size_t)(2 * a.K + 1));
    }
    ALLOC(b.r2max, 1);
    ALLOC(b.dev_flags, 1);
    const size_t Mc = (size_t)std::max<int64_t>(M_max, 1);
    ALLOC(b.u_tmp, 3 * Mc);
    ALLOC(b.u_sorted, 3 * Mc);
    ALLOC(b.pts32, Mc);
    ALLOC(b.rec_tmp, Mc);
    if (precision == SGL_FP32_MIXED) ALLOC(b.ys32, Mc);
    ALLOC(b.perm, Mc);
    ALLOC(b.bin_of, Mc);
    ALLOC(b.rank_of, Mc);
    ALLOC(b.bin_count, (size_t)p->nbins);
    ALLOC(b.bin_off, (size_t)p->nbins);
    ALLOC(b.scan_tmp, (size_t)(p->nbins / 2048 + 2));
    ALLOC(b.piece_cnt, (size_t)(4 * p->bins.nsuper));
    ALLOC(b.piece_off, (size_t)(4 * p->bins.nsuper));
    ALLOC(b.work[0], (size_t)work_list_cap(Mc, p->bins.nsuper, kTcPass));
    ALLOC(b.work[1], (size_t)work_list_cap(Mc, p->bins.nsuper, spread_chunk(precision)));
    ALLOC(b.work_len, 2);
    ALLOC(b.df_max, 3);
    ALLOC(b.scalar, 1);
    ALLOC(b.sched, 4);
    ALLOC(b.wtab, (size_t)kWinTab);
    ALLOC(b.wtab_df, (size_t)kWinTab);
    ALLOC(b.rot, (size_t)(2 * kRotK + 1));
    ALLOC(b.rotf, (size_t)(2 * kRotK + 1));
    if (flags & SGL_FLAG_HOST_IO) {
        ALLOC(b.io_xyz, 3 * Mc);
        ALLOC(b.io_coef, (size_t)(2 * p->Nc));
        ALLOC(b.io_vals, 2 * Mc);
        ALLOC(b.io_grad, 3 * Mc);
        ALLOC(b.io_out, 2 * Mc);
    }
    p->tc = tc_eligible(p);
    tc_choose(p);
    p->tc = p->tc_interp || p->tc_grad || p->tc_spread;
    if (p->tc) ALLOC(b.planes, (size_t)tc_plane_floats(p));
#undef ALLOC
    p->work_bytes = A.bytes;
    if (p->tc && (e = tc_make_tensor_map(p)) != cudaSuccess)
        return fail(SGL_ERR_CUDA, std::string("TMA descriptor of the grid planes: ") + cudaGetErrorString(e));
    if (flags & SGL_FLAG_PROFILE) p->prof = new (std::nothrow) Profiler();

    // ---- host precompute (FP64) and upload
    const ConvTables &ct = cached_conversion_tables(B);
    const std::vector<double> &P = ct.P, &costab = ct.costab;
    std::vector<double> dec[3];
    for (int d = 0; d < 3; ++d) {
        Axis &a = p->ax[d];
        dec[d].resize(2 * a.K + 1);
        for (int k = -a.K; k <= a.K; ++k)
            dec[d][k + a.K] = 1.0 / window_hat(window, 2.0 * kPi * k / a.N, (double)q, a.wpar);
        std::vector<double2> twd(a.N);
        std::vector<float2> twf(a.N);
        std::vector<float4> twdf(a.N);
        for (int m = 0; m < a.N; ++m) {
            const long double ang = 2.0L * 3.14159265358979323846264338327950288L * m / a.N;
            const long double c = cosl(ang), sn = sinl(ang);
            twd[m] = make_double2((double)c, (double)sn);
            twf[m] = make_float2((float)twd[m].x, (float)twd[m].y);
            const float ch = (float)c, sh = (float)sn;
            twdf[m] = make_float4(ch, (float)(c - (long double)ch), sh, (float)(sn - (long double)sh));
        }
        std::vector<int> rev(a.N);
        for (int k = 0; k < a.N; ++k) {
            int kk = k, pos = 0, S = a.N;
            for (int s = 0; s < a.nrad; ++s) {
                S /= a.rad[s];
                pos += (kk % a.rad[s]) * S;
                kk /= a.rad[s];
            }
            rev[k] = pos;
        }
        if ((e = upload(a.tw_d, twd, p->stream)) != cudaSuccess) return fail(SGL_ERR_CUDA, "upload twiddles");
        if ((e = upload(a.tw_f, twf, p->stream)) != cudaSuccess) return fail(SGL_ERR_CUDA, "upload twiddles");
        if ((e = upload(a.tw_df, twdf, p->stream)) != cudaSuccess) return fail(SGL_ERR_CUDA, "upload twiddles");
        if ((e = upload(a.rev, rev, p->stream)) != cudaSuccess) return fail(SGL_ERR_CUDA, "upload digit reversal");
        if ((e = upload(a.deconv, dec[d], p->stream)) != cudaSuccess) return fail(SGL_ERR_CUDA, "upload deconvolution");
        if ((e = upload(a.deconv_df, df_pairs(dec[d]), p->stream)) != cudaSuccess) return fail(SGL_ERR_CUDA, "upload deconvolution");
    }
    std::vector<double> ls((size_t)(W * W));
    for (int k1 = -K1; k1 <= K1; ++k1)
        for (int m = -K1; m <= K1; ++m) ls[(size_t)(k1 + K1) * W + (m + K1)] = dec[1][k1 + K1] * dec[2][m + K1];
    if ((e = upload(b.linescale_df, df_pairs(ls), p->stream)) != cudaSuccess) return fail(SGL_ERR_CUDA, "upload line scales");
    if ((e = upload(b.P, P, p->stream)) != cudaSuccess) return fail(SGL_ERR_CUDA, "upload polar matrices");
    if ((e = upload(b.costab, costab, p->stream)) != cudaSuccess) return fail(SGL_ERR_CUDA, "upload cosine table");
    if ((e = upload(b.linescale, ls, p->stream)) != cudaSuccess) return fail(SGL_ERR_CUDA, "upload line scales");
    if (precision == SGL_FP64 && !(flags & SGL_FLAG_NATIVE_FP64)) {      // read by the double-float kernels only
        std::vector<double> wt;
        window_tables(p, wt);
        if ((e = upload(b.wtab, wt, p->stream)) != cudaSuccess) return fail(SGL_ERR_CUDA, "upload window tables");
        if ((e = upload(b.wtab_df, df_pairs(wt), p->stream)) != cudaSuccess) return fail(SGL_ERR_CUDA, "upload window tables");
    }
    {
        // (cos, sin) of k pi / kRotK in extended precision, rounded to binary64 and to double-float pairs
        struct RotTables { std::vector<double2> d; std::vector<float4> f; };
        static const RotTables rot = [] {
            RotTables t;
            t.d.resize(2 * kRotK + 1);
            t.f.resize(2 * kRotK + 1);
            const long double pi = 3.14159265358979323846264338327950288L;
            auto pair = [](long double v, float &h, float &l) {
                h = (float)v;
                l = (float)(v - (long double)h);
            };
            for (int k = -kRotK; k <= kRotK; ++k) {
                const long double th = pi * k / kRotK, c = cosl(th), s = sinl(th);
                t.d[k + kRotK] = make_double2((double)c, (double)s);
                float4 &f = t.f[k + kRotK];
                pair(c, f.x, f.y);
                pair(s, f.z, f.w);
            }
            return t;
        }();
        if ((e = upload(b.rot, rot.d, p->stream)) != cudaSuccess || (e = upload(b.rotf, rot.f, p->stream)) != cudaSuccess)
            return fail(SGL_ERR_CUDA, "upload angle tables");
    }
    if ((e = cudaMemsetAsync(b.dev_flags, 0, sizeof(int), p->stream)) != cudaSuccess) return fail(SGL_ERR_CUDA, "memset");
    if ((flags & SGL_FLAG_OVERLAP_POINTS) && !shared) {   // the plans of a batch bin on the batch stream
        e = cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_bins, cudaEventDisableTiming);
        if (e != cudaSuccess) return fail(SGL_ERR_CUDA, std::string("binning stream: ") + cudaGetErrorString(e));
    }
    // the host vectors above are released on return: wait for the copies
    if ((e = cudaStreamSynchronize(p->stream)) != cudaSuccess) return fail(SGL_ERR_CUDA, std::string("plan upload: ") + cudaGetErrorString(e));
    *out = p;
    return ok();
}

// FFT work-buffer sizes (bytes) a plan with these parameters needs.
sgl_status plan_work_sizes(int B, int precision, int q, double sigma, size_t *bytesA, size_t *bytesB) {
    if (B < 1 || B > 128 || q < 1 || q > kMaxQ || !(sigma >= 1.5 && sigma <= 4.0)) return set_error(SGL_ERR_ARG, "invalid plan parameters");
    const int nsz[3] = {4 * B, 2 * B, 2 * B};
    int N[3], rows[3];
    for (int d = 0; d < 3; ++d) {
        N[d] = next_fft_size(sigma * nsz[d]);
        rows[d] = (d < 2 && N[d] / 2 + 2 * q + 1 <= N[d]) ? N[d] / 2 + 2 * q + 1 : N[d];
    }
    const int64_t W = 2 * (B - 1) + 1;
    const size_t csz = precision == SGL_FP32_MIXED ? sizeof(float2) : sizeof(double2);
    *bytesA = std::max<size_t>(std::max<size_t>((size_t)rows[0] * W * W, (size_t)rows[0] * rows[1] * N[2]) * csz,
                               (size_t)(2 * (2 * B - 2) + 1) * B * W * sizeof(double2));
    *bytesB = std::max<size_t>((size_t)rows[0] * rows[1] * W * csz, (size_t)(2 * (2 * B - 2) + 1) * W * W * sizeof(double2));
    return SGL_OK;
}

}  // namespace sgl

extern "C" {

sgl_status sgl_plan_create(sgl_plan **out, int B, int64_t M_max, int precision, int window, int q, double sigma,
                           unsigned flags, void *cuda_stream) {
    return plan_create_impl(out, B, M_max, precision, window, q, sigma, flags, cuda_stream, nullptr);
}

void sgl_plan_destroy(sgl_plan *plan) {
    if (!plan) return;
    PlanHolder *h = holder_of(plan);
    join_points(plan);
    cudaStreamSynchronize(plan->stream);
    release_side(plan);
    delete plan->prof;
    inverse_work_free(plan);
    h->alloc.release();
    delete h;
}

sgl_status sgl_set_stream(sgl_plan *plan, void *cuda_stream) {
    if (sgl_status s = check_plan(plan)) return s;
    plan->stream = (cudaStream_t)cuda_stream;
    return ok();
}

sgl_status sgl_plan_info(const sgl_plan *plan, sgl_plan_info_t *info) {
    if (sgl_status s = check_plan(plan)) return s;
    if (!info) return set_error(SGL_ERR_ARG, "info is NULL");
    info->B = plan->B; info->q = plan->q; info->precision = plan->prec; info->window = plan->window;
    info->num_coeffs = plan->Nc; info->M_max = plan->M_max; info->M = plan->M;
    for (int d = 0; d < 3; ++d) {
        info->n[d] = plan->ax[d].n; info->N[d] = plan->ax[d].N; info->rows[d] = plan->ax[d].rows;
        info->sigma_eff[d] = plan->ax[d].sigma;
    }
    info->workspace_bytes = plan->work_bytes;
    info->kernel_launches = plan->launches;
    info->tensor_cores = (plan->tc_interp ? 1 : 0) | (plan->tc_grad ? 2 : 0) | (plan->tc_spread ? 4 : 0);
    info->sym_grid = plan->half_grid ? 1 : 0;
    return ok();
}

sgl_status sgl_set_points(sgl_plan *plan, const double *xyz_dev, int64_t M) {
    if (sgl_status s = check_plan(plan)) return s;
    if (M < 0 || M > plan->M_max) return set_error(SGL_ERR_ARG, "M must be in [0, M_max]");
    if (M > 0 && (!xyz_dev || !aligned8(xyz_dev))) return set_error(SGL_ERR_ARG, "xyz must be a non-NULL, 8-byte aligned device pointer");
    // rho on the plan's stream (after the previous binning, which still reads it).  With
    // SGL_FLAG_OVERLAP_POINTS the binning then runs on the plan's binning stream, after everything
    // already on the plan's stream, so that it overlaps the conversions and the FFT of the next
    // forward; it reads a copy of the points in plan memory (u_sorted is rewritten only by its
    // own scatter), so the caller may reuse xyz in stream order.  In a stream capture it stays
    // on the plan's stream.
    cudaError_t e = join_points(plan);
    const bool fork = plan->side && !capturing(plan->stream);
    if (e == cudaSuccess) {
        StageScope sc(plan, ST_POINTS);   // from rho to the end of the binning
        e = launch_points_rho(plan, xyz_dev, M, fork ? plan->b.u_sorted : nullptr);
        bool forked = false;
        if (e == cudaSuccess && fork) {
            e = cudaEventRecord(plan->ev_fork, plan->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->side, plan->ev_fork, 0);
            if (e == cudaSuccess) {
                forked = true;
                sc.s = plan->side;
            }
        }
        if (e == cudaSuccess)
            e = launch_points_bins(plan, fork ? plan->b.u_sorted : xyz_dev, M, fork ? plan->side : plan->stream);
        if (e == cudaSuccess && fork) e = cudaEventRecord(plan->ev_bins, plan->side);
        // the join waits on ev_bins: only a recorded event may be waited on; after a failure past
        // the fork, drain the side stream and leave the plan without points
        if (e == cudaSuccess && fork) plan->bins_pending = true;
        if (e != cudaSuccess && forked) cudaStreamSynchronize(plan->side);
    }
    if (e != cudaSuccess) {
        plan->points_set = false;
        plan->M = 0;
        return launch_status(e, "set_points");
    }
    {
        StageScope sc(plan, ST_RADIAL_MATRIX);
        e = launch_radial_matrices(plan);
    }
    if (e != cudaSuccess) {
        plan->points_set = false;
        plan->M = 0;
        return launch_status(e, "radial matrices");
    }
    plan->M = M;
    plan->points_set = true;
    return ok();
}

sgl_status sgl_get_rho(sgl_plan *plan, double *rho_host) {
    if (sgl_status s = check_plan(plan)) return s;
    if (!rho_host) return set_error(SGL_ERR_ARG, "rho_host is NULL");
    if (!plan->points_set) return set_error(SGL_ERR_STATE, "sgl_set_points has not been called");
    unsigned long long bits = 0;
    SGL_CUDA_TRY(cudaMemcpyAsync(&bits, plan->b.r2max, sizeof(bits), cudaMemcpyDeviceToHost, plan->stream));
    SGL_CUDA_TRY(cudaStreamSynchronize(plan->stream));
    double r2;
    std::memcpy(&r2, &bits, sizeof(r2));
    double rho = std::sqrt(r2) * (1.0 + 0x1p-20);
    *rho_host = rho > 0.0 ? rho : 1.0;
    return ok();
}

static sgl_status coef_to_zeta(sgl_plan *plan, const double *coef_dev) {
    cudaError_t e;
    {
        StageScope sc(plan, ST_RADIAL);
        e = launch_radial_forward(plan, (const double2 *)coef_dev);
    }
    if (e != cudaSuccess) return launch_status(e, "radial conversion");
    {
        StageScope sc(plan, ST_POLAR);
        e = launch_polar_forward(plan);
    }
    if (e != cudaSuccess) return launch_status(e, "polar conversion");
    return ok();
}

static sgl_status zeta_to_grid(sgl_plan *plan) {
    StageScope sc(plan, ST_FFT_FWD);
    return launch_status(launch_fft_forward(plan), "forward FFT");
}

sgl_status sgl_forward(sgl_plan *plan, const double *coef_dev, double *vals_dev) {
    if (sgl_status s = check_plan(plan)) return s;
    if (!plan->points_set) return set_error(SGL_ERR_STATE, "sgl_set_points has not been called");
    if (!coef_dev || !aligned8(coef_dev)) return set_error(SGL_ERR_ARG, "coef must be a non-NULL, 8-byte aligned device pointer");
    if (plan->M > 0 && (!vals_dev || !aligned8(vals_dev))) return set_error(SGL_ERR_ARG, "vals must be a non-NULL, 8-byte aligned device pointer");
    if (plan->M == 0) return ok();
    if (sgl_status s = coef_to_zeta(plan, coef_dev)) return s;
    if (sgl_status s = zeta_to_grid(plan)) return s;
    SGL_CUDA_TRY(join_points(plan));
    StageScope sc(plan, ST_INTERP);
    return launch_status(launch_interp(plan, (double2 *)vals_dev), "interpolation");
}

sgl_status sgl_adjoint(sgl_plan *plan, const double *vals_dev, double *coef_dev) {
    if (sgl_status s = check_plan(plan)) return s;
    if (!plan->points_set) return set_error(SGL_ERR_STATE, "sgl_set_points has not been called");
    if (!coef_dev || !aligned8(coef_dev)) return set_error(SGL_ERR_ARG, "coef must be a non-NULL, 8-byte aligned device pointer");
    if (plan->M > 0 && (!vals_dev || !aligned8(vals_dev))) return set_error(SGL_ERR_ARG, "vals must be a non-NULL, 8-byte aligned device pointer");
    if (plan->M == 0) {
        SGL_CUDA_TRY(cudaMemsetAsync(coef_dev, 0, sizeof(double2) * plan->Nc, plan->stream));
        return ok();
    }
    const Axis &A0 = plan->ax[0], &A1 = plan->ax[1], &A2 = plan->ax[2];
    const size_t csz = plan->prec == SGL_FP32_MIXED ? sizeof(float2) : sizeof(double2);
    cudaError_t e = join_points(plan);
    if (e != cudaSuccess) return launch_status(e, "spreading");
    {
        StageScope sc(plan, ST_SPREAD);
        e = cudaMemsetAsync(plan->b.bufA, 0, (size_t)A0.rows * A1.rows * A2.N * csz, plan->stream);
        if (e == cudaSuccess) e = launch_spread(plan, (const double2 *)vals_dev);
    }
    if (e != cudaSuccess) return launch_status(e, "spreading");
    {
        StageScope sc(plan, ST_FFT_ADJ);
        e = launch_fft_adjoint(plan);
    }
    if (e != cudaSuccess) return launch_status(e, "adjoint FFT");
    {
        StageScope sc(plan, ST_POLAR_ADJ);
        // the adjoint FFT's output: eta' in bufB, or (symmetry-reduced) its kappa1 >= 0 half in bufA
        e = launch_polar_adjoint(plan, (const double2 *)(plan->half_grid ? plan->b.bufA : plan->b.bufB));
    }
    if (e != cudaSuccess) return launch_status(e, "adjoint polar conversion");
    StageScope sc(plan, ST_RADIAL_ADJ);
    return launch_status(launch_radial_adjoint(plan, (double2 *)coef_dev), "adjoint radial conversion");
}

sgl_status sgl_grad_points(sgl_plan *plan, const double *coef_dev, const double *gout_dev, double *gxyz_dev) {
    if (sgl_status s = check_plan(plan)) return s;
    if (!plan->points_set) return set_error(SGL_ERR_STATE, "sgl_set_points has not been called");
    if (!coef_dev || !aligned8(coef_dev)) return set_error(SGL_ERR_ARG, "coef must be a non-NULL, 8-byte aligned device pointer");
    if (plan->M > 0 && (!gout_dev || !gxyz_dev || !aligned8(gout_dev) || !aligned8(gxyz_dev)))
        return set_error(SGL_ERR_ARG, "gout and gxyz must be non-NULL, 8-byte aligned device pointers");
    if (plan->M == 0) return ok();
    if (sgl_status s = coef_to_zeta(plan, coef_dev)) return s;
    if (sgl_status s = zeta_to_grid(plan)) return s;
    SGL_CUDA_TRY(join_points(plan));
    StageScope sc(plan, ST_GRAD);
    return launch_status(launch_grad(plan, (const double2 *)gout_dev, gxyz_dev, nullptr), "gradient interpolation");
}

sgl_status sgl_forward_grad(sgl_plan *plan, const double *coef_dev, const double *gout_dev, double *vals_dev,
                            double *gxyz_dev) {
    if (sgl_status s = check_plan(plan)) return s;
    if (!plan->points_set) return set_error(SGL_ERR_STATE, "sgl_set_points has not been called");
    if (!coef_dev || !aligned8(coef_dev)) return set_error(SGL_ERR_ARG, "coef must be a non-NULL, 8-byte aligned device pointer");
    if (plan->M > 0 && (!gout_dev || !gxyz_dev || !vals_dev || !aligned8(gout_dev) || !aligned8(gxyz_dev) || !aligned8(vals_dev)))
        return set_error(SGL_ERR_ARG, "gout, vals and gxyz must be non-NULL, 8-byte aligned device pointers");
    if (plan->M == 0) return ok();
    if (sgl_status s = coef_to_zeta(plan, coef_dev)) return s;
    if (sgl_status s = zeta_to_grid(plan)) return s;
    SGL_CUDA_TRY(join_points(plan));
    StageScope sc(plan, ST_GRAD);
    return launch_status(launch_grad(plan, (const double2 *)gout_dev, gxyz_dev, (double2 *)vals_dev),
                         "gradient interpolation");
}

sgl_status sgl_trig_coeffs(sgl_plan *plan, const double *coef_dev, double *eta_dev) {
    if (sgl_status s = check_plan(plan)) return s;
    if (!plan->points_set) return set_error(SGL_ERR_STATE, "sgl_set_points has not been called");
    if (!coef_dev || !eta_dev || !aligned8(coef_dev) || !aligned8(eta_dev))
        return set_error(SGL_ERR_ARG, "coef and eta must be non-NULL, 8-byte aligned device pointers");
    if (sgl_status s = coef_to_zeta(plan, coef_dev)) return s;
    StageScope sc(plan, ST_TRIG);
    return launch_status(launch_trig_export(plan, (double2 *)eta_dev), "trig export");
}

}  // extern "C"

namespace {
// host variants: copy the points and bin them, or (xyz_host NULL) keep the plan's current points
sgl_status host_points(sgl_plan *plan, const double *xyz_host, int64_t M) {
    if (!xyz_host) {
        if (!plan->points_set || M != plan->M)
            return set_error(SGL_ERR_ARG, "xyz_host NULL reuses the current points: they must be set and M must equal their number");
        return SGL_OK;
    }
    if (M > 0)
        SGL_CUDA_TRY(cudaMemcpyAsync(plan->b.io_xyz, xyz_host, sizeof(double) * 3 * M, cudaMemcpyHostToDevice, plan->stream));
    return sgl_set_points(plan, plan->b.io_xyz, M);
}
}  // namespace

extern "C" {

sgl_status sgl_forward_host(sgl_plan *plan, const double *xyz_host, int64_t M, const double *coef_host, double *vals_host) {
    if (sgl_status s = check_plan(plan)) return s;
    if (!(plan->flags & SGL_FLAG_HOST_IO)) return set_error(SGL_ERR_STATE, "plan was created without SGL_FLAG_HOST_IO");
    if (M < 0 || M > plan->M_max) return set_error(SGL_ERR_ARG, "M must be in [0, M_max]");
    if (!coef_host || (M > 0 && !vals_host)) return set_error(SGL_ERR_ARG, "NULL host buffer");
    cudaStream_t st = plan->stream;
    if (sgl_status s = host_points(plan, xyz_host, M)) return s;
    SGL_CUDA_TRY(cudaMemcpyAsync(plan->b.io_coef, coef_host, sizeof(double2) * plan->Nc, cudaMemcpyHostToDevice, st));
    if (sgl_status s = sgl_forward(plan, plan->b.io_coef, plan->b.io_vals)) return s;
    if (M > 0) SGL_CUDA_TRY(cudaMemcpyAsync(vals_host, plan->b.io_vals, sizeof(double2) * M, cudaMemcpyDeviceToHost, st));
    return sgl_sync(plan);
}

sgl_status sgl_adjoint_host(sgl_plan *plan, const double *xyz_host, int64_t M, const double *vals_host, double *coef_host) {
    if (sgl_status s = check_plan(plan)) return s;
    if (!(plan->flags & SGL_FLAG_HOST_IO)) return set_error(SGL_ERR_STATE, "plan was created without SGL_FLAG_HOST_IO");
    if (M < 0 || M > plan->M_max) return set_error(SGL_ERR_ARG, "M must be in [0, M_max]");
    if (!coef_host || (M > 0 && !vals_host)) return set_error(SGL_ERR_ARG, "NULL host buffer");
    cudaStream_t st = plan->stream;
    if (sgl_status s = host_points(plan, xyz_host, M)) return s;
    if (M > 0) SGL_CUDA_TRY(cudaMemcpyAsync(plan->b.io_vals, vals_host, sizeof(double2) * M, cudaMemcpyHostToDevice, st));
    if (sgl_status s = sgl_adjoint(plan, plan->b.io_vals, plan->b.io_coef)) return s;
    SGL_CUDA_TRY(cudaMemcpyAsync(coef_host, plan->b.io_coef, sizeof(double2) * plan->Nc, cudaMemcpyDeviceToHost, st));
    return sgl_sync(plan);
}

const char *sgl_stage_name(int stage) {
    if (stage < 0 || stage >= ST_COUNT) return "";
    return kStageNames[stage];
}

sgl_status sgl_profile(sgl_plan *plan, double *ms_out, int64_t *count_out) {
    if (sgl_status s = check_plan(plan)) return s;
    if (!plan->prof) return set_error(SGL_ERR_STATE, "plan was created without SGL_FLAG_PROFILE");
    SGL_CUDA_TRY(join_points(plan));
    SGL_CUDA_TRY(cudaStreamSynchronize(plan->stream));
    double ms[ST_COUNT] = {0};
    int64_t cnt[ST_COUNT] = {0};
    for (auto &pr : plan->prof->open) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, pr.a, pr.b) == cudaSuccess) { ms[pr.stage] += t; cnt[pr.stage] += 1; }
        plan->prof->pool.push_back({pr.a, nullptr, 0});
        plan->prof->pool.push_back({pr.b, nullptr, 0});
    }
    plan->prof->open.clear();
    for (int i = 0; i < ST_COUNT; ++i) {
        if (ms_out) ms_out[i] = ms[i];
        if (count_out) count_out[i] = cnt[i];
    }
    return ok();
}

sgl_status sgl_grad_points_host(sgl_plan *plan, const double *xyz_host, int64_t M, const double *coef_host,
                                const double *gout_host, double *gxyz_host) {
    if (sgl_status s = check_plan(plan)) return s;
    if (!(plan->flags & SGL_FLAG_HOST_IO)) return set_error(SGL_ERR_STATE, "plan was created without SGL_FLAG_HOST_IO");
    if (M < 0 || M > plan->M_max) return set_error(SGL_ERR_ARG, "M must be in [0, M_max]");
    if (!coef_host || (M > 0 && (!gout_host || !gxyz_host))) return set_error(SGL_ERR_ARG, "NULL host buffer");
    cudaStream_t st = plan->stream;
    if (sgl_status s = host_points(plan, xyz_host, M)) return s;
    if (M > 0) SGL_CUDA_TRY(cudaMemcpyAsync(plan->b.io_vals, gout_host, sizeof(double2) * M, cudaMemcpyHostToDevice, st));
    SGL_CUDA_TRY(cudaMemcpyAsync(plan->b.io_coef, coef_host, sizeof(double2) * plan->Nc, cudaMemcpyHostToDevice, st));
    if (sgl_status s = sgl_grad_points(plan, plan->b.io_coef, plan->b.io_vals, plan->b.io_grad)) return s;
    if (M > 0) SGL_CUDA_TRY(cudaMemcpyAsync(gxyz_host, plan->b.io_grad, sizeof(double) * 3 * M, cudaMemcpyDeviceToHost, st));
    return sgl_sync(plan);
}

sgl_status sgl_forward_grad_host(sgl_plan *plan, const double *xyz_host, int64_t M, const double *coef_host,
                                 const double *gout_host, double *vals_host, double *gxyz_host) {
    if (sgl_status s = check_plan(plan)) return s;
    if (!(plan->flags & SGL_FLAG_HOST_IO)) return set_error(SGL_ERR_STATE, "plan was created without SGL_FLAG_HOST_IO");
    if (M < 0 || M > plan->M_max) return set_error(SGL_ERR_ARG, "M must be in [0, M_max]");
    if (!coef_host || (M > 0 && (!gout_host || !vals_host || !gxyz_host))) return set_error(SGL_ERR_ARG, "NULL host buffer");
    cudaStream_t st = plan->stream;
    if (sgl_status s = host_points(plan, xyz_host, M)) return s;
    if (M > 0) SGL_CUDA_TRY(cudaMemcpyAsync(plan->b.io_vals, gout_host, sizeof(double2) * M, cudaMemcpyHostToDevice, st));
    SGL_CUDA_TRY(cudaMemcpyAsync(plan->b.io_coef, coef_host, sizeof(double2) * plan->Nc, cudaMemcpyHostToDevice, st));
    if (sgl_status s = sgl_forward_grad(plan, plan->b.io_coef, plan->b.io_vals, plan->b.io_out, plan->b.io_grad)) return s;
    if (M > 0) {
        SGL_CUDA_TRY(cudaMemcpyAsync(vals_host, plan->b.io_out, sizeof(double2) * M, cudaMemcpyDeviceToHost, st));
        SGL_CUDA_TRY(cudaMemcpyAsync(gxyz_host, plan->b.io_grad, sizeof(double) * 3 * M, cudaMemcpyDeviceToHost, st));
    }
    return sgl_sync(plan);
}

sgl_status sgl_nfft_error_bound(int B, int window, int q, double sigma, double *bound) {
    if (!bound) return set_error(SGL_ERR_ARG, "bound must be non-NULL");
    if (B < 1 || B > 128 || q < 1 || q > kMaxQ || !(sigma >= 1.5 && sigma <= 4.0) ||
        (window != SGL_WIN_KB && window != SGL_WIN_GAUSS))
        return set_error(SGL_ERR_ARG, "invalid B, window, q or sigma");
    const int n[3] = {4 * B, 2 * B, 2 * B}, K[3] = {2 * B - 2, B - 1, B - 1};
    int N[3];
    for (int d = 0; d < 3; ++d) {
        N[d] = next_fft_size(sigma * n[d]);
        if (q >= N[d]) return set_error(SGL_ERR_ARG, "q must be smaller than every oversampled grid size");
    }
    *bound = error_bound_of(window, N, n, K, q);
    return ok();
}

sgl_status sgl_plan_error_bound(const sgl_plan *plan, double *bound) {
    if (sgl_status s = check_plan(plan)) return s;
    if (!bound) return set_error(SGL_ERR_ARG, "bound must be non-NULL");
    int N[3], n[3], K[3];
    for (int d = 0; d < 3; ++d) { N[d] = plan->ax[d].N; n[d] = plan->ax[d].n; K[d] = plan->ax[d].K; }
    *bound = error_bound_of(plan->window, N, n, K, plan->q);
    return ok();
}

sgl_status sgl_choose_cutoff(int B, int window, double sigma, double tol, int *q) {
    if (!q) return set_error(SGL_ERR_ARG, "q must be non-NULL");
    if (!(tol > 0.0)) return set_error(SGL_ERR_ARG, "tol must be positive");
    for (int qq = 1; qq <= kMaxQ; ++qq) {
        double b = 0.0;
        if (sgl_status s = sgl_nfft_error_bound(B, window, qq, sigma, &b)) return s;
        if (b <= tol) {
            *q = qq;
            return ok();
        }
    }
    return set_error(SGL_ERR_UNSUPPORTED, "no cutoff q <= 16 reaches the requested bound");
}

// Cost model of sgl_choose_params: one forward and one adjoint transform at M points cost
//   M (2q)^3 c_tap + (stored grid cells) c_cell   milliseconds,
// windowed loops (interpolation + spreading) per tap and FFT passes (forward + adjoint) per grid
// cell, measured on GB300 at B = 64, 10^6 points, q = 8, sigma = 2 (FP32-mixed: 0.89 + 1.49 ms of
// loops, 0.69 ms of FFT passes over 273 x 145 x 256 cells; FP64 with double-float loops: 9.3 +
// 15.9 ms and 3.81 ms).  The conversions do not depend on (sigma, q) and are left out.
namespace {
constexpr double kTapMs[2] = {(9.3 + 15.9) / 4.096e9, (0.89 + 1.49) / 4.096e9};   // [SGL_FP64, SGL_FP32_MIXED]
constexpr double kCellMs[2] = {3.81 / (273.0 * 145.0 * 256.0), 0.69 / (273.0 * 145.0 * 256.0)};
}  // namespace

sgl_status sgl_choose_params(int B, int64_t M, int precision, int window, double tol, double *sigma, int *q,
                             double *model_ms) {
    if (!sigma || !q) return set_error(SGL_ERR_ARG, "sigma and q must be non-NULL");
    if (!(tol > 0.0)) return set_error(SGL_ERR_ARG, "tol must be positive");
    if (M < 0) return set_error(SGL_ERR_ARG, "M must be >= 0");
    if (precision != SGL_FP64 && precision != SGL_FP32_MIXED) return set_error(SGL_ERR_ARG, "unknown precision");
    if (B < 1 || B > 128 || (window != SGL_WIN_KB && window != SGL_WIN_GAUSS))
        return set_error(SGL_ERR_ARG, "invalid B or window");
    const int nsz[3] = {4 * B, 2 * B, 2 * B}, K[3] = {2 * B - 2, B - 1, B - 1};
    double best = -1.0, best_sigma = 0.0;
    int best_q = 0;
    for (double sg : {1.5, 2.0, 2.5, 3.0, 4.0}) {
        int N[3];
        for (int d = 0; d < 3; ++d) N[d] = next_fft_size(sg * nsz[d]);
        // the bound falls with q: bisection for the smallest q <= 16 (and < every N) that meets tol
        int lo = 1, hi = std::min(kMaxQ, std::min(N[0], std::min(N[1], N[2])) - 1);
        if (hi < 1 || error_bound_of(window, N, nsz, K, hi) > tol) continue;
        while (lo < hi) {
            const int mid = (lo + hi) / 2;
            if (error_bound_of(window, N, nsz, K, mid) <= tol) hi = mid; else lo = mid + 1;
        }
        double cells = 1.0;
        for (int d = 0; d < 3; ++d) cells *= (d < 2 && N[d] / 2 + 2 * lo + 1 <= N[d]) ? N[d] / 2 + 2 * lo + 1 : N[d];
        const double taps = 8.0 * lo * lo * lo;
        const double cost = (double)M * taps * kTapMs[precision] + cells * kCellMs[precision];
        if (best < 0.0 || cost < best) { best = cost; best_sigma = sg; best_q = lo; }
    }
    if (best < 0.0) return set_error(SGL_ERR_UNSUPPORTED, "no oversampling factor with q <= 16 reaches the requested bound");
    *sigma = best_sigma;
    *q = best_q;
    if (model_ms) *model_ms = best;
    return ok();
}

sgl_status sgl_eta_l1(sgl_plan *plan, const double *coef_dev, double *l1) {
    if (sgl_status s = check_plan(plan)) return s;
    if (!plan->points_set) return set_error(SGL_ERR_STATE, "sgl_set_points has not been called");
    if (!coef_dev || !aligned8(coef_dev) || !l1) return set_error(SGL_ERR_ARG, "coef must be an 8-byte aligned device pointer, l1 non-NULL");
    if (sgl_status s = coef_to_zeta(plan, coef_dev)) return s;
    // the full eta array, (4B-3) x (2B-1) x (2B-1) complex128, in the FFT work buffer B (it holds
    // the adjoint's eta' of the same size)
    const int64_t n = (int64_t)(4 * plan->B - 3) * (2 * plan->B - 1) * (2 * plan->B - 1);
    double2 *eta = (double2 *)plan->b.bufB;
    if ((size_t)n * sizeof(double2) > plan->b.bufB_bytes) return set_error(SGL_ERR_STATE, "work buffer too small for eta");
    if (sgl_status s = launch_status(launch_trig_export(plan, eta), "trig export")) return s;
    SGL_CUDA_TRY(cudaMemsetAsync(plan->b.scalar, 0, sizeof(double), plan->stream));
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4 * 152);
    k_abs_sum<<<blocks, 256, 0, plan->stream>>>(eta, n, plan->b.scalar);
    plan->launches += 1;
    SGL_CUDA_TRY(cudaGetLastError());
    SGL_CUDA_TRY(cudaMemcpyAsync(l1, plan->b.scalar, sizeof(double), cudaMemcpyDeviceToHost, plan->stream));
    return sgl_sync(plan);
}

sgl_status sgl_test_hooks(sgl_plan *plan, unsigned hooks, int64_t wait_cycles) {
    if (sgl_status s = check_plan(plan)) return s;
    if (hooks & ~SGL_TEST_WITHHOLD_ARRIVAL) return set_error(SGL_ERR_ARG, "unknown test hook bits");
    if (wait_cycles < 0) return set_error(SGL_ERR_ARG, "wait_cycles must be >= 0");
    plan->test_hooks = hooks;
    plan->wait_cycles = wait_cycles;
    return ok();
}

sgl_status sgl_test_fail_alloc(int after) {
    g_fail_alloc_after.store(after < 0 ? -1 : after);
    return ok();
}

sgl_status sgl_sync(sgl_plan *plan) {
    if (sgl_status s = check_plan(plan)) return s;
    SGL_CUDA_TRY(join_points(plan));
    SGL_CUDA_TRY(cudaStreamSynchronize(plan->stream));
    int flagsv = 0;
    SGL_CUDA_TRY(cudaMemcpy(&flagsv, plan->b.dev_flags, sizeof(int), cudaMemcpyDeviceToHost));
    if (flagsv & 2) {
        SGL_CUDA_TRY(cudaMemset(plan->b.dev_flags, 0, sizeof(int)));
        return set_error(SGL_ERR_TIMEOUT, "a tensor-core pipeline wait gave up (results of the last call are invalid)");
    }
    if (flagsv & 1) {
        SGL_CUDA_TRY(cudaMemset(plan->b.dev_flags, 0, sizeof(int)));
        return set_error(SGL_ERR_NONFINITE, "a point coordinate was NaN or infinite (treated as the origin)");
    }
    return ok();
}

}  // extern "C"
