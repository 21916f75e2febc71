// sgl_convert.cu -- the exact part of the NFSGLFT factorization (Sect. 6), in FP64.
//
// Radial subtransform (Sect. 6, eqs. for alpha_{kappa l m} and beta_{kappa l m}):
//   g_lm(r) = sum_{n=l+1}^{B} fhat_nlm N_nl R_nl(r) is a polynomial of degree <= 2B-2 on
//   [0, rho]; sampled at r_j = rho (1 + cos w_j)/2, w_j = (2j+1) pi / (4B), j < 2B, and
//   expanded by the DCT, its exponential coefficients are
//     beta_{kappa0 l m} = (1/2B) sum_j cos(|kappa0| w_j) g_lm(r_j)        (|kappa0| <= 2B-2),
//   the same for kappa0 and -kappa0.  With the values matrix V_l[j, n] = N_nl R_nl(r_j)
//   (normalized Laguerre recurrence, below) this is beta = K_l fhat_{.lm} with
//   K_l = (1/2B) [cos(kappa0 w_j)] V_l, a (2B-1) x (B-l) matrix built on the device once rho is known.
// Spherical subtransform (Sect. 6, eqs. for eps and zeta, even and odd m):
//   zeta_{kappa0 kappa1 m} = sum_{l=|m|}^{B-1} P_m[kappa1, l] beta_{kappa0 l m}
//   with the plan's precomputed P_m = W_m D C~ (V_B) L~_m^T diag(Q) (P_m purely imaginary for odd m).
// The adjoints apply the transposed conjugate factors in reverse order (Sect. 6, corollary).
#include "sgl_internal.cuh"

namespace sgl {
namespace {

constexpr int kT = 256;

__host__ __device__ __forceinline__ int64_t radv_off(int B, int l) {     // sum_{l'<l} 2B (B - l')
    return (int64_t)2 * B * ((int64_t)l * B - (int64_t)l * (l - 1) / 2);
}
__host__ __device__ __forceinline__ int64_t kmat_off(int B, int K0, int l) {  // sum_{l'<l} (K0+1)(B - l')
    return (int64_t)(K0 + 1) * ((int64_t)l * B - (int64_t)l * (l - 1) / 2);
}
__device__ __forceinline__ int64_t mu_index(int n, int l, int m) {
    return (int64_t)n * (n - 1) * (2 * n - 1) / 6 + (int64_t)l * (l + 1) + m;
}
__device__ __forceinline__ double rho_from(const unsigned long long *r2max) {
    double rho = sqrt(__longlong_as_double((long long)*r2max)) * (1.0 + 0x1p-20);
    return rho > 0.0 ? rho : 1.0;
}

// V_l[j, k] = N_nl R_nl(r_j), n = l + 1 + k, via the normalized Laguerre recurrence
//   psi_{k+1} = ((2k+1+a-x) psi_k - sqrt(k(k+a)) psi_{k-1}) / sqrt((k+1)(k+1+a)),  a = l + 1/2, x = r^2,
// started from psi_0 = r^l / sqrt(Gamma(l + 3/2)) (so N_nl R_nl = sqrt(2) psi_k).  The square
// roots depend on l and k only: the block (one l) computes them once into shared memory, so that
// each thread's recurrence step is a few multiply-adds (FP64 square roots and divisions are long
// instruction sequences on GB300's FP64 pipe).
constexpr int kRvMax = 128;                    // B <= 128
__global__ void __launch_bounds__(128) k_radial_values(int B, const unsigned long long *__restrict__ r2max,
                                                       const double *__restrict__ costab, double *__restrict__ radv) {
    __shared__ double sq[kRvMax], isq[kRvMax], fac[kRvMax];
    const int l = blockIdx.y;
    const int K = B - l;
    const double a = l + 0.5;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        sq[k] = sqrt(k * (k + a));                          // sqrt(k (k + a))
        isq[k] = 1.0 / sqrt((k + 1.0) * (k + 1.0 + a));     // 1 / sqrt((k + 1)(k + 1 + a))
    }
    for (int i = threadIdx.x; i < l; i += blockDim.x) fac[i] = 1.0 / sqrt(i + 1.5);   // 1 / sqrt(i' + 1/2), i' = i + 1
    __syncthreads();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= B || j >= 2 * B) return;
    const double rho = rho_from(r2max);
    const double r = 0.5 * rho * (1.0 + costab[2 * j + 1]);   // cos w_j = cos((2j+1) pi / 4B)
    const double x = r * r;
    // r^l / sqrt(Gamma(l + 3/2)) = prod_{i=1}^{l} r / sqrt(i + 1/2) / sqrt(Gamma(3/2))
    double t = 1.0 / sqrt(0.5 * sqrt(kPi));
    for (int i = 0; i < l; ++i) t *= r * fac[i];
    double *out = radv + radv_off(B, l) + (int64_t)j * K;
    double pm1 = 0.0, p = t;
    out[0] = 1.4142135623730951 * p;
    for (int k = 0; k + 1 < K; ++k) {
        const double nx = fma(2.0 * k + 1.0 + a - x, p, -sq[k] * pm1) * isq[k];
        pm1 = p;
        p = nx;
        out[k + 1] = 1.4142135623730951 * p;
    }
}

// K_l[kappa0, k] = (1/2B) sum_j cos(kappa0 w_j) V_l[j, k],  kappa0 = 0..K0.  A thread takes
// kRmK0 kappa0 and kRmK k (each V loaded serves kRmK0 multiply-adds; small tiles keep enough
// threads in flight); cos(kappa0 w_j) comes from the table cos(m pi / 4B),
// m = (2j + 1) kappa0 mod 8B, stepped by 2 kappa0 per j.
constexpr int kRmK0 = 2, kRmK = 1;
__global__ void __launch_bounds__(128) k_radial_matrix(int B, int K0, const double *__restrict__ costab,
                                                       const double *__restrict__ radv, double *__restrict__ Kmat) {
    const int l = blockIdx.y;
    const int K = B - l;
    const int nk = (K + kRmK - 1) / kRmK;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ((K0 + 1 + kRmK0 - 1) / kRmK0) * nk) return;
    const int ka = (idx / nk) * kRmK0, k = (idx % nk) * kRmK;
    const double *v = radv + radv_off(B, l);
    const int per = 8 * B;                     // costab holds cos(m pi / 4B), m < 8B
    int m[kRmK0], step[kRmK0];
#pragma unroll
    for (int a = 0; a < kRmK0; ++a) {
        const int kap = min(ka + a, K0);
        m[a] = kap % per;
        step[a] = (2 * kap) % per;
    }
    double s[kRmK0][kRmK] = {};
    for (int j = 0; j < 2 * B; ++j) {
        double vv[kRmK];
#pragma unroll
        for (int b = 0; b < kRmK; ++b) vv[b] = k + b < K ? v[(int64_t)j * K + k + b] : 0.0;
#pragma unroll
        for (int a = 0; a < kRmK0; ++a) {
            const double c = costab[m[a]];
#pragma unroll
            for (int b = 0; b < kRmK; ++b) s[a][b] = fma(c, vv[b], s[a][b]);
            m[a] += step[a];
            if (m[a] >= per) m[a] -= per;
        }
    }
    double *out = Kmat + kmat_off(B, K0, l);
    const double n2 = 2.0 * B;
#pragma unroll
    for (int a = 0; a < kRmK0; ++a) {
        if (ka + a > K0) break;
#pragma unroll
        for (int b = 0; b < kRmK; ++b)
            if (k + b < K) out[(int64_t)(ka + a) * K + k + b] = s[a][b] / n2;
    }
}
inline dim3 radial_matrix_grid(int B, int K0, int threads) {
    const int tiles = ((K0 + 1 + kRmK0 - 1) / kRmK0) * ((B + kRmK - 1) / kRmK);   // the largest (l = 0)
    return dim3((unsigned)((tiles + threads - 1) / threads), (unsigned)B);
}

// beta[m + B - 1][kappa0][l] = sum_k K_l[kappa0, k] fhat_{l+1+k, l, m}
__global__ void k_radial_forward(int B, int K0, const double *__restrict__ Kmat, const double2 *__restrict__ coef,
                                 double2 *__restrict__ beta) {
    const int l = blockIdx.y;
    const int K = B - l;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (2 * l + 1) * (K0 + 1)) return;
    const int kap = idx % (K0 + 1);
    const int m = idx / (K0 + 1) - l;
    const double *kr = Kmat + kmat_off(B, K0, l) + (int64_t)kap * K;
    double re = 0.0, im = 0.0;
#pragma unroll 4
    for (int k = 0; k < K; ++k) {
        const double2 c = coef[mu_index(l + 1 + k, l, m)];
        const double w = kr[k];
        re = fma(w, c.x, re);
        im = fma(w, c.y, im);
    }
    beta[((int64_t)(m + B - 1) * (K0 + 1) + kap) * B + l] = make_double2(re, im);
}

// zeta[kappa0][kappa1][m + K1] = c_m sum_{l=|m|}^{B-1} P[|m|][kappa1][l] beta[m][kappa0][l],
// c_m = (-1)^m for m < 0 (P_{-m} = (-1)^m P_m), times -i for odd m (W_m carries 1/(4i)).
// One m per blockIdx.y; a thread takes two kappa0 and four kappa1, so that each loaded P entry
// and beta value serves several multiply-adds (P_m and beta_m of one m stay in L1).
constexpr int kPfK0 = 2, kPfK1 = 4;
__global__ void __launch_bounds__(128) k_polar_forward(int B, int K0, int K1, const double *__restrict__ P,
                                                       const double2 *__restrict__ beta, double2 *__restrict__ zeta) {
    const int W = 2 * K1 + 1;
    const int mi = blockIdx.y, m = mi - K1, am = m < 0 ? -m : m;
    const int n1 = (K1 + 1 + kPfK1 - 1) / kPfK1;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ((K0 + 1 + kPfK0 - 1) / kPfK0) * n1) return;
    const int k1a = (idx % n1) * kPfK1, k0a = (idx / n1) * kPfK0;
    const double *pr[kPfK1];
    const double2 *br[kPfK0];
#pragma unroll
    for (int i = 0; i < kPfK1; ++i) pr[i] = P + ((int64_t)am * (K1 + 1) + min(k1a + i, K1)) * B;
#pragma unroll
    for (int j = 0; j < kPfK0; ++j) br[j] = beta + ((int64_t)(m + B - 1) * (K0 + 1) + min(k0a + j, K0)) * B;
    double re[kPfK0][kPfK1] = {}, im[kPfK0][kPfK1] = {};
    for (int l = am; l < B; ++l) {
        double w[kPfK1];
        double2 v[kPfK0];
#pragma unroll
        for (int i = 0; i < kPfK1; ++i) w[i] = pr[i][l];
#pragma unroll
        for (int j = 0; j < kPfK0; ++j) v[j] = br[j][l];
#pragma unroll
        for (int j = 0; j < kPfK0; ++j)
#pragma unroll
            for (int i = 0; i < kPfK1; ++i) {
                re[j][i] = fma(w[i], v[j].x, re[j][i]);
                im[j][i] = fma(w[i], v[j].y, im[j][i]);
            }
    }
#pragma unroll
    for (int j = 0; j < kPfK0; ++j)
#pragma unroll
        for (int i = 0; i < kPfK1; ++i) {
            if (k0a + j > K0 || k1a + i > K1) continue;
            double a = re[j][i], b = im[j][i];
            if (m < 0 && (am & 1)) { a = -a; b = -b; }
            if (am & 1) { const double t = a; a = b; b = -t; }      // multiply by -i
            zeta[((int64_t)(k0a + j) * (K1 + 1) + (k1a + i)) * W + mi] = make_double2(a, b);
        }
}
inline dim3 polar_forward_grid(int K0, int K1, int threads) {
    const int tiles = ((K0 + 1 + kPfK0 - 1) / kPfK0) * ((K1 + 1 + kPfK1 - 1) / kPfK1);
    return dim3((unsigned)((tiles + threads - 1) / threads), (unsigned)(2 * K1 + 1));
}

__global__ void k_trig_export(int K0, int K1, const double2 *__restrict__ zeta, double2 *__restrict__ eta) {
    const int W = 2 * K1 + 1;
    const int64_t total = (int64_t)(2 * K0 + 1) * W * W;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int mi = (int)(idx % W);
    const int k1 = (int)((idx / W) % W) - K1;
    const int k0 = (int)(idx / ((int64_t)W * W)) - K0;
    const int m = mi - K1;
    double2 v = zeta[((int64_t)abs(k0) * (K1 + 1) + abs(k1)) * W + mi];
    if (k1 < 0 && (m & 1)) { v.x = -v.x; v.y = -v.y; }
    eta[idx] = v;
}

// adjoint of the mirroring: zeta'[kappa0][kappa1][m] = sum over the preimages of eta'.  With
// `half`, eta' holds kappa1 >= 0 only ([2K0+1][K1+1][2K1+1]: the symmetry-reduced adjoint FFT has
// folded kappa1 already) and only kappa0 is folded here.
__global__ void k_fold(int K0, int K1, int half, const double2 *__restrict__ etap, double2 *__restrict__ zetap) {
    const int W = 2 * K1 + 1;
    const int64_t total = (int64_t)(K0 + 1) * (K1 + 1) * W;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int mi = (int)(idx % W);
    const int k1 = (int)((idx / W) % (K1 + 1));
    const int k0 = (int)(idx / ((int64_t)W * (K1 + 1)));
    const int m = mi - K1;
    const double par = (m & 1) ? -1.0 : 1.0;
    double re = 0.0, im = 0.0;
    for (int s0 = 0; s0 < (k0 ? 2 : 1); ++s0) {
        const int kk0 = s0 ? -k0 : k0;
        for (int s1 = 0; s1 < (k1 && !half ? 2 : 1); ++s1) {
            const int kk1 = s1 ? -k1 : k1;
            const double f = s1 ? par : 1.0;
            const int64_t at = half ? ((int64_t)(kk0 + K0) * (K1 + 1) + k1) * W + mi : ((int64_t)(kk0 + K0) * W + (kk1 + K1)) * W + mi;
            const double2 v = etap[at];
            re = fma(f, v.x, re);
            im = fma(f, v.y, im);
        }
    }
    zetap[idx] = make_double2(re, im);
}

// beta'[m][kappa0][l] = conj(c_m) sum_{kappa1} P[|m|][kappa1][l] zeta'[kappa0][kappa1][m],  l >= |m|.
// One m per blockIdx.y; a thread takes four consecutive l of one kappa0 (one loaded zeta' value
// serves four multiply-adds; a larger tile leaves too few threads to hide the loads).
constexpr int kPaL = 4, kPaK0 = 1;
__global__ void __launch_bounds__(128) k_polar_adjoint(int B, int K0, int K1, const double *__restrict__ P,
                                                       const double2 *__restrict__ zetap, double2 *__restrict__ beta) {
    const int W = 2 * K1 + 1;
    const int mi = blockIdx.y, m = mi - K1, am = m < 0 ? -m : m;
    const int nl = (B - am + kPaL - 1) / kPaL;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ((K0 + 1 + kPaK0 - 1) / kPaK0) * nl) return;
    const int la = am + (idx % nl) * kPaL, k0a = (idx / nl) * kPaK0;
    double re[kPaK0][kPaL] = {}, im[kPaK0][kPaL] = {};
    const double *pbase = P + (int64_t)am * (K1 + 1) * B;
#pragma unroll 4
    for (int k1 = 0; k1 <= K1; ++k1) {
        double w[kPaL];
        double2 v[kPaK0];
#pragma unroll
        for (int i = 0; i < kPaL; ++i) w[i] = pbase[(int64_t)k1 * B + min(la + i, B - 1)];
#pragma unroll
        for (int j = 0; j < kPaK0; ++j) v[j] = zetap[((int64_t)min(k0a + j, K0) * (K1 + 1) + k1) * W + mi];
#pragma unroll
        for (int j = 0; j < kPaK0; ++j)
#pragma unroll
            for (int i = 0; i < kPaL; ++i) {
                re[j][i] = fma(w[i], v[j].x, re[j][i]);
                im[j][i] = fma(w[i], v[j].y, im[j][i]);
            }
    }
#pragma unroll
    for (int j = 0; j < kPaK0; ++j)
#pragma unroll
        for (int i = 0; i < kPaL; ++i) {
            if (k0a + j > K0 || la + i >= B) continue;
            double a = re[j][i], b = im[j][i];
            if (m < 0 && (am & 1)) { a = -a; b = -b; }
            if (am & 1) { const double t = a; a = -b; b = t; }      // conj(-i) = +i
            beta[((int64_t)mi * (K0 + 1) + (k0a + j)) * B + (la + i)] = make_double2(a, b);
        }
}
inline dim3 polar_adjoint_grid(int B, int K0, int K1, int threads) {
    const int tiles = ((K0 + 1 + kPaK0 - 1) / kPaK0) * ((B + kPaL - 1) / kPaL);   // the largest (m = 0)
    return dim3((unsigned)((tiles + threads - 1) / threads), (unsigned)(2 * K1 + 1));
}

// fhat'_{n l m} = sum_{kappa0} K_l[kappa0, n-l-1] beta'[m][kappa0][l]
__global__ void k_radial_adjoint(int B, int K0, int64_t Nc, const double *__restrict__ Kmat, const double2 *__restrict__ beta,
                                 double2 *__restrict__ coef) {
    const int64_t mu = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (mu >= Nc) return;
    int n = 1;
    while ((int64_t)(n + 1) * n * (2 * n + 1) / 6 <= mu) ++n;   // n(mu): largest n with n(n-1)(2n-1)/6 <= mu
    const int64_t rem = mu - (int64_t)n * (n - 1) * (2 * n - 1) / 6;
    int l = (int)sqrt((double)rem);
    while ((int64_t)(l + 1) * (l + 1) <= rem) ++l;
    while ((int64_t)l * l > rem) --l;
    const int m = (int)(rem - (int64_t)l * (l + 1));
    const int K = B - l, k = n - l - 1;
    const double *kr = Kmat + kmat_off(B, K0, l) + k;
    const double2 *br = beta + (int64_t)(m + B - 1) * (K0 + 1) * B + l;
    double re = 0.0, im = 0.0;
#pragma unroll 4
    for (int kap = 0; kap <= K0; ++kap) {
        const double w = kr[(int64_t)kap * K];
        const double2 v = br[(int64_t)kap * B];
        re = fma(w, v.x, re);
        im = fma(w, v.y, im);
    }
    coef[mu] = make_double2(re, im);
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_radial_matrices(sgl_plan *p) {
    const int B = p->B, K0 = p->K0;
    Buffers &b = p->b;
    dim3 g1(blocks_for(2 * B, 128), B);
    k_radial_values<<<g1, 128, 0, p->stream>>>(B, b.r2max, b.costab, b.radv);
    k_radial_matrix<<<radial_matrix_grid(B, K0, 128), 128, 0, p->stream>>>(B, K0, b.costab, b.radv, b.Kmat);
    p->launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_radial_forward(sgl_plan *p, const double2 *coef) {
    const int B = p->B, K0 = p->K0;
    dim3 g(blocks_for((int64_t)(2 * B - 1) * (K0 + 1), kT), B);
    k_radial_forward<<<g, kT, 0, p->stream>>>(B, K0, p->b.Kmat, coef, p->b.beta);
    p->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_polar_forward(sgl_plan *p) {
    const int64_t total = (int64_t)(p->K0 + 1) * (p->K1 + 1) * (2 * p->K1 + 1);
    (void)total;
    k_polar_forward<<<polar_forward_grid(p->K0, p->K1, 128), 128, 0, p->stream>>>(p->B, p->K0, p->K1, p->b.P, p->b.beta, p->b.zeta);
    p->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_trig_export(sgl_plan *p, double2 *eta) {
    const int64_t W = 2 * p->K1 + 1;
    const int64_t total = (int64_t)(2 * p->K0 + 1) * W * W;
    k_trig_export<<<blocks_for(total, kT), kT, 0, p->stream>>>(p->K0, p->K1, p->b.zeta, eta);
    p->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_polar_adjoint(sgl_plan *p, const double2 *eta_full) {
    const int B = p->B, K0 = p->K0, K1 = p->K1;
    const int64_t W = 2 * K1 + 1;
    k_fold<<<blocks_for((int64_t)(K0 + 1) * (K1 + 1) * W, kT), kT, 0, p->stream>>>(K0, K1, p->half_grid ? 1 : 0, eta_full,
                                                                                    p->b.zeta);
    k_polar_adjoint<<<polar_adjoint_grid(B, K0, K1, 128), 128, 0, p->stream>>>(B, K0, K1, p->b.P, p->b.zeta, p->b.beta);
    p->launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_trig_raw(cudaStream_t s, int B, const unsigned long long *r2max, const double *costab, const double *P,
                            double *radv, double *Kmat, double2 *beta, double2 *zeta, const double2 *coef, double2 *eta) {
    const int K0 = 2 * B - 2, K1 = B - 1;
    const int64_t W = 2 * K1 + 1;
    k_radial_values<<<dim3(blocks_for(2 * B, 128), B), 128, 0, s>>>(B, r2max, costab, radv);
    k_radial_matrix<<<radial_matrix_grid(B, K0, 128), 128, 0, s>>>(B, K0, costab, radv, Kmat);
    k_radial_forward<<<dim3(blocks_for((int64_t)(2 * B - 1) * (K0 + 1), kT), B), kT, 0, s>>>(B, K0, Kmat, coef, beta);
    k_polar_forward<<<polar_forward_grid(K0, K1, 128), 128, 0, s>>>(B, K0, K1, P, beta, zeta);
    k_trig_export<<<blocks_for((int64_t)(2 * K0 + 1) * W * W, kT), kT, 0, s>>>(K0, K1, zeta, eta);
    return cudaGetLastError();
}

cudaError_t launch_radial_adjoint(sgl_plan *p, double2 *coef) {
    k_radial_adjoint<<<blocks_for(p->Nc, kT), kT, 0, p->stream>>>(p->B, p->K0, p->Nc, p->b.Kmat, p->b.beta, coef);
    p->launches += 1;
    return cudaGetLastError();
}

}  // namespace sgl
