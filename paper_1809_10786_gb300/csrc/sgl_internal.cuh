// sgl_internal.cuh -- plan layout and kernel entry points shared by the CUDA
// translation units of libsgl.so.  Not part of the public C-ABI (include/sgl.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

#include "../../include/sgl.h"

namespace sgl {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxQ = 16;          // 2q taps per axis must fit one warp
constexpr int kMaxRadices = 16;
// Spatial bins: a column bin holds the points of one (i0, i1) cell column and one chunk of
// S2 = 33 - 2q cells on the azimuthal axis, so the taps of all its points cover one warp's
// 32 lanes on that axis and share their (2q)^2 rows.  C0 x C1 columns form a super-bin.
struct BinGeom {
    int S2;             // azimuthal cells per chunk
    int C0, C1;         // columns per super-bin along axes 0 and 1
    int nsb[3];         // super-bins per axis (axis 2 counts chunks)
    int ncell[2];       // cell columns per axis 0 and 1 (N/2 + 1)
    int64_t nbins;      // nsb0 * nsb2 * nsb1 * C0 * C1
    int64_t nsuper;     // nsb0 * nsb2 * nsb1
};

// Work lists over the super-bins, rebuilt by every set_points: each entry (super-bin, first
// sorted point, points, 0) is one piece of at most P points of one super-bin, the full pieces
// of all super-bins first, then the remainders, so that equal pieces are scheduled before the
// smaller ones and no super-bin's point count bounds a kernel's run time.  List 0 has pieces of
// kTcPass points (a pass of the tensor-core kernels), list 1 of spread_chunk(prec) points (a
// CTA of the CUDA-core spreading kernel).
constexpr int kTcPass = 128;

// angles of the points (sgl_points.cu): a binary32 first guess picks the nearest k pi / kRotK, whose
// cosine and sine come from a table; an arctangent series in binary64 adds the small rest
constexpr int kRotK = 2048;

// Tabulated windows of the double-float FP64 kernels: psi (even) and psi' (odd) of each axis on
// [0, q] as kWinNI pieces of degree kWinDeg in the offset from the piece's midpoint (psi is an
// entire function of x: sinh(b s) / s is a power series in s^2 = q^2 - x^2), fitted on the host in
// extended precision.  Layout [axis][psi, psi'][piece][coefficient, constant term first].
constexpr int kWinNI = 64, kWinDeg = 12;
constexpr int kWinTab = 3 * 2 * kWinNI * (kWinDeg + 1);
#ifndef SGL_SPREAD_CHUNK32
#define SGL_SPREAD_CHUNK32 1024
#endif
#ifndef SGL_SPREAD_CHUNK64
#define SGL_SPREAD_CHUNK64 128
#endif
__host__ __device__ inline int spread_chunk(int prec) { return prec == SGL_FP64 ? SGL_SPREAD_CHUNK64 : SGL_SPREAD_CHUNK32; }
// capacity of a list of pieces of P points for M points in nsuper super-bins
__host__ __device__ inline int64_t work_list_cap(int64_t M, int64_t nsuper, int P) {
    return (M < nsuper ? M : nsuper) + M / P + 1;
}

// Sets the thread-local message returned by sgl_last_error() and returns code.
sgl_status set_error(sgl_status code, const std::string &msg);

// One axis of the oversampled grid and its pruned 1-D FFT.
struct Axis {
    int n;          // conversion grid size (4B or 2B)
    int N;          // oversampled FFT length (2-3-5-smooth, even)
    int K;          // support half-width of eta on this axis (2B-2 or B-1)
    int rows;       // rows kept after the pruned inverse FFT (N if periodic)
    int first;      // first kept grid index (-q if windowed, 0 if periodic)
    bool windowed;  // rows = N/2 + 2q + 1 < N: only [-q, N/2+q] is stored
    double sigma;   // N / n
    double wpar;    // Kaiser-Bessel shape b, or Gaussian lambda
    int nrad;
    int rad[kMaxRadices];
    // device tables
    double2 *tw_d;  // exp(2 pi i m / N), m < N
    float2 *tw_f;
    float4 *tw_df;  // the same as double-float pairs (re hi, re lo, im hi, im lo)
    int *rev;       // digit-reversed slot of output index p after the DIF passes
    double *deconv; // 1 / Psihat(2 pi k / N), k = -K..K (index k + K)
    float2 *deconv_df; // the same as double-float pairs (h, l)
};

// Description of one batched, pruned 1-D DFT pass (see sgl_fft.cu).
struct FftPass {
    int N, nrad, rad[kMaxRadices];
    int sign;                       // +1: e^{+2 pi i kl/N}; -1: e^{-2 pi i kl/N}
    int L_in, in_first;             // input element e sits at position (e + in_first) mod N
    int L_out, out_first;           // output element e is position (e + out_first) mod N
    int64_t nb_outer, nb_inner;     // lines = outer x inner; inner lines are adjacent in memory
    int64_t in_so, in_si, in_se;    // input strides in complex elements
    int64_t out_so, out_si, out_se; // output strides in complex elements
    const double *elem_scale;       // optional factor per element index (input or output side, per launch)
    const double *line_scale;       // optional factor per flattened line index outer*nb_inner+inner
    const float2 *elem_scale_df;    // the same factors as double-float pairs (double-float passes)
    const float2 *line_scale_df;
    const void *tw;                 // twiddle table (double2 or float2)
    const void *tw64;               // the binary64 table (passes that fall back to binary64 arithmetic)
    const unsigned long long *scale_bits;   // double-float passes with binary64 input and output: bits of
                                            // max |input|; the pass runs on x 2^-E (E its exponent)
    const int *rev;
    // optional FP32 split-plane output (the tensor-core interpolation's layout): instead of out,
    // line i writes Re, Im of position (e - halo) mod N at planes[i pitch + e], planes[plane_n + i pitch + e],
    // e in [0, pitch)
    float *planes;
    int64_t plane_n;
    int pitch, halo;
    // symmetry-reduced passes (see sgl_fft.cu): element e of a line is read
    // at |e - mir_c| (mir_c = 0: plain), negated where e < mir_c and inner - mir_c is odd (the polar
    // parity (-1)^m); the line-scale index is offset by ls_off; with planes, line (outer, inner) is
    // plane row outer * plane_so + inner + plane_off
    int mir_c;
    int64_t ls_off, plane_so, plane_off;
};

struct Buffers {
    // conversions (FP64)
    double *P;        // polar matrices [B][K1+1][B]  (m >= 0; P_{-m} = (-1)^m P_m)
    double *costab;   // cos(m pi / 4B), m < 8B
    double *radv;     // radial values [sum_l 2B (B-l)]
    double *Kmat;     // radial conversion matrices [sum_l (K0+1)(B-l)]
    double2 *beta;    // [2B-1][K0+1][B]     beta_{kappa0, l, m}, kappa0 >= 0
    double2 *zeta;    // [K0+1][K1+1][2B-1]  zeta_{kappa0, kappa1, m}, kappa0, kappa1 >= 0
    double *linescale;// [(2K1+1)^2] d1[k1] d2[m]
    float2 *linescale_df; // the same as double-float pairs (h, l)
    // FFT work buffers (complex, precision of the plan)
    void *bufA, *bufB;
    size_t bufA_bytes, bufB_bytes;
    // points
    unsigned long long *r2max; // bit pattern of max |x|^2 (non-negative doubles order like integers)
    int *dev_flags;            // bit 0: non-finite coordinate seen
    double *u_tmp;             // [M][3] grid coordinates, input order
    double *u_sorted;          // [M][3] grid coordinates, bin order
    float4 *pts32;             // [M] bin order: (u0 - c0, u1 - c1, u2 - c2, cells c0 | c1 << 10 | c2 << 20 as bits)
    float2 *ys32;              // [M] bin order: the values to spread (FP32-mixed adjoint)
    int *perm;                 // sorted position -> input index
    int *bin_of, *rank_of;     // per input point
    int *bin_count, *bin_off;  // [nbins]
    int *scan_tmp;             // block sums
    int *piece_cnt, *piece_off;// [4 nsuper] full and remainder pieces per super-bin, both lists, and their scan
    int4 *work[2];             // work lists (see kTcPass): tensor-core passes, spreading chunks
    int *work_len;             // [2] entries in each list (written on the device)
    unsigned long long *df_max;// [3] FP64 plans: bits of max |grid|, max |values| and max |FFT input| (scales of the
                               // double-float passes)
    double *scalar;            // [1] device accumulator of small reductions (sgl_eta_l1)
    int *sched;                // [4] work counters of the persistent kernels (zeroed before each launch)
    double *wtab;              // [kWinTab] tabulated windows (FP64 plans)
    float2 *wtab_df;           // [kWinTab] the same as double-float pairs (FP64 plans)
    double2 *rot;              // [2 kRotK + 1] (cos, sin) of k pi / kRotK, k = -kRotK .. kRotK (point angles)
    float4 *rotf;              // [2 kRotK + 1] the same as double-float pairs (cos h, cos l, sin h, sin l)
    float4 *rec_tmp;           // [M] binary32 point records (as pts32) in input order
    // host-IO staging
    double *io_xyz, *io_coef, *io_vals, *io_grad, *io_out;
    // tensor-core interpolation (FP32-mixed): grid as planes Re, Im [rows0][rows1][pitch] with an azimuthal halo
    float *planes;
};

// Tensor-core interpolation layout on the azimuthal axis: a super-bin's 32 lanes start at
// grid index sb2 * S2 - tc_halo(q) (a multiple of 4, as a TMA box origin must be), and the
// planes store columns -tc_halo(q) ... pitch - tc_halo(q) - 1, wrapped.
__host__ __device__ inline int tc_halo(int q) { return 4 * ((q + 2) / 4); }
__host__ __device__ inline int tc_pitch(int N2) { return (N2 + 32 + 3) / 4 * 4; }

}  // namespace sgl

namespace sgl {
enum Stage {
    ST_POINTS = 0, ST_RADIAL_MATRIX, ST_RADIAL, ST_POLAR, ST_FFT_FWD, ST_INTERP,
    ST_SPREAD, ST_FFT_ADJ, ST_POLAR_ADJ, ST_RADIAL_ADJ, ST_GRAD, ST_TRIG, ST_COUNT
};
static_assert(ST_COUNT == SGL_NUM_STAGES, "stage list and SGL_NUM_STAGES disagree");
struct Profiler;   // CUDA-event bookkeeping (sgl_capi.cu)
struct InverseWork;   // work vectors of the inverse transform (sgl_inverse.cu)
void inverse_work_free(sgl_plan *p);
}  // namespace sgl

struct sgl_plan {
    int device;
    int num_sms;            // multiprocessors of the device (persistent kernels)
    int64_t launches;       // kernels launched (host-side count)
    sgl::Profiler *prof;    // non-NULL with SGL_FLAG_PROFILE
    sgl::InverseWork *inv;  // allocated by the first sgl_inverse / sgl_midpoint_guess
    cudaStream_t stream;
    // Binning of the points on a plan-owned stream (SGL_FLAG_OVERLAP_POINTS; NULL otherwise):
    // sgl_set_points forks it after everything already on `stream`; the first call that reads
    // the bins joins it.
    cudaStream_t side;
    cudaEvent_t ev_fork, ev_bins;
    bool bins_pending;
    int B, q, prec, window;
    unsigned flags;
    double sigma;
    int64_t M_max, M, Nc;
    int K0, K1;
    sgl::Axis ax[3];
    sgl::BinGeom bins;
    int64_t nbins;
    int64_t work_bytes;
    bool points_set;
    bool tc;                            // tensor-core kernels usable (planes and TMA map exist)
    bool tc_interp, tc_grad, tc_spread; // ... and chosen for the interpolation / gradient / spreading
    bool half_grid;                     // symmetry-reduced FFT passes (sgl_fft.cu)
    unsigned test_hooks;                // sgl_test_hooks: fault injection for tests (0 in normal use)
    long long wait_cycles;              // limit of the tensor-core kernels' waits (0: the default)
    alignas(64) unsigned char tc_map[2][128];   // TMA descriptors of b.planes (CUtensorMap): interpolation, gradient
    sgl::Buffers b;
};

namespace sgl {

// FFT work buffers shared by the plans of a batch (the plans run one after another on one stream).
struct SharedWork {
    void *bufA, *bufB;
    size_t bytesA, bytesB;
};
sgl_status plan_create_impl(sgl_plan **out, int B, int64_t M_max, int precision, int window, int q, double sigma,
                            unsigned flags, void *cuda_stream, const SharedWork *shared);
sgl_status plan_work_sizes(int B, int precision, int q, double sigma, size_t *bytesA, size_t *bytesB);

// ---- launchers (all asynchronous on plan->stream); return cudaGetLastError() ----
// rho on plan->stream (and, with `copy` non-NULL, a copy of the points there), then the binning
// of the points (read from xyz) on stream s
cudaError_t launch_points_rho(sgl_plan *p, const double *xyz, int64_t M, double *copy);
cudaError_t launch_points_bins(sgl_plan *p, const double *xyz, int64_t M, cudaStream_t s);
cudaError_t launch_radial_matrices(sgl_plan *p);
cudaError_t launch_radial_forward(sgl_plan *p, const double2 *coef);
cudaError_t launch_polar_forward(sgl_plan *p);
cudaError_t launch_trig_export(sgl_plan *p, double2 *eta);
cudaError_t launch_polar_adjoint(sgl_plan *p, const double2 *eta_full);
cudaError_t launch_radial_adjoint(sgl_plan *p, double2 *coef);
cudaError_t launch_max_abs(sgl_plan *p, const double *x, int64_t n, unsigned long long *bits);   // bits = max |x| (zeroed first)
cudaError_t launch_fft_forward(sgl_plan *p);    // zeta -> grid (bufA; b.planes when the interpolation is on tensor cores)
cudaError_t launch_fft_adjoint(sgl_plan *p);    // grid (bufA) -> eta' full support (bufB, FP64)
cudaError_t launch_interp(sgl_plan *p, double2 *vals);
cudaError_t launch_spread(sgl_plan *p, const double2 *vals);
cudaError_t launch_grad(sgl_plan *p, const double2 *gout, double *gxyz, double2 *vals);   // vals: NULL or the values too
// FP64 kernels (sgl_nufft64.cu), called by the three above for FP64 plans
cudaError_t launch_interp64(sgl_plan *p, double2 *vals);
cudaError_t launch_spread64(sgl_plan *p, const double2 *vals);
cudaError_t launch_grad64(sgl_plan *p, const double2 *gout, double *gxyz, double2 *vals);
// tensor-core interpolation / gradient (sgl_nufft_tc.cu)
bool tc_eligible(const sgl_plan *p);
void tc_choose(sgl_plan *p);
int64_t tc_plane_floats(const sgl_plan *p);
cudaError_t tc_make_tensor_map(sgl_plan *p);
cudaError_t launch_interp_tc(sgl_plan *p, double2 *vals);
cudaError_t launch_grad_tc(sgl_plan *p, const double2 *gout, double *gxyz, double2 *vals);

// cudaMalloc, or a failure injected by sgl_test_fail_alloc (every device allocation of the library)
cudaError_t device_malloc(void **p, size_t bytes);

// Host tables of the conversions for bandwidth B (sgl_capi.cu): the polar matrices P [B][B][B]
// ([m >= 0][kappa1][l]) and cos(m pi / 4B), m < 8B; leg is caller scratch of 2 B^3 doubles.  No
// heap use.
void conversion_tables(int B, double *P, double *costab, double *leg);

// explicit-pointer launchers (no plan) used by the allocation-free entry point
cudaError_t launch_max_radius_raw(cudaStream_t s, const double *xyz, int64_t M, unsigned long long *r2max, int *flags);
cudaError_t launch_trig_raw(cudaStream_t s, int B, const unsigned long long *r2max, const double *costab, const double *P,
                            double *radv, double *Kmat, double2 *beta, double2 *zeta, const double2 *coef, double2 *eta);

}  // namespace sgl

#define SGL_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t _e = (expr);                                                        \
        if (_e != cudaSuccess)                                                          \
            return sgl::set_error(SGL_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)
