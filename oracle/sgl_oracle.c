/*
 * sgl_oracle.c -- plain, slow, direct-summation oracle for the non-lattice
 * discrete SGL Fourier transform (NDSGLFT) of Wuelker, "Fast SGL Fourier
 * transforms for scattered data" (arXiv:1809.10786).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code with
 * the CUDA implementation and never calls it.
 *
 * What it computes (all straight from the definitions, O(M * Nc) work):
 *   - H_nlm(x) = N_nl R_nl(r) Y_lm(theta, phi)                 (Sect. 1, Def. of H_nlm)
 *       N_nl   = sqrt(2 (n-l-1)! / Gamma(n+1/2))
 *       R_nl   = L_{n-l-1}^{(l+1/2)}(r^2) r^l   (generalized Laguerre polynomial)
 *       Y_lm   = Q_lm P_lm(cos theta) e^{i m phi},
 *       Q_lm   = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)                (Sect. 6, spherical subtransform)
 *       P_lm   = associated Legendre function with the (-1)^m (Condon-Shortley)
 *                factor of its Rodrigues formula (Sect. 4); the same formula read for
 *                negative m gives P_{l,-m} = (-1)^m (l-m)!/(l+m)! P_lm.
 *   - coefficient order mu(n,l,m) = n(n-1)(2n-1)/6 + l(l+1) + m       (Sect. 1)
 *   - forward   f_i   = sum_mu c_mu H_mu(x_i)            (Def. NDSGLFT, f = Lambda fhat)
 *   - adjoint   c'_mu = sum_i conj(H_mu(x_i)) y_i        (Lambda^H, Sect. 1)
 *   - point gradient of the forward map:  grad_i = Re(conj(g_i) * grad_x f(x_i))
 *       d/dx L_k^{(a)}(x) = -L_{k-1}^{(a+1)}(x)  (textbook Laguerre identity)
 *       dP_lm(cos t)/dt   = (1/2){P_{l,m+1} - (l+m)(l-m+1) P_{l,m-1}}   (Sect. 7, Arfken-Weber identity)
 *       P_lm / sin t      = -(1/2m){P_{l+1,m+1} + (l-m+1)(l-m+2) P_{l+1,m-1}}  (Sect. 7, Lemma on P_lm/sqrt(1-x^2))
 *
 * Recurrences used:
 *   Laguerre  (k+1) L_{k+1} = (2k+1+a-x) L_k - (k+a) L_{k-1},  L_0 = 1, L_1 = 1+a-x
 *   Legendre  (l+1-m) P_{l+1,m} = (2l+1) x P_lm - (l+m) P_{l-1,m}       (Sect. 4, three-term recurrence)
 *             P_mm = (-1)^m (2m-1)!! (1-x^2)^{m/2},  P_{m+1,m} = (2m+1) x P_mm
 *
 * The arithmetic type is ORACLE_REAL (double by default).  The same source is also
 * built with long double, which gives an independent rounding of every step.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <unistd.h>

#ifndef ORACLE_REAL
#define ORACLE_REAL double
#endif
typedef ORACLE_REAL real;

#define R(x) ((real)(x))

static real r_sqrt(real x) { return sizeof(real) == sizeof(double) ? (real)sqrt((double)x) : (real)sqrtl((long double)x); }
static real r_cos(real x) { return sizeof(real) == sizeof(double) ? (real)cos((double)x) : (real)cosl((long double)x); }
static real r_sin(real x) { return sizeof(real) == sizeof(double) ? (real)sin((double)x) : (real)sinl((long double)x); }
static real r_atan2(real y, real x) { return sizeof(real) == sizeof(double) ? (real)atan2((double)y, (double)x) : (real)atan2l((long double)y, (long double)x); }
static real r_tgamma(real x) { return sizeof(real) == sizeof(double) ? (real)tgamma((double)x) : (real)tgammal((long double)x); }
static const real PI_R = R(3.14159265358979323846264338327950288L);

int64_t oracle_num_coeffs(int B) { return (int64_t)B * (B + 1) * (2 * B + 1) / 6; }

static inline int64_t mu_of(int n, int l, int m) { return (int64_t)n * (n - 1) * (2 * n - 1) / 6 + (int64_t)l * (l + 1) + m; }

static real factorial_loop(int k) { real f = 1; for (int j = 2; j <= k; ++j) f *= (real)j; return f; }

/* Per-point scratch: everything the basis and its derivatives need. */
typedef struct {
    int B;
    real r, ct, st, phi;      /* spherical coordinates, ct = cos theta, st = sin theta */
    real *NR;                 /* [B+1][B] : N_nl R_nl(r), index n*B + l            */
    real *dNR;                /* [B+1][B] : d/dr of N_nl R_nl(r)                   */
    real *NRr;                /* [B+1][B] : N_nl R_nl(r) / r  (finite for l >= 1)   */
    real *P;                  /* [B+2][B+2] : P_lm(cos theta), l <= B, 0 <= m <= l+1 */
    real *Q;                  /* [B+1][B+1] : Q_lm, m >= 0                           */
    real *cm, *sm;            /* cos(m phi), sin(m phi), m = 0..B                    */
    real *fact;               /* k! for k = 0..2B+3                                   */
} point_ws;

static void ws_alloc(point_ws *w, int B) {
    w->B = B;
    w->NR = (real *)calloc((size_t)(B + 1) * B, sizeof(real));
    w->dNR = (real *)calloc((size_t)(B + 1) * B, sizeof(real));
    w->NRr = (real *)calloc((size_t)(B + 1) * B, sizeof(real));
    w->P = (real *)calloc((size_t)(B + 2) * (B + 2), sizeof(real));
    w->Q = (real *)calloc((size_t)(B + 1) * (B + 1), sizeof(real));
    w->cm = (real *)calloc((size_t)B + 1, sizeof(real));
    w->sm = (real *)calloc((size_t)B + 1, sizeof(real));
    w->fact = (real *)calloc((size_t)2 * B + 4, sizeof(real));
    for (int k = 0; k < 2 * B + 4; ++k) w->fact[k] = factorial_loop(k);
    /* Q_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) for 0 <= m <= l <= B */
    for (int l = 0; l <= B; ++l)
        for (int m = 0; m <= l; ++m)
            w->Q[l * (B + 1) + m] = r_sqrt(R(2 * l + 1) / (R(4) * PI_R) * w->fact[l - m] / w->fact[l + m]);
}
static void ws_free(point_ws *w) { free(w->NR); free(w->dNR); free(w->NRr); free(w->P); free(w->Q); free(w->cm); free(w->sm); free(w->fact); }

#define PIDX(w, l, m) ((l) * ((w)->B + 2) + (m))

/* Generalized Laguerre L_k^{(a)}(x) for k = 0..K by the three-term recurrence. */
static void laguerre_all(int K, real a, real x, real *L) {
    L[0] = 1;
    if (K >= 1) L[1] = 1 + a - x;
    for (int k = 1; k < K; ++k) L[k + 1] = ((R(2 * k + 1) + a - x) * L[k] - (R(k) + a) * L[k - 1]) / R(k + 1);
}

/* Fill the workspace for point (x, y, z). */
static void ws_point(point_ws *w, real x, real y, real z) {
    const int B = w->B;
    real rho_xy = r_sqrt(x * x + y * y);
    w->r = r_sqrt(x * x + y * y + z * z);
    if (w->r > 0) { w->ct = z / w->r; w->st = rho_xy / w->r; } else { w->ct = 1; w->st = 0; }
    w->phi = r_atan2(y, x);
    const real r = w->r, t = r * r;
    real *L = (real *)malloc(sizeof(real) * (B + 1));
    real *L1 = (real *)malloc(sizeof(real) * (B + 1));
    for (int l = 0; l < B; ++l) {
        const real a = R(l) + R(0.5);
        const int K = B - l - 1;                /* n = l+1..B  <=>  k = n-l-1 = 0..K */
        laguerre_all(K, a, t, L);
        laguerre_all(K, a + 1, t, L1);
        real rl = 1, rlm1 = 1;                  /* r^l and r^(l-1) */
        for (int j = 0; j < l; ++j) rl *= r;
        for (int j = 0; j < l - 1; ++j) rlm1 *= r;
        for (int k = 0; k <= K; ++k) {
            const int n = l + 1 + k;
            const real N = r_sqrt(R(2) * w->fact[k] / r_tgamma(R(n) + R(0.5)));
            w->NR[n * B + l] = N * L[k] * rl;
            /* d/dr [L_k(r^2) r^l] = -2r L_{k-1}^{(a+1)}(r^2) r^l + l r^(l-1) L_k(r^2) */
            real d = (k >= 1 ? -R(2) * r * L1[k - 1] * rl : R(0));
            if (l >= 1) d += R(l) * rlm1 * L[k];
            w->dNR[n * B + l] = N * d;
            w->NRr[n * B + l] = (l >= 1) ? N * L[k] * rlm1 : R(0);
        }
    }
    free(L); free(L1);
    /* P_lm(cos theta) for 0 <= m <= l <= B (P_{l,m} = 0 for m > l). */
    memset(w->P, 0, sizeof(real) * (B + 2) * (B + 2));
    const real xi = w->ct, s = w->st;
    real pmm = 1;                               /* P_00 */
    for (int m = 0; m <= B; ++m) {
        if (m > 0) pmm = -R(2 * m - 1) * s * pmm;   /* P_mm = (-1)^m (2m-1)!! s^m */
        w->P[PIDX(w, m, m)] = pmm;
        if (m + 1 <= B) w->P[PIDX(w, m + 1, m)] = R(2 * m + 1) * xi * pmm;
        for (int l = m + 1; l < B; ++l)
            w->P[PIDX(w, l + 1, m)] = (R(2 * l + 1) * xi * w->P[PIDX(w, l, m)] - R(l + m) * w->P[PIDX(w, l - 1, m)]) / R(l + 1 - m);
    }
    for (int m = 0; m <= B; ++m) { w->cm[m] = r_cos(R(m) * w->phi); w->sm[m] = r_sin(R(m) * w->phi); }
}

/* P_{l,m} for any integer m (negative m through the Rodrigues formula), l <= B. */
static real P_any(const point_ws *w, int l, int m) {
    if (m > l || -m > l || l < 0) return 0;
    if (m >= 0) return w->P[PIDX(w, l, m)];
    const int am = -m;
    real sgn = (am & 1) ? -1 : 1;
    return sgn * w->fact[l - am] / w->fact[l + am] * w->P[PIDX(w, l, am)];
}

/* Y_lm (re, im), any m with |m| <= l < B. */
static void Y_lm(const point_ws *w, int l, int m, real *re, real *im) {
    const int am = m < 0 ? -m : m;
    /* Q_{l,m} P_{l,m} for m < 0 equals (-1)^m Q_{l,|m|} P_{l,|m|} (Rodrigues formula, negative order) */
    real v = w->Q[l * (w->B + 1) + am] * w->P[PIDX(w, l, am)];
    if (m < 0 && (am & 1)) v = -v;
    *re = v * w->cm[am];
    *im = (m < 0 ? -v : v) * w->sm[am];
}

/* ---------------------------------------------------------------- forward */
typedef struct {
    int B; int64_t i0, i1;
    const double *xyz, *coef; double *out; /* coef interleaved complex */
    const double *gout; double *grad;      /* gradient job */
    double *cacc;                          /* adjoint job: private accumulator [Nc*2] */
    const double *yv;
} job_t;

static void *fwd_worker(void *arg) {
    job_t *j = (job_t *)arg;
    const int B = j->B;
    point_ws w; ws_alloc(&w, B);
    for (int64_t i = j->i0; i < j->i1; ++i) {
        ws_point(&w, R(j->xyz[3 * i]), R(j->xyz[3 * i + 1]), R(j->xyz[3 * i + 2]));
        real fr = 0, fi = 0;
        for (int n = 1; n <= B; ++n)
            for (int l = 0; l < n; ++l) {
                const real rad = w.NR[n * B + l];
                for (int m = -l; m <= l; ++m) {
                    real yr, yi; Y_lm(&w, l, m, &yr, &yi);
                    const int64_t mu = mu_of(n, l, m);
                    const real cr = R(j->coef[2 * mu]), ci = R(j->coef[2 * mu + 1]);
                    const real hr = rad * yr, hi = rad * yi;
                    fr += cr * hr - ci * hi;
                    fi += cr * hi + ci * hr;
                }
            }
        j->out[2 * i] = (double)fr; j->out[2 * i + 1] = (double)fi;
    }
    ws_free(&w);
    return NULL;
}

static void *adj_worker(void *arg) {
    job_t *j = (job_t *)arg;
    const int B = j->B;
    const int64_t Nc = oracle_num_coeffs(B);
    real *acc = (real *)calloc((size_t)Nc * 2, sizeof(real));
    point_ws w; ws_alloc(&w, B);
    for (int64_t i = j->i0; i < j->i1; ++i) {
        ws_point(&w, R(j->xyz[3 * i]), R(j->xyz[3 * i + 1]), R(j->xyz[3 * i + 2]));
        const real vr = R(j->yv[2 * i]), vi = R(j->yv[2 * i + 1]);
        for (int n = 1; n <= B; ++n)
            for (int l = 0; l < n; ++l) {
                const real rad = w.NR[n * B + l];
                for (int m = -l; m <= l; ++m) {
                    real yr, yi; Y_lm(&w, l, m, &yr, &yi);
                    const int64_t mu = mu_of(n, l, m);
                    const real hr = rad * yr, hi = -rad * yi;     /* conj(H) */
                    acc[2 * mu] += hr * vr - hi * vi;
                    acc[2 * mu + 1] += hr * vi + hi * vr;
                }
            }
    }
    for (int64_t k = 0; k < 2 * Nc; ++k) j->cacc[k] = (double)acc[k];
    free(acc);
    ws_free(&w);
    return NULL;
}

static void *grad_worker(void *arg) {
    job_t *j = (job_t *)arg;
    const int B = j->B;
    point_ws w; ws_alloc(&w, B);
    for (int64_t i = j->i0; i < j->i1; ++i) {
        ws_point(&w, R(j->xyz[3 * i]), R(j->xyz[3 * i + 1]), R(j->xyz[3 * i + 2]));
        /* df/dr, (1/r) df/dtheta, (1/(r sin theta)) df/dphi, each complex */
        real dr_r = 0, dr_i = 0, dt_r = 0, dt_i = 0, dp_r = 0, dp_i = 0;
        for (int n = 1; n <= B; ++n)
            for (int l = 0; l < n; ++l) {
                const real drad = w.dNR[n * B + l], radr = w.NRr[n * B + l];
                for (int m = -l; m <= l; ++m) {
                    const int64_t mu = mu_of(n, l, m);
                    const real cr = R(j->coef[2 * mu]), ci = R(j->coef[2 * mu + 1]);
                    const int am = m < 0 ? -m : m;
                    const real ph_r = w.cm[am], ph_i = (m < 0 ? -w.sm[am] : w.sm[am]);   /* e^{i m phi} */
                    /* Q_{l,m} for any sign of m */
                    const real Qlm = r_sqrt(R(2 * l + 1) / (R(4) * PI_R) * w.fact[l - m] / w.fact[l + m]);
                    const real Plm = P_any(&w, l, m);
                    /* angular derivative dP_lm(cos t)/dt = (1/2){P_{l,m+1} - (l+m)(l-m+1) P_{l,m-1}} */
                    const real dP = R(0.5) * (P_any(&w, l, m + 1) - R(l + m) * R(l - m + 1) * P_any(&w, l, m - 1));
                    /* P_lm / sin t = -(1/2m){P_{l+1,m+1} + (l-m+1)(l-m+2) P_{l+1,m-1}}, m != 0 */
                    real Ps = 0;
                    if (m != 0) Ps = -(P_any(&w, l + 1, m + 1) + R(l - m + 1) * R(l - m + 2) * P_any(&w, l + 1, m - 1)) / (R(2) * R(m));
                    /* c * e^{i m phi} */
                    const real ar = cr * ph_r - ci * ph_i, ai = cr * ph_i + ci * ph_r;
                    const real yv = Qlm * Plm, dyt = Qlm * dP, ys = Qlm * Ps;
                    dr_r += drad * yv * ar; dr_i += drad * yv * ai;
                    dt_r += radr * dyt * ar; dt_i += radr * dyt * ai;
                    /* d/dphi gives the factor i m:  i m (ar + i ai) = -m ai + i m ar */
                    dp_r += radr * ys * (-R(m) * ai); dp_i += radr * ys * (R(m) * ar);
                }
            }
        const real st = w.st, ct = w.ct, cp = r_cos(w.phi), sp = r_sin(w.phi);
        /* unit vectors r^, theta^, phi^ */
        const real er[3] = {st * cp, st * sp, ct}, et[3] = {ct * cp, ct * sp, -st}, ep[3] = {-sp, cp, 0};
        const real gr = R(j->gout[2 * i]), gi = R(j->gout[2 * i + 1]);
        for (int d = 0; d < 3; ++d) {
            const real vr = dr_r * er[d] + dt_r * et[d] + dp_r * ep[d];
            const real vi = dr_i * er[d] + dt_i * et[d] + dp_i * ep[d];
            j->grad[3 * i + d] = (double)(gr * vr + gi * vi);   /* Re(conj(g) v) */
        }
    }
    ws_free(&w);
    return NULL;
}

static int pick_threads(int nthreads, int64_t M) {
    if (nthreads <= 0) { long c = sysconf(_SC_NPROCESSORS_ONLN); nthreads = c > 0 ? (int)c : 1; }
    if (nthreads > M) nthreads = (int)(M > 0 ? M : 1);
    if (nthreads > 256) nthreads = 256;
    return nthreads;
}

static void run_jobs(void *(*fn)(void *), job_t *jobs, int T) {
    pthread_t th[256];
    for (int t = 1; t < T; ++t) pthread_create(&th[t], NULL, fn, &jobs[t]);
    fn(&jobs[0]);
    for (int t = 1; t < T; ++t) pthread_join(th[t], NULL);
}

static void split(job_t *jobs, int T, int64_t M) {
    for (int t = 0; t < T; ++t) { jobs[t].i0 = M * t / T; jobs[t].i1 = M * (t + 1) / T; }
}

/* f = Lambda c.  xyz [M][3], coef complex [Nc], out complex [M].  Returns threads used. */
int oracle_forward(int B, int64_t M, const double *xyz, const double *coef, double *out, int nthreads) {
    if (B < 1 || M < 0) return -1;
    if (M == 0) return 0;
    const int T = pick_threads(nthreads, M);
    job_t jobs[256]; memset(jobs, 0, sizeof(jobs));
    for (int t = 0; t < T; ++t) { jobs[t].B = B; jobs[t].xyz = xyz; jobs[t].coef = coef; jobs[t].out = out; }
    split(jobs, T, M);
    run_jobs(fwd_worker, jobs, T);
    return T;
}

/* c' = Lambda^H y.  y complex [M], out complex [Nc]. */
int oracle_adjoint(int B, int64_t M, const double *xyz, const double *y, double *out, int nthreads) {
    if (B < 1 || M < 0) return -1;
    const int64_t Nc = oracle_num_coeffs(B);
    memset(out, 0, sizeof(double) * 2 * Nc);
    if (M == 0) return 0;
    const int T = pick_threads(nthreads, M);
    job_t jobs[256]; memset(jobs, 0, sizeof(jobs));
    double *acc = (double *)calloc((size_t)T * 2 * Nc, sizeof(double));
    for (int t = 0; t < T; ++t) { jobs[t].B = B; jobs[t].xyz = xyz; jobs[t].yv = y; jobs[t].cacc = acc + (size_t)t * 2 * Nc; }
    split(jobs, T, M);
    run_jobs(adj_worker, jobs, T);
    for (int t = 0; t < T; ++t)
        for (int64_t k = 0; k < 2 * Nc; ++k) out[k] += acc[(size_t)t * 2 * Nc + k];
    free(acc);
    return T;
}

/* grad [M][3] = Re(conj(g_i) grad_x f(x_i)), f = Lambda c.  g complex [M]. */
int oracle_grad_points(int B, int64_t M, const double *xyz, const double *coef, const double *g, double *grad, int nthreads) {
    if (B < 1 || M < 0) return -1;
    if (M == 0) return 0;
    const int T = pick_threads(nthreads, M);
    job_t jobs[256]; memset(jobs, 0, sizeof(jobs));
    for (int t = 0; t < T; ++t) { jobs[t].B = B; jobs[t].xyz = xyz; jobs[t].coef = coef; jobs[t].gout = g; jobs[t].grad = grad; }
    split(jobs, T, M);
    run_jobs(grad_worker, jobs, T);
    return T;
}

/* All Nc basis values H_mu(x) at one point; out complex [Nc]. */
int oracle_basis(int B, const double *x, double *out) {
    if (B < 1) return -1;
    point_ws w; ws_alloc(&w, B);
    ws_point(&w, R(x[0]), R(x[1]), R(x[2]));
    for (int n = 1; n <= B; ++n)
        for (int l = 0; l < n; ++l)
            for (int m = -l; m <= l; ++m) {
                real yr, yi; Y_lm(&w, l, m, &yr, &yi);
                const int64_t mu = mu_of(n, l, m);
                out[2 * mu] = (double)(w.NR[n * B + l] * yr);
                out[2 * mu + 1] = (double)(w.NR[n * B + l] * yi);
            }
    ws_free(&w);
    return 0;
}

/* Generalized Laguerre values L_k^{(a)}(x), k = 0..K (exposed for closed-form pins). */
int oracle_laguerre(int K, double a, double x, double *out) {
    real *L = (real *)malloc(sizeof(real) * (K + 2));
    laguerre_all(K, R(a), R(x), L);
    for (int k = 0; k <= K; ++k) out[k] = (double)L[k];
    free(L);
    return 0;
}

/* Index maps (Sect. 1): (n,l,m) -> mu and back, by search over n (no closed form). */
int64_t oracle_mu(int n, int l, int m) { return mu_of(n, l, m); }
int oracle_nlm(int64_t mu, int *n, int *l, int *m) {
    if (mu < 0) return -1;
    int nn = 1;
    while (mu_of(nn + 1, 0, 0) <= mu) ++nn;
    int64_t rem = mu - mu_of(nn, 0, 0);
    int ll = 0;
    while ((int64_t)(ll + 1) * (ll + 1) <= rem) ++ll;
    *n = nn; *l = ll; *m = (int)(rem - (int64_t)ll * (ll + 1));
    return 0;
}

/* size of the arithmetic type this build uses (8: double, 10/16: long double) */
int oracle_real_bytes(void) { return (int)sizeof(real); }

/* N_nl R_nl(r) for 1 <= n <= B, 0 <= l < n; out [B+1][B] (index n*B + l), zero elsewhere. */
int oracle_radial(int B, double r, double *out) {
    if (B < 1) return -1;
    point_ws w; ws_alloc(&w, B);
    ws_point(&w, R(0), R(0), R(r));
    for (int k = 0; k < (B + 1) * B; ++k) out[k] = (double)w.NR[k];
    ws_free(&w);
    return 0;
}

/* Q_lm P_lm(cos theta) for 0 <= m <= l < B; out [B][B] (index l*B + m), zero for m > l. */
int oracle_legendre(int B, double theta, double *out) {
    if (B < 1) return -1;
    point_ws w; ws_alloc(&w, B);
    ws_point(&w, R(sin(theta)), R(0), R(cos(theta)));
    for (int l = 0; l < B; ++l)
        for (int m = 0; m < B; ++m)
            out[l * B + m] = (m <= l) ? (double)(w.Q[l * (B + 1) + m] * w.P[PIDX(&w, l, m)]) : 0.0;
    ws_free(&w);
    return 0;
}
