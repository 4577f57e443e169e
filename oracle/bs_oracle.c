/*
 * bs_oracle.c -- plain FP64 CPU oracle for the Ewald-split periodic
 * Biot-Savart velocity (and streamfunction) on closed or periodic vortex
 * filaments, after J. I. Polanco, "Fast and accurate evaluation of
 * Biot-Savart integrals over spatial curves in periodic domains"
 * (arXiv:2406.07366).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code with the CUDA library.
 *
 * Design rule: every routine is the plain definition written out, in double
 * precision, with no blocking, fusion or reordering beyond the definition.
 *   - Gauss-Legendre rule: Newton iteration on the three-term Legendre
 *     recurrence (Sec. 2.6, Eq. line_integral_quadrature).
 *   - Curve: chord-length parameter and periodic B-spline of order k, basis
 *     evaluated by the Cox-de Boor recursion, coefficients from the dense
 *     collocation system solved by Gaussian elimination with partial
 *     pivoting (Appendix B).
 *   - Short range: brute force over every source point, either the minimum
 *     image with a cut-off r_c (the build's own split, Eq.
 *     velocity_shortrange) or all 27 images with no cut-off (the converged
 *     split used as ground truth).
 *   - Long range: direct Fourier sum over a cube of modes (Eqs.
 *     vorticity_fourier_coefs, velocity_longrange_physical), each 1-D phase
 *     from a direct cos/sin call; no NUFFT.
 *   - Self term: Eqs. streamfunction_longrange_self / velocity_longrange_self
 *     on the quadrature points of the two segments adjacent to the node.
 *   - Local term: Eqs. BS_local and streamfunction_local.
 * Sums over many terms use Neumaier compensated summation.
 *
 * Readings of the paper this file takes (where it is silent):
 *   - l^- and l^+ are arc lengths of the adjacent segments, integrated with
 *     the same Q-point rule.
 *   - The omitted portion C_0 is the unwrapped pair of segments adjacent to
 *     the node; every periodic image of C_0 is an ordinary source.
 *   - An unclosed curve with s(tau+T) = s(tau) + n L is interpolated through
 *     its periodic part s(tau) - n L tau / T; the linear part is added back.
 *   - A source coinciding exactly with a target (r == 0) contributes nothing.
 *
 * Pins (tests/test_oracle_pins.py): Gauss-Legendre against numpy, splines
 * against scipy's periodic interpolants, exact net vorticity of closed
 * curves, arc length and curvature of circles, the small-argument series of
 * g^(f), invariance of the total in alpha, the alpha = 0 limit, the
 * open-space limit, the Kelvin ring speed, and zero velocity on symmetric
 * straight-line lattices.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------ */
/* Neumaier compensated summation                                      */
/* ------------------------------------------------------------------ */
typedef struct { double s, c; } csum;

static inline void cs_add(csum* a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static inline double cs_get(const csum* a) { return a->s + a->c; }

void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int or_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Gauss-Legendre rule on [0, 1] (Sec. 2.6): nodes h_i, weights w_i,  */
/* sum w_i = 1.  Newton iteration on P_Q from the Legendre recurrence  */
/* (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}.                           */
/* ------------------------------------------------------------------ */
static void legendre_pd(int n, double x, double* p, double* dp)
{
    double p0 = 1.0, p1 = x;
    if (n == 0) { *p = 1.0; *dp = 0.0; return; }
    for (int k = 1; k < n; k++) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *p = p1;
    *dp = n * (x * p1 - p0) / (x * x - 1.0);
}

int or_gauss_legendre(int Q, double* h, double* w)
{
    if (Q < 1 || Q > 64) return -1;
    for (int i = 0; i < Q; i++) {
        double x = cos(OR_PI * (i + 0.75) / (Q + 0.5));
        for (int it = 0; it < 100; it++) {
            double p, dp;
            legendre_pd(Q, x, &p, &dp);
            double dx = p / dp;
            x -= dx;
            if (fabs(dx) < 1e-17) break;
        }
        double p, dp;
        legendre_pd(Q, x, &p, &dp);
        /* x decreases with i, so h = (1 - x)/2 increases with i. */
        h[i] = 0.5 * (1.0 - x);
        w[i] = 1.0 / ((1.0 - x * x) * dp * dp);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Periodic B-splines (Appendix B)                                     */
/* Knots t_l = tau_{l mod n} + floor(l / n) T; B_{l,r} has support     */
/* [t_l, t_{l+r}] and is evaluated by the Cox-de Boor recursion.       */
/* ------------------------------------------------------------------ */
typedef struct {
    const double* t;
    long n;
    double T;
} kseq;

static long floor_div(long a, long b)
{
    long q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q--;
    return q;
}

static long pmod(long a, long b) { return a - floor_div(a, b) * b; }

static double knot(const kseq* K, long l)
{
    long p = floor_div(l, K->n);
    return K->t[l - p * K->n] + (double)p * K->T;
}

/* der-th derivative of B_{l,r} at x. */
static double bspl(const kseq* K, long l, int r, double x, int der)
{
    if (der > 0) {
        if (r == 1) return 0.0;
        double a = knot(K, l + r - 1) - knot(K, l);
        double b = knot(K, l + r) - knot(K, l + 1);
        double s = 0.0;
        if (a > 0.0) s += bspl(K, l, r - 1, x, der - 1) / a;
        if (b > 0.0) s -= bspl(K, l + 1, r - 1, x, der - 1) / b;
        return (r - 1) * s;
    }
    if (r == 1) return (knot(K, l) <= x && x < knot(K, l + 1)) ? 1.0 : 0.0;
    double a = knot(K, l + r - 1) - knot(K, l);
    double b = knot(K, l + r) - knot(K, l + 1);
    double s = 0.0;
    if (a > 0.0) s += (x - knot(K, l)) / a * bspl(K, l, r - 1, x, 0);
    if (b > 0.0) s += (knot(K, l + r) - x) / b * bspl(K, l + 1, r - 1, x, 0);
    return s;
}

/* Solve A X = B in place (A n x n row-major, B n x m), partial pivoting. */
static int dense_solve(long n, double* A, long m, double* B)
{
    for (long c = 0; c < n; c++) {
        long piv = c;
        double best = fabs(A[c * n + c]);
        for (long r = c + 1; r < n; r++) {
            double v = fabs(A[r * n + c]);
            if (v > best) { best = v; piv = r; }
        }
        if (best == 0.0) return -1;
        if (piv != c) {
            for (long k = 0; k < n; k++) {
                double t = A[c * n + k]; A[c * n + k] = A[piv * n + k]; A[piv * n + k] = t;
            }
            for (long k = 0; k < m; k++) {
                double t = B[c * m + k]; B[c * m + k] = B[piv * m + k]; B[piv * m + k] = t;
            }
        }
        for (long r = c + 1; r < n; r++) {
            double f = A[r * n + c] / A[c * n + c];
            if (f == 0.0) continue;
            for (long k = c; k < n; k++) A[r * n + k] -= f * A[c * n + k];
            for (long k = 0; k < m; k++) B[r * m + k] -= f * B[c * m + k];
        }
    }
    for (long c = n - 1; c >= 0; c--) {
        for (long k = 0; k < m; k++) {
            double s = B[c * m + k];
            for (long j = c + 1; j < n; j++) s -= A[c * n + j] * B[j * m + k];
            B[c * m + k] = s / A[c * n + c];
        }
    }
    return 0;
}

/* Coefficients d (n x 3) of the periodic order-k spline through p at tau. */
static int spline_fit(const kseq* K, int k, const double* p, double* d)
{
    long n = K->n;
    double* A = (double*)calloc((size_t)(n * n), sizeof(double));
    if (!A) return -2;
    for (long i = 0; i < n; i++) {
        double x = K->t[i];
        for (long l = i - k + 1; l <= i; l++)
            A[i * n + pmod(l, n)] += bspl(K, l, k, x, 0);
    }
    memcpy(d, p, (size_t)(n * 3) * sizeof(double));
    int rc = dense_solve(n, A, 3, d);
    free(A);
    return rc;
}

/* der-th derivative of the spline at x, where t_i <= x < t_{i+1}. */
static void spline_eval(const kseq* K, int k, const double* d, long i, double x, int der, double out[3])
{
    out[0] = out[1] = out[2] = 0.0;
    for (long l = i - k + 1; l <= i; l++) {
        double b = bspl(K, l, k, x, der);
        long c = pmod(l, K->n);
        out[0] += d[3 * c + 0] * b;
        out[1] += d[3 * c + 1] * b;
        out[2] += d[3 * c + 2] * b;
    }
}

static double norm3(const double a[3]) { return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Chord-length parameter of one filament (Appendix B): tau_0 = 0,
 * tau_j = tau_{j-1} + |s_j - s_{j-1}|, T = tau_{n-1} + |s_0 + shift - s_{n-1}|. */
static double chord_params(long n, const double* s, const double* shift, double* tau)
{
    tau[0] = 0.0;
    for (long j = 1; j < n; j++) {
        double d[3] = { s[3 * j] - s[3 * j - 3], s[3 * j + 1] - s[3 * j - 2], s[3 * j + 2] - s[3 * j - 1] };
        tau[j] = tau[j - 1] + norm3(d);
    }
    double d[3] = { s[0] + shift[0] - s[3 * n - 3], s[1] + shift[1] - s[3 * n - 2], s[2] + shift[2] - s[3 * n - 1] };
    return tau[n - 1] + norm3(d);
}

/* Fit one filament: returns tau (n), T, coefficients d (n x 3) of the
 * periodic part p = s - shift tau / T. */
static int fit_filament(long n, const double* s, const double* shift, int k, double* tau, double* T, double* d)
{
    *T = chord_params(n, s, shift, tau);
    double* p = (double*)malloc((size_t)(n * 3) * sizeof(double));
    if (!p) return -2;
    for (long j = 0; j < n; j++)
        for (int c = 0; c < 3; c++) p[3 * j + c] = s[3 * j + c] - shift[c] * tau[j] / *T;
    kseq K = { tau, n, *T };
    int rc = spline_fit(&K, k, p, d);
    free(p);
    return rc;
}

/*
 * Evaluate the fitted curve of one filament (nodes s, n x 3; shift = n_l L)
 * at parameters x (m values, any real), derivative order der in {0,1,2,3}.
 * Used by the pin tests against scipy.
 */
int or_spline_eval(long n, const double* s, const double* shift, int k, long m, const double* x, int der,
                   double* out, double* tau_out, double* T_out)
{
    double* tau = (double*)malloc((size_t)n * sizeof(double));
    double* d = (double*)malloc((size_t)(n * 3) * sizeof(double));
    double T;
    int rc = fit_filament(n, s, shift, k, tau, &T, d);
    if (rc == 0) {
        kseq K = { tau, n, T };
        for (long q = 0; q < m; q++) {
            double xr = x[q] - floor(x[q] / T) * T; /* reduce into [0, T) */
            long per = (long)floor(x[q] / T);
            long i = n - 1;
            for (long j = 0; j < n - 1; j++)
                if (tau[j] <= xr && xr < tau[j + 1]) { i = j; break; }
            double v[3];
            spline_eval(&K, k, d, i, xr, der, v);
            for (int c = 0; c < 3; c++) {
                if (der == 0) v[c] += shift[c] * (xr / T) + shift[c] * per;
                else if (der == 1) v[c] += shift[c] / T;
                out[3 * q + c] = v[c];
            }
        }
        if (tau_out) memcpy(tau_out, tau, (size_t)n * sizeof(double));
        if (T_out) *T_out = T;
    }
    free(tau);
    free(d);
    return rc;
}

/*
 * Geometry of all filaments (Sec. 2.6, Eq. line_integral_quadrature;
 * Sec. 3.3, Eq. vorticity_fourier_coefs; Sec. 2.3, Eq. BS_local):
 *   qX  (N*Q x 3): quadrature points s(tau_j + h_i dtau_j), unwrapped
 *   qq  (N*Q x 3): charges w_i dtau_j s'(tau) (tau-derivative)
 *   sp  (N x 3)  : unit tangent at the node
 *   sxs (N x 3)  : s' x s'' in arc length, = (sdot x sddot) / |sdot|^3
 *   lm, lp (N)   : arc lengths of the segments before / after the node
 *   tau (N), Tf (nfil): parameters
 * Point (j, i) is stored at index j*Q + i, j the global node index of the
 * segment start.  shift (nfil x 3) = n_l L of each filament.
 */
int or_geometry(long nfil, const int64_t* off, const double* nodes, const double* shift, int k, int Q,
                double* qX, double* qq, double* sp, double* sxs, double* lm, double* lp,
                double* tau_all, double* Tf)
{
    double h[64], w[64];
    if (or_gauss_legendre(Q, h, w) != 0) return -1;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (long f = 0; f < nfil; f++) {
        long n = off[f + 1] - off[f];
        const double* s = nodes + 3 * off[f];
        const double* sh = shift + 3 * f;
        if (n < k) {
#pragma omp atomic write
            err = -3;
            continue;
        }
        double* tau = tau_all + off[f];
        double* d = (double*)malloc((size_t)(n * 3) * sizeof(double));
        double* len = (double*)malloc((size_t)n * sizeof(double));
        double T;
        if (fit_filament(n, s, sh, k, tau, &T, d) != 0) {
#pragma omp atomic write
            err = -4;
            free(d);
            free(len);
            continue;
        }
        Tf[f] = T;
        kseq K = { tau, n, T };
        double drift[3] = { sh[0] / T, sh[1] / T, sh[2] / T };
        for (long j = 0; j < n; j++) {
            long g = off[f] + j;
            double dtau = (j < n - 1 ? tau[j + 1] : T) - tau[j];
            csum L = { 0, 0 };
            for (int i = 0; i < Q; i++) {
                double x = tau[j] + h[i] * dtau;
                double p0[3], p1[3];
                spline_eval(&K, k, d, j, x, 0, p0);
                spline_eval(&K, k, d, j, x, 1, p1);
                for (int c = 0; c < 3; c++) {
                    p0[c] += drift[c] * x;
                    p1[c] += drift[c];
                }
                long qi = g * Q + i;
                for (int c = 0; c < 3; c++) {
                    qX[3 * qi + c] = p0[c];
                    qq[3 * qi + c] = w[i] * dtau * p1[c];
                }
                cs_add(&L, w[i] * dtau * norm3(p1));
            }
            len[j] = cs_get(&L);
            double d1[3], d2[3], bxs[3];
            spline_eval(&K, k, d, j, tau[j], 1, d1);
            spline_eval(&K, k, d, j, tau[j], 2, d2);
            for (int c = 0; c < 3; c++) d1[c] += drift[c];
            double sn = norm3(d1);
            cross3(d1, d2, bxs);
            for (int c = 0; c < 3; c++) {
                sp[3 * g + c] = d1[c] / sn;
                sxs[3 * g + c] = bxs[c] / (sn * sn * sn);
            }
        }
        for (long j = 0; j < n; j++) {
            long g = off[f] + j;
            lp[g] = len[j];
            lm[g] = len[(j + n - 1) % n];
        }
        free(d);
        free(len);
    }
    return err;
}

/* ------------------------------------------------------------------ */
/* Local terms, Eqs. BS_local and streamfunction_local                 */
/* ------------------------------------------------------------------ */
void or_local(long N, const double* sp, const double* sxs, const double* lm, const double* lp,
              double kappa, double a, double delta, double* v, double* psi)
{
    for (long j = 0; j < N; j++) {
        double lg = log(2.0 * sqrt(lm[j] * lp[j]) / a);
        for (int c = 0; c < 3; c++) {
            v[3 * j + c] = kappa / (4.0 * OR_PI) * sxs[3 * j + c] * (lg - delta);
            if (psi) psi[3 * j + c] = kappa * sp[3 * j + c] / (2.0 * OR_PI) * (lg - (delta - 1.0));
        }
    }
}

/*
 * Local terms with the local segments subdivided (Sec. 5.2): the Taylor
 * expansions of Eqs. BS_local and streamfunction_local are applied only on
 * the central portions of the two local segments, the fraction frac of each
 * next to node j (l^- and l^+ their arc lengths, Q-point Gauss-Legendre),
 * and the remaining portions of the two segments are integrated with the
 * plain Biot-Savart kernel.  The paper does not say how; here each remaining
 * portion is cut, from the node outwards, into pieces of the segment
 * fraction [f, 2f], [2f, 4f], ..., [2^m f, 1] (a 1/r^2 integrand varies by at
 * most 4x on a piece), with Q-point Gauss-Legendre on each:
 *   v   += kappa/4pi sum w (s(x) - s_j) x s'(x) / |s(x) - s_j|^3,
 *   psi += kappa/4pi sum w s'(x) / |s(x) - s_j|.
 * frac = 1 gives or_local.  Per node: v, psi (N x 3).
 */
int or_local_sub(long nfil, const int64_t* off, const double* nodes, const double* shift, int k, int Q, double frac,
                 double kappa, double a, double delta, double* v, double* psi)
{
    double h[64], w[64];
    if (or_gauss_legendre(Q, h, w) != 0) return -1;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (long f = 0; f < nfil; f++) {
        long n = off[f + 1] - off[f];
        const double* s = nodes + 3 * off[f];
        const double* sh = shift + 3 * f;
        double* tau = (double*)malloc((size_t)n * sizeof(double));
        double* d = (double*)malloc((size_t)(n * 3) * sizeof(double));
        double T;
        if (n < k || fit_filament(n, s, sh, k, tau, &T, d) != 0) {
#pragma omp atomic write
            err = -4;
            free(tau);
            free(d);
            continue;
        }
        kseq K = { tau, n, T };
        const double drift[3] = { sh[0] / T, sh[1] / T, sh[2] / T };
        for (long j = 0; j < n; j++) {
            long g = off[f] + j;
            long jm = (j + n - 1) % n;
            const double t0 = tau[j];
            const double hp = (j < n - 1 ? tau[j + 1] : T) - t0;      /* segment j */
            const double tm = tau[jm];
            const double hm = (jm < n - 1 ? tau[jm + 1] : T) - tm;    /* segment j-1 */
            /* position (unwrapped) and tangent at parameter x of segment seg */
            double sj[3];
            for (int c = 0; c < 3; c++) sj[c] = s[3 * j + c];
            csum lp = { 0, 0 }, lm = { 0, 0 };
            csum av[3] = { { 0, 0 }, { 0, 0 }, { 0, 0 } }, ap[3] = { { 0, 0 }, { 0, 0 }, { 0, 0 } };
            /* pieces: central of j and of j-1, then the geometric pieces of the
             * remaining portions (fractions measured from the node) */
            double pa[2 * 64 + 2], pb[2 * 64 + 2];
            int pseg[2 * 64 + 2], pkind[2 * 64 + 2], np = 0;
            pa[np] = 0.0; pb[np] = frac; pseg[np] = 0; pkind[np++] = 0;
            pa[np] = 0.0; pb[np] = frac; pseg[np] = 1; pkind[np++] = 1;
            for (int sd = 0; sd < 2; sd++) {
                double x0 = frac;
                while (x0 < 1.0 && np < 2 * 64) {
                    double x1 = 2.0 * x0 < 1.0 ? 2.0 * x0 : 1.0;
                    pa[np] = x0; pb[np] = x1; pseg[np] = sd; pkind[np++] = 2;
                    x0 = x1;
                }
            }
            for (int part = 0; part < np; part++) {
                /* segment j runs away from the node, segment j-1 towards it */
                long seg = pseg[part] == 0 ? j : jm;
                double lo, len;
                if (pseg[part] == 0) { lo = t0 + pa[part] * hp; len = (pb[part] - pa[part]) * hp; }
                else { lo = tm + (1.0 - pb[part]) * hm; len = (pb[part] - pa[part]) * hm; }
                for (int i = 0; i < Q; i++) {
                    double x = lo + h[i] * len;
                    double p0[3], p1[3];
                    spline_eval(&K, k, d, seg, x, 0, p0);
                    spline_eval(&K, k, d, seg, x, 1, p1);
                    for (int c = 0; c < 3; c++) {
                        p0[c] += drift[c] * x;
                        p1[c] += drift[c];
                    }
                    /* the segment before node 0 ends at s_0 + shift */
                    if (seg == jm && j == 0)
                        for (int c = 0; c < 3; c++) p0[c] -= sh[c];
                    double wt = w[i] * len;
                    if (pkind[part] == 0) cs_add(&lp, wt * norm3(p1));
                    else if (pkind[part] == 1) cs_add(&lm, wt * norm3(p1));
                    else {
                        double r[3] = { p0[0] - sj[0], p0[1] - sj[1], p0[2] - sj[2] };
                        double rr = norm3(r);
                        double q[3] = { wt * p1[0], wt * p1[1], wt * p1[2] };
                        double cr[3];
                        cross3(r, q, cr);
                        for (int c = 0; c < 3; c++) {
                            cs_add(&av[c], cr[c] / (rr * rr * rr));
                            cs_add(&ap[c], q[c] / rr);
                        }
                    }
                }
            }
            double d1[3], d2[3], bxs[3];
            spline_eval(&K, k, d, j, tau[j], 1, d1);
            spline_eval(&K, k, d, j, tau[j], 2, d2);
            for (int c = 0; c < 3; c++) d1[c] += drift[c];
            double sn = norm3(d1);
            cross3(d1, d2, bxs);
            double lg = log(2.0 * sqrt(cs_get(&lm) * cs_get(&lp)) / a);
            for (int c = 0; c < 3; c++) {
                v[3 * g + c] = kappa / (4.0 * OR_PI) * (bxs[c] / (sn * sn * sn) * (lg - delta) + cs_get(&av[c]));
                if (psi)
                    psi[3 * g + c] = kappa * d1[c] / sn / (2.0 * OR_PI) * (lg - (delta - 1.0)) +
                                     kappa / (4.0 * OR_PI) * cs_get(&ap[c]);
            }
        }
        free(tau);
        free(d);
    }
    return err;
}

/* ------------------------------------------------------------------ */
/* Weight functions, Eq. ewald_derivative_weight_functions             */
/* ------------------------------------------------------------------ */
static double g_near(double x) { return erfc(x) + 2.0 * x / sqrt(OR_PI) * exp(-x * x); }

/* g^(f)(x) = erf(x) - 2x/sqrt(pi) e^{-x^2}.  For x < 1/2 the difference
 * cancels, so use the series of the two Taylor expansions:
 * g^(f)(x) = (2/sqrt(pi)) sum_{n>=1} (-1)^{n+1} 2n x^{2n+1} / (n! (2n+1)). */
double or_g_far(double x)
{
    if (x < 0.5) {
        double x2 = x * x, term = x, s = 0.0; /* term = x^{2n+1}/n! */
        for (int n = 1; n < 60; n++) {
            term *= x2 / n;
            double t = 2.0 * n * term / (2.0 * n + 1.0);
            s += (n % 2 == 1) ? t : -t;
            if (t < 1e-18 * fabs(s)) break;
        }
        return 2.0 / sqrt(OR_PI) * s;
    }
    return erf(x) - 2.0 * x / sqrt(OR_PI) * exp(-x * x);
}

double or_g_near(double x) { return g_near(x); }

/* Index of the node before global node j within its filament. */
static long prev_node(const int64_t* off, const int64_t* fil_of, long j)
{
    long f = fil_of[j];
    long n = off[f + 1] - off[f];
    long jj = j - off[f];
    return off[f] + (jj + n - 1) % n;
}

/*
 * Short-range sums, Eqs. velocity_shortrange and streamfunction_shortrange,
 * by brute force over every quadrature point.
 *   all_images == 0: minimum image of each source, kept if r < rc.
 *   all_images == 1: the 27 images n in {-1,0,1}^3 of the minimum image,
 *                    no cut-off (used with alpha >= beta_o / min L).
 * The unwrapped local segments C_0 of the target are omitted; their images
 * are ordinary sources.  fil_of (N) is the filament of each node.
 */
void or_short_range(long ntgt, const int64_t* tgt, const double* nodes, const int64_t* off, const int64_t* fil_of,
                    const double* shift, long NQ, int Q, const double* qX, const double* qq, const double* L,
                    double kappa, double alpha, double rc, int all_images, double* v, double* psi)
{
    const double pref = kappa / (4.0 * OR_PI);
#pragma omp parallel for schedule(dynamic, 1)
    for (long t = 0; t < ntgt; t++) {
        long j = tgt[t];
        long jp = prev_node(off, fil_of, j);
        long f = fil_of[j];
        int first = (j == off[f]);
        const double* x = nodes + 3 * j;
        csum av[3] = { { 0, 0 }, { 0, 0 }, { 0, 0 } }, ap[3] = { { 0, 0 }, { 0, 0 }, { 0, 0 } };
        for (long qi = 0; qi < NQ; qi++) {
            long seg = qi / Q;
            int local = (seg == j || seg == jp);
            double du[3], d[3], rl[3] = { 0, 0, 0 };
            for (int c = 0; c < 3; c++) {
                du[c] = qX[3 * qi + c] - x[c];
                d[c] = du[c] - L[c] * nearbyint(du[c] / L[c]);
            }
            long nloc[3] = { 0, 0, 0 };
            if (local) {
                /* the omitted vector: the adjacent segment as it touches the node */
                for (int c = 0; c < 3; c++) {
                    rl[c] = du[c] - ((first && seg == jp) ? shift[3 * f + c] : 0.0);
                    nloc[c] = (long)nearbyint((rl[c] - d[c]) / L[c]);
                }
            }
            const double* q = qq + 3 * qi;
            int lo = all_images ? -1 : 0, hi = all_images ? 1 : 0;
            for (int n0 = lo; n0 <= hi; n0++)
                for (int n1 = lo; n1 <= hi; n1++)
                    for (int n2 = lo; n2 <= hi; n2++) {
                        if (local && n0 == nloc[0] && n1 == nloc[1] && n2 == nloc[2]) continue;
                        double r0[3] = { d[0] + n0 * L[0], d[1] + n1 * L[1], d[2] + n2 * L[2] };
                        double r = norm3(r0);
                        if (r == 0.0) continue;
                        if (!all_images && r >= rc) continue;
                        double xa = alpha * r;
                        double fv = pref * g_near(xa) / (r * r * r);
                        double cr[3];
                        cross3(r0, q, cr);
                        double fp = pref * erfc(xa) / r;
                        for (int c = 0; c < 3; c++) {
                            cs_add(&av[c], fv * cr[c]);
                            cs_add(&ap[c], fp * q[c]);
                        }
                    }
        }
        for (int c = 0; c < 3; c++) {
            v[3 * t + c] = cs_get(&av[c]);
            if (psi) psi[3 * t + c] = cs_get(&ap[c]);
        }
    }
}

/*
 * Long-range fields by a direct Fourier sum (Eqs. vorticity_fourier_coefs
 * and velocity_longrange_physical) over the cube |m_d| <= K_d, m != 0:
 *   omega_k = (kappa/V) sum_q q e^{-i k.X_q},
 *   v(x)   = sum_k Re[ i k x omega_k e^{-k^2/4 alpha^2} / k^2 e^{i k.x} ],
 *   psi(x) = sum_k Re[ omega_k e^{-k^2/4 alpha^2} / k^2 e^{i k.x} ].
 * Two steps: or_fourier_coefs (the sum over sources) and or_fourier_eval
 * (the synthesis at the targets); or_long_range does both.
 * omega layout: [m0][m1][m2][c][re,im], m_d from -K_d to K_d.
 */
void or_fourier_coefs(long NQ, const double* qX, const double* qq, const double* L, double kappa, const int* K,
                      double* om)
{
    const long n0 = 2 * K[0] + 1, n1 = 2 * K[1] + 1, n2 = 2 * K[2] + 1;
    const long nm = n0 * n1 * n2;
    const long nax = n0 + n1 + n2;
    const double V = L[0] * L[1] * L[2];
    double kk[3] = { 2.0 * OR_PI / L[0], 2.0 * OR_PI / L[1], 2.0 * OR_PI / L[2] };
    memset(om, 0, (size_t)(nm * 6) * sizeof(double));
    double* omc = (double*)calloc((size_t)(nm * 6), sizeof(double)); /* compensation */
    const long B = 1024;
    double* tab = (double*)malloc((size_t)(B * nax * 2) * sizeof(double));
    for (long q0 = 0; q0 < NQ; q0 += B) {
        long nb = (NQ - q0 < B) ? NQ - q0 : B;
        /* per-source 1-D phases e^{-i k_d m_d X_d}, direct cos/sin */
#pragma omp parallel for
        for (long b = 0; b < nb; b++) {
            const double* X = qX + 3 * (q0 + b);
            double* tb = tab + b * nax * 2;
            long o = 0;
            for (int dd = 0; dd < 3; dd++) {
                double xw = X[dd] - L[dd] * floor(X[dd] / L[dd]);
                for (long m = -K[dd]; m <= K[dd]; m++, o++) {
                    double ph = kk[dd] * (double)m * xw;
                    tb[2 * o] = cos(ph);
                    tb[2 * o + 1] = -sin(ph);
                }
            }
        }
#pragma omp parallel for schedule(static)
        for (long mi = 0; mi < nm; mi++) {
            long i0 = mi / (n1 * n2), i1 = (mi / n2) % n1, i2 = mi % n2;
            csum acc[6];
            for (int c = 0; c < 6; c++) { acc[c].s = om[6 * mi + c]; acc[c].c = omc[6 * mi + c]; }
            for (long b = 0; b < nb; b++) {
                const double* tb = tab + b * nax * 2;
                double ar = tb[2 * i0], ai = tb[2 * i0 + 1];
                double br = tb[2 * (n0 + i1)], bi = tb[2 * (n0 + i1) + 1];
                double cr = tb[2 * (n0 + n1 + i2)], ci = tb[2 * (n0 + n1 + i2) + 1];
                double er = ar * br - ai * bi, ei = ar * bi + ai * br;
                double pr = er * cr - ei * ci, pi = er * ci + ei * cr;
                const double* q = qq + 3 * (q0 + b);
                for (int c = 0; c < 3; c++) {
                    cs_add(&acc[2 * c], q[c] * pr);
                    cs_add(&acc[2 * c + 1], q[c] * pi);
                }
            }
            for (int c = 0; c < 6; c++) { om[6 * mi + c] = acc[c].s; omc[6 * mi + c] = acc[c].c; }
        }
    }
    for (long mi = 0; mi < nm; mi++)
        for (int c = 0; c < 6; c++) om[6 * mi + c] = (om[6 * mi + c] + omc[6 * mi + c]) * kappa / V;
    free(omc);
    free(tab);
}

void or_fourier_eval(long ntgt, const int64_t* tgt, const double* nodes, const double* L, double alpha, const int* K,
                     const double* om, double* v, double* psi)
{
    const long n0 = 2 * K[0] + 1, n1 = 2 * K[1] + 1, n2 = 2 * K[2] + 1;
    const long nm = n0 * n1 * n2;
    const long nax = n0 + n1 + n2;
    double kk[3] = { 2.0 * OR_PI / L[0], 2.0 * OR_PI / L[1], 2.0 * OR_PI / L[2] };
    /* per-mode multipliers G_k = e^{-k^2/4 alpha^2} / k^2 (0 at k = 0) */
    double* G = (double*)malloc((size_t)nm * sizeof(double));
    for (long mi = 0; mi < nm; mi++) {
        long m0 = mi / (n1 * n2) - K[0], m1 = (mi / n2) % n1 - K[1], m2 = mi % n2 - K[2];
        double k0 = kk[0] * m0, k1 = kk[1] * m1, k2 = kk[2] * m2;
        double k2s = k0 * k0 + k1 * k1 + k2 * k2;
        G[mi] = (k2s == 0.0) ? 0.0 : exp(-k2s / (4.0 * alpha * alpha)) / k2s;
    }

#pragma omp parallel for schedule(dynamic, 1)
    for (long t = 0; t < ntgt; t++) {
        const double* x = nodes + 3 * tgt[t];
        double* tb = (double*)malloc((size_t)(nax * 2) * sizeof(double));
        long o = 0;
        for (int dd = 0; dd < 3; dd++) {
            double xw = x[dd] - L[dd] * floor(x[dd] / L[dd]);
            for (long m = -K[dd]; m <= K[dd]; m++, o++) {
                double ph = kk[dd] * (double)m * xw;
                tb[2 * o] = cos(ph);
                tb[2 * o + 1] = sin(ph);
            }
        }
        csum av[3] = { { 0, 0 }, { 0, 0 }, { 0, 0 } }, ap[3] = { { 0, 0 }, { 0, 0 }, { 0, 0 } };
        for (long mi = 0; mi < nm; mi++) {
            if (G[mi] == 0.0) continue;
            long i0 = mi / (n1 * n2), i1 = (mi / n2) % n1, i2 = mi % n2;
            double kv[3] = { kk[0] * (i0 - K[0]), kk[1] * (i1 - K[1]), kk[2] * (i2 - K[2]) };
            double ar = tb[2 * i0], ai = tb[2 * i0 + 1];
            double br = tb[2 * (n0 + i1)], bi = tb[2 * (n0 + i1) + 1];
            double cr = tb[2 * (n0 + n1 + i2)], ci = tb[2 * (n0 + n1 + i2) + 1];
            double er = ar * br - ai * bi, ei = ar * bi + ai * br;
            double pr = er * cr - ei * ci, pi = er * ci + ei * cr; /* e^{i k.x} */
            const double* w = om + 6 * mi;
            double wr[3] = { w[0], w[2], w[4] }, wi[3] = { w[1], w[3], w[5] };
            /* i k x omega: (k x wr) i - (k x wi) */
            double cxr[3], cxi[3];
            cross3(kv, wr, cxr);
            cross3(kv, wi, cxi);
            for (int c = 0; c < 3; c++) {
                double vr = -cxi[c], vi = cxr[c]; /* i (a + i b) = -b + i a */
                cs_add(&av[c], G[mi] * (vr * pr - vi * pi));
                cs_add(&ap[c], G[mi] * (wr[c] * pr - wi[c] * pi));
            }
        }
        for (int c = 0; c < 3; c++) {
            v[3 * t + c] = cs_get(&av[c]);
            if (psi) psi[3 * t + c] = cs_get(&ap[c]);
        }
        free(tb);
    }
    free(G);
}

void or_long_range(long ntgt, const int64_t* tgt, const double* nodes, long NQ, const double* qX, const double* qq,
                   const double* L, double kappa, double alpha, const int* K, double* v, double* psi,
                   double* omega_out)
{
    const long nm = (2L * K[0] + 1) * (2L * K[1] + 1) * (2L * K[2] + 1);
    double* om = (double*)malloc((size_t)(nm * 6) * sizeof(double));
    or_fourier_coefs(NQ, qX, qq, L, kappa, K, om);
    if (omega_out) memcpy(omega_out, om, (size_t)(nm * 6) * sizeof(double));
    or_fourier_eval(ntgt, tgt, nodes, L, alpha, K, om, v, psi);
    free(om);
}

/*
 * Long-range self terms, Eqs. velocity_longrange_self and
 * streamfunction_longrange_self, on the Q quadrature points of each of the
 * two segments adjacent to the node (unwrapped, no periodic images).
 */
void or_self(long ntgt, const int64_t* tgt, const double* nodes, const int64_t* off, const int64_t* fil_of,
             const double* shift, int Q, const double* qX, const double* qq, double kappa, double alpha,
             double* v, double* psi)
{
    const double pref = kappa / (4.0 * OR_PI);
#pragma omp parallel for schedule(static)
    for (long t = 0; t < ntgt; t++) {
        long j = tgt[t];
        long jp = prev_node(off, fil_of, j);
        long f = fil_of[j];
        int first = (j == off[f]);
        const double* x = nodes + 3 * j;
        double av[3] = { 0, 0, 0 }, ap[3] = { 0, 0, 0 };
        long segs[2] = { jp, j };
        for (int sidx = 0; sidx < 2; sidx++) {
            long seg = segs[sidx];
            for (int i = 0; i < Q; i++) {
                long qi = seg * Q + i;
                double r0[3];
                for (int c = 0; c < 3; c++)
                    r0[c] = qX[3 * qi + c] - x[c] - ((first && sidx == 0) ? shift[3 * f + c] : 0.0);
                double r = norm3(r0);
                double xa = alpha * r;
                double fv = pref * or_g_far(xa) / (r * r * r);
                double fp = pref * erf(xa) / r;
                double cr[3];
                cross3(r0, qq + 3 * qi, cr);
                for (int c = 0; c < 3; c++) {
                    av[c] += fv * cr[c];
                    ap[c] += fp * qq[3 * qi + c];
                }
            }
        }
        for (int c = 0; c < 3; c++) {
            v[3 * t + c] = av[c];
            if (psi) psi[3 * t + c] = ap[c];
        }
    }
}

/*
 * Kinetic energy (Sec. 2.4, Eq. kinetic_energy_streamfunction,
 * E = kappa/(2V) oint psi . ds), split as in the Ewald decomposition:
 *   long range: kappa/(2V) sum_q q . psi^(f)(s_q) = (1/2) sum_{k != 0}
 *               e^{-k^2/4 alpha^2} |omega_k|^2 / k^2   (or_energy_fourier,
 *               over the full cube of omega from or_fourier_coefs);
 *   the rest:   psi_local + psi^(n) - psi^(f)_self known at the nodes, f_j =
 *               psi_j . sdot(tau_j) interpolated by the same periodic spline
 *               in tau and integrated over each filament with Gauss-Legendre
 *               (or_energy_line returns sum over filaments of int f dtau).
 */
double or_energy_fourier(const double* om, const int* K, const double* L, double alpha)
{
    const long n0 = 2 * K[0] + 1, n1 = 2 * K[1] + 1, n2 = 2 * K[2] + 1;
    const long nm = n0 * n1 * n2;
    double kk[3] = { 2.0 * OR_PI / L[0], 2.0 * OR_PI / L[1], 2.0 * OR_PI / L[2] };
    csum acc = { 0, 0 };
    for (long mi = 0; mi < nm; mi++) {
        long m0 = mi / (n1 * n2) - K[0], m1 = (mi / n2) % n1 - K[1], m2 = mi % n2 - K[2];
        double k0 = kk[0] * m0, k1 = kk[1] * m1, k2 = kk[2] * m2;
        double k2s = k0 * k0 + k1 * k1 + k2 * k2;
        if (k2s == 0.0) continue;
        double w2 = 0.0;
        for (int c = 0; c < 6; c++) w2 += om[6 * mi + c] * om[6 * mi + c];
        cs_add(&acc, 0.5 * exp(-k2s / (4.0 * alpha * alpha)) * w2 / k2s);
    }
    return cs_get(&acc);
}

double or_energy_line(long nfil, const int64_t* off, const double* nodes, const double* shift, int k,
                      const double* psi_nodes)
{
    double h[8], w[8];
    or_gauss_legendre(4, h, w);
    csum tot = { 0, 0 };
    for (long f = 0; f < nfil; f++) {
        long n = off[f + 1] - off[f];
        const double* s = nodes + 3 * off[f];
        const double* sh = shift + 3 * f;
        double* tau = (double*)malloc((size_t)n * sizeof(double));
        double* d = (double*)malloc((size_t)(n * 3) * sizeof(double));
        double* fv = (double*)malloc((size_t)(n * 3) * sizeof(double));
        double* fc = (double*)malloc((size_t)(n * 3) * sizeof(double));
        double T;
        fit_filament(n, s, sh, k, tau, &T, d);
        kseq K = { tau, n, T };
        /* f_j = psi_j . sdot(tau_j); carried in the first of three columns */
        for (long j = 0; j < n; j++) {
            double d1[3];
            spline_eval(&K, k, d, j, tau[j], 1, d1);
            for (int c = 0; c < 3; c++) d1[c] += sh[c] / T;
            const double* ps = psi_nodes + 3 * (off[f] + j);
            fv[3 * j] = ps[0] * d1[0] + ps[1] * d1[1] + ps[2] * d1[2];
            fv[3 * j + 1] = 0.0;
            fv[3 * j + 2] = 0.0;
        }
        spline_fit(&K, k, fv, fc);
        for (long j = 0; j < n; j++) {
            double dtau = (j < n - 1 ? tau[j + 1] : T) - tau[j];
            for (int i = 0; i < 4; i++) {
                double v[3];
                spline_eval(&K, k, fc, j, tau[j] + h[i] * dtau, 0, v);
                cs_add(&tot, w[i] * dtau * v[0]);
            }
        }
        free(tau);
        free(d);
        free(fv);
        free(fc);
    }
    return cs_get(&tot);
}

/*
 * Naive open-space Biot-Savart sum (Eq. BS_on_vortex with no periodic
 * images, the alpha = 0 reading of Sec. 3.2): every quadrature point except
 * those of the two unwrapped segments adjacent to the node.
 */
void or_open_space(long ntgt, const int64_t* tgt, const double* nodes, const int64_t* off, const int64_t* fil_of,
                   long NQ, int Q, const double* qX, const double* qq, double kappa, double* v, double* psi)
{
    const double pref = kappa / (4.0 * OR_PI);
#pragma omp parallel for schedule(dynamic, 1)
    for (long t = 0; t < ntgt; t++) {
        long j = tgt[t];
        long jp = prev_node(off, fil_of, j);
        const double* x = nodes + 3 * j;
        csum av[3] = { { 0, 0 }, { 0, 0 }, { 0, 0 } }, ap[3] = { { 0, 0 }, { 0, 0 }, { 0, 0 } };
        for (long qi = 0; qi < NQ; qi++) {
            long seg = qi / Q;
            if (seg == j || seg == jp) continue;
            double r0[3] = { qX[3 * qi] - x[0], qX[3 * qi + 1] - x[1], qX[3 * qi + 2] - x[2] };
            double r = norm3(r0);
            if (r == 0.0) continue;
            double cr[3];
            cross3(r0, qq + 3 * qi, cr);
            for (int c = 0; c < 3; c++) {
                cs_add(&av[c], pref * cr[c] / (r * r * r));
                cs_add(&ap[c], pref * qq[3 * qi + c] / r);
            }
        }
        for (int c = 0; c < 3; c++) {
            v[3 * t + c] = cs_get(&av[c]);
            if (psi) psi[3 * t + c] = cs_get(&ap[c]);
        }
    }
}
