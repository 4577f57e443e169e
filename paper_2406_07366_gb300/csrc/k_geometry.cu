// Curve geometry on the GPU: periodic cubic spline fit per filament, then one
// pass per node that produces the quadrature sources of its outgoing segment
// (Sec. 2.6, Eq. line_integral_quadrature; Sec. 3.3 charges
// q = w_i dtau_j s'(tau)), the local term (Eqs. BS_local,
// streamfunction_local) and the long-range self term on the 2Q points of
// the two adjacent segments (Eqs. velocity_longrange_self,
// streamfunction_longrange_self).
//
// Spline form.  Appendix B fits a periodic B-spline with knots at the
// chord-length parameters.  For order 4 the same curve (the unique periodic
// C2 cubic through the nodes with those knots) is obtained here from its
// second derivatives M_j at the knots, which solve the cyclic tridiagonal
// system
//   h_{j-1} M_{j-1} + 2 (h_{j-1} + h_j) M_j + h_j M_{j+1}
//       = 6 (dp_j / h_j - dp_{j-1} / h_{j-1}),
// solved with the Sherman-Morrison correction and the Thomas algorithm (the
// procedure the appendix names for the cyclic system).  On segment j, with
// u = tau - tau_j in [0, h_j],
//   p(u) - p_j = b_j u + M_j u^2 / 2 + (M_{j+1} - M_j) u^3 / (6 h_j),
//   b_j = dp_j / h_j - h_j (2 M_j + M_{j+1}) / 6.
// Unclosed curves with s(tau + T) = s(tau) + n L interpolate the periodic
// part p = s - n L tau / T and add the drift n L / T back.
//
// Precision.  Node positions stay float64.  Every quantity that is a small
// difference (chords, increments, moments, the offset of a quadrature point
// from its node) is carried in T; the absolute position of a source is
// s_j (float64) + offset (T), wrapped and split into a cell index plus a
// T-precision offset from the cell origin.
#include <math.h>

#include "bs_internal.cuh"

namespace bsw {

template <typename T>
__device__ __forceinline__ T tsqrt(T x) { return sqrt(x); }

// g^(f)(x) = erf(x) - 2x/sqrt(pi) exp(-x^2) (Eq. ewald_derivative_weight_functions).
// Below x = 1/2 the two terms cancel; there the Taylor series of both terms,
// combined term by term, gives (2/sqrt(pi)) sum_{n>=1} (-1)^{n+1} 2n x^{2n+1}/(n!(2n+1)).
template <typename T>
__device__ __forceinline__ T g_far(T x)
{
    const T two_over_sqrtpi = (T)1.12837916709551257390;
    if (x < (T)0.5) {
        const int nterms = sizeof(T) == 4 ? 8 : 15;
        T x2 = x * x, pw = x, s = 0;
        T fact = 1;
        for (int n = 1; n <= nterms; ++n) {
            pw *= x2;          // x^{2n+1}
            fact *= (T)n;      // n!
            T t = (T)(2 * n) * pw / (fact * (T)(2 * n + 1));
            s += (n & 1) ? t : -t;
        }
        return two_over_sqrtpi * s;
    }
    return erf(x) - two_over_sqrtpi * x * exp(-x * x);
}

// ---------------------------------------------------------------------------
// Spline fit: one thread per filament.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_spline(const double* __restrict__ nodes, const int64_t* __restrict__ off,
                         const double* __restrict__ shift, int nfil, T* __restrict__ hseg, T* __restrict__ dp,
                         T* __restrict__ ds, T* __restrict__ Mm, T* __restrict__ cpr, T* __restrict__ zz,
                         T* __restrict__ Tper)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfil) return;
    const int64_t o = off[f];
    const int n = (int)(off[f + 1] - o);
    const double sh0 = shift[3 * f], sh1 = shift[3 * f + 1], sh2 = shift[3 * f + 2];

    // chord lengths and period (Appendix B chord-length parameter)
    double Tsum = 0.0;
    for (int j = 0; j < n; ++j) {
        const double* a = nodes + 3 * (o + j);
        double b0, b1, b2;
        if (j + 1 < n) {
            const double* b = a + 3;
            b0 = b[0]; b1 = b[1]; b2 = b[2];
        } else {
            const double* b = nodes + 3 * o;
            b0 = b[0] + sh0; b1 = b[1] + sh1; b2 = b[2] + sh2;
        }
        const double d0 = b0 - a[0], d1 = b1 - a[1], d2 = b2 - a[2];
        const double h = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        Tsum += h;
        hseg[o + j] = (T)h;
        ds[3 * (o + j) + 0] = (T)d0;
        ds[3 * (o + j) + 1] = (T)d1;
        ds[3 * (o + j) + 2] = (T)d2;
        dp[3 * (o + j) + 0] = (T)d0;  // closed curve: dp = ds; drift removed below otherwise
        dp[3 * (o + j) + 1] = (T)d1;
        dp[3 * (o + j) + 2] = (T)d2;
    }
    Tper[f] = (T)Tsum;
    const bool closed = (sh0 == 0.0 && sh1 == 0.0 && sh2 == 0.0);
    if (!closed) {
        // periodic increments dp_j = ds_j - n L h_j / T
        const double invT = 1.0 / Tsum;
        for (int j = 0; j < n; ++j) {
            const double h = (double)hseg[o + j];
            dp[3 * (o + j) + 0] = (T)((double)ds[3 * (o + j) + 0] - sh0 * h * invT);
            dp[3 * (o + j) + 1] = (T)((double)ds[3 * (o + j) + 1] - sh1 * h * invT);
            dp[3 * (o + j) + 2] = (T)((double)ds[3 * (o + j) + 2] - sh2 * h * invT);
        }
    }

    // Cyclic tridiagonal system, row j: a_j M_{j-1} + b_j M_j + c_j M_{j+1} = r_j,
    // a_j = h_{j-1}, b_j = 2 (h_{j-1} + h_j), c_j = h_j; corners a_0 (col n-1)
    // and c_{n-1} (col 0).  Sherman-Morrison with gamma = -b_0:
    //   B = A - u v^T, u = (gamma, 0, ..., c_{n-1}), v = (1, 0, ..., a_0 / gamma).
    const T hl = hseg[o + n - 1];
    const T a0 = hl, cn = hl;
    const T b0 = (T)2 * (hl + hseg[o]);
    const T gamma = -b0;
    T cprev = 0, dprev0 = 0, dprev1 = 0, dprev2 = 0, zprev = 0;
    T dpm0 = dp[3 * (o + n - 1) + 0], dpm1 = dp[3 * (o + n - 1) + 1], dpm2 = dp[3 * (o + n - 1) + 2];
    T hm = hl;
    for (int j = 0; j < n; ++j) {
        const T hj = hseg[o + j];
        const T dj0 = dp[3 * (o + j) + 0], dj1 = dp[3 * (o + j) + 1], dj2 = dp[3 * (o + j) + 2];
        const T a = (j == 0) ? (T)0 : hm;
        T b = (T)2 * (hm + hj);
        if (j == 0) b -= gamma;
        if (j == n - 1) b -= a0 * cn / gamma;
        const T c = (j == n - 1) ? (T)0 : hj;
        const T r0 = (T)6 * (dj0 / hj - dpm0 / hm);
        const T r1 = (T)6 * (dj1 / hj - dpm1 / hm);
        const T r2 = (T)6 * (dj2 / hj - dpm2 / hm);
        const T uj = (j == 0) ? gamma : ((j == n - 1) ? cn : (T)0);
        const T m = b - a * cprev;
        const T im = (T)1 / m;
        cprev = c * im;
        dprev0 = (r0 - a * dprev0) * im;
        dprev1 = (r1 - a * dprev1) * im;
        dprev2 = (r2 - a * dprev2) * im;
        zprev = (uj - a * zprev) * im;
        cpr[o + j] = cprev;
        Mm[3 * (o + j) + 0] = dprev0;
        Mm[3 * (o + j) + 1] = dprev1;
        Mm[3 * (o + j) + 2] = dprev2;
        zz[o + j] = zprev;
        hm = hj;
        dpm0 = dj0; dpm1 = dj1; dpm2 = dj2;
    }
    // back substitution (in place)
    T x0 = Mm[3 * (o + n - 1) + 0], x1 = Mm[3 * (o + n - 1) + 1], x2 = Mm[3 * (o + n - 1) + 2];
    T zx = zz[o + n - 1];
    for (int j = n - 2; j >= 0; --j) {
        const T cj = cpr[o + j];
        x0 = Mm[3 * (o + j) + 0] - cj * x0;
        x1 = Mm[3 * (o + j) + 1] - cj * x1;
        x2 = Mm[3 * (o + j) + 2] - cj * x2;
        zx = zz[o + j] - cj * zx;
        Mm[3 * (o + j) + 0] = x0;
        Mm[3 * (o + j) + 1] = x1;
        Mm[3 * (o + j) + 2] = x2;
        zz[o + j] = zx;
    }
    const T vfac = a0 / gamma;
    const T z0 = zz[o], zn = zz[o + n - 1];
    const T den = (T)1 + z0 + vfac * zn;
    const T f0 = (Mm[3 * o + 0] + vfac * Mm[3 * (o + n - 1) + 0]) / den;
    const T f1 = (Mm[3 * o + 1] + vfac * Mm[3 * (o + n - 1) + 1]) / den;
    const T f2 = (Mm[3 * o + 2] + vfac * Mm[3 * (o + n - 1) + 2]) / den;
    for (int j = 0; j < n; ++j) {
        const T zj = zz[o + j];
        Mm[3 * (o + j) + 0] -= f0 * zj;
        Mm[3 * (o + j) + 1] -= f1 * zj;
        Mm[3 * (o + j) + 2] -= f2 * zj;
    }
}

// The same fit with one warp per filament, staged in shared memory: the
// lanes compute chords, increments and right-hand sides in parallel; lanes
// 0..3 then run the four sequential Thomas sweeps (x, y, z and the
// Sherman-Morrison vector) out of shared memory; all lanes apply the
// correction and write the moments.  smem: 9 * nmax values of T.
template <typename T>
__device__ __forceinline__ void k_spline_warp_body(const double* __restrict__ nodes, const int64_t* __restrict__ off,
                                                   const double* __restrict__ shift, int nfil, int nmax,
                                                   T* __restrict__ hseg, T* __restrict__ dp, T* __restrict__ ds,
                                                   T* __restrict__ Mm, T* __restrict__ Tper, int bid)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    T* sh_h = reinterpret_cast<T*>(sm_raw);  // n
    T* sh_dp = sh_h + nmax;                   // 3 n
    T* sh_r = sh_dp + 3 * nmax;               // 4 n: right-hand sides, then solutions
    T* sh_cp = sh_r + 4 * nmax;               // n: modified super-diagonal
    const int f = bid;
    if (f >= nfil) return;
    const int lane = threadIdx.x;
    const int64_t o = off[f];
    const int n = (int)(off[f + 1] - o);
    const double s0 = shift[3 * f], s1 = shift[3 * f + 1], s2 = shift[3 * f + 2];

    double tpart = 0.0;
    for (int j = lane; j < n; j += 32) {
        const double* a = nodes + 3 * (o + j);
        const double* b = nodes + 3 * (j + 1 < n ? o + j + 1 : o);
        const double w0 = (j + 1 < n) ? 0.0 : s0, w1 = (j + 1 < n) ? 0.0 : s1, w2 = (j + 1 < n) ? 0.0 : s2;
        const double d0 = b[0] + w0 - a[0], d1 = b[1] + w1 - a[1], d2 = b[2] + w2 - a[2];
        const double h = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        tpart += h;
        sh_h[j] = (T)h;
        hseg[o + j] = (T)h;
        ds[3 * (o + j) + 0] = (T)d0;
        ds[3 * (o + j) + 1] = (T)d1;
        ds[3 * (o + j) + 2] = (T)d2;
    }
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) tpart += __shfl_xor_sync(0xffffffffu, tpart, k);
    const double Tsum = tpart;
    if (lane == 0) Tper[f] = (T)Tsum;
    const double invT = 1.0 / Tsum;
    for (int j = lane; j < n; j += 32) {
        const double* a = nodes + 3 * (o + j);
        const double* b = nodes + 3 * (j + 1 < n ? o + j + 1 : o);
        const double w0 = (j + 1 < n) ? 0.0 : s0, w1 = (j + 1 < n) ? 0.0 : s1, w2 = (j + 1 < n) ? 0.0 : s2;
        const double h = sqrt((b[0] + w0 - a[0]) * (b[0] + w0 - a[0]) + (b[1] + w1 - a[1]) * (b[1] + w1 - a[1]) +
                              (b[2] + w2 - a[2]) * (b[2] + w2 - a[2]));
        const T p0 = (T)(b[0] + w0 - a[0] - s0 * h * invT);
        const T p1 = (T)(b[1] + w1 - a[1] - s1 * h * invT);
        const T p2 = (T)(b[2] + w2 - a[2] - s2 * h * invT);
        sh_dp[j] = p0;
        sh_dp[nmax + j] = p1;
        sh_dp[2 * nmax + j] = p2;
        dp[3 * (o + j) + 0] = p0;
        dp[3 * (o + j) + 1] = p1;
        dp[3 * (o + j) + 2] = p2;
    }
    __syncwarp();
    // right-hand sides 6 (dp_j / h_j - dp_{j-1} / h_{j-1}) and the vector u
    const T hl = sh_h[n - 1];
    const T gamma = -(T)2 * (hl + sh_h[0]);
    for (int j = lane; j < n; j += 32) {
        const int jm = j == 0 ? n - 1 : j - 1;
        const T hj = sh_h[j], hm = sh_h[jm];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            sh_r[c * nmax + j] = (T)6 * (sh_dp[c * nmax + j] / hj - sh_dp[c * nmax + jm] / hm);
        sh_r[3 * nmax + j] = (j == 0) ? gamma : ((j == n - 1) ? hl : (T)0);
    }
    __syncwarp();
    if (lane < 4) {
        T* r = sh_r + lane * nmax;
        const T a0 = hl, cn = hl;
        T cprev = 0, dprev = 0, hm = hl;
        for (int j = 0; j < n; ++j) {
            const T hj = sh_h[j];
            const T a = (j == 0) ? (T)0 : hm;
            T bb = (T)2 * (hm + hj);
            if (j == 0) bb -= gamma;
            if (j == n - 1) bb -= a0 * cn / gamma;
            const T c = (j == n - 1) ? (T)0 : hj;
            const T im = (T)1 / (bb - a * cprev);
            cprev = c * im;
            dprev = (r[j] - a * dprev) * im;
            if (lane == 0) sh_cp[j] = cprev;
            r[j] = dprev;
            hm = hj;
        }
        __syncwarp(0xfu);
        T x = r[n - 1];
        for (int j = n - 2; j >= 0; --j) {
            x = r[j] - sh_cp[j] * x;
            r[j] = x;
        }
    }
    __syncwarp();
    const T vfac = hl / gamma;
    const T* z = sh_r + 3 * nmax;
    const T den = (T)1 + z[0] + vfac * z[n - 1];
    T fc[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) fc[c] = (sh_r[c * nmax] + vfac * sh_r[c * nmax + n - 1]) / den;
    for (int j = lane; j < n; j += 32) {
#pragma unroll
        for (int c = 0; c < 3; ++c) Mm[3 * (o + j) + c] = sh_r[c * nmax + j] - fc[c] * z[j];
    }
}

template <typename T>
__global__ void k_spline_warp(const double* __restrict__ nodes, const int64_t* __restrict__ off,
                              const double* __restrict__ shift, int nfil, int nmax, T* __restrict__ hseg,
                              T* __restrict__ dp, T* __restrict__ ds, T* __restrict__ Mm, T* __restrict__ Tper)
{
    k_spline_warp_body<T>(nodes, off, shift, nfil, nmax, hseg, dp, ds, Mm, Tper, blockIdx.x);
}

// Wrap x into [0, L) (iL = 1/L); non-finite input maps to 0 and raises the flag.
__device__ __forceinline__ double wrap_box(double x, double L, double iL, bool& bad)
{
    if (!isfinite(x)) {
        bad = true;
        return 0.0;
    }
    double y = x - L * floor(x * iL);
    if (y >= L) y -= L;
    if (y < 0.0) y = 0.0;
    return y;
}

template <typename T>
struct SegPoly {
    T b[3], m[3], c3[3], c4[3], c5[3], drift[3], h;
    // p(u) - p_j = b u + m u^2 / 2 + c3 u^3 + c4 u^4 + c5 u^5 (+ drift u)
    __device__ __forceinline__ void eval(T u, T* delta, T* sdot) const
    {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            delta[c] = (((((c5[c] * u + c4[c]) * u + c3[c]) * u + (T)0.5 * m[c]) * u + b[c]) + drift[c]) * u;
            sdot[c] = (((((T)5 * c5[c] * u + (T)4 * c4[c]) * u + (T)3 * c3[c]) * u + m[c]) * u + b[c]) + drift[c];
        }
    }
};

// Segment j (to jn).  Cubic (Dd == nullptr): from the moments M, b_j =
// dp_j / h - h (2 M_j + M_{j+1}) / 6, c3 = (M_{j+1} - M_j) / (6 h).  Quintic:
// the Hermite quintic through p_j, p_{j+1} with first derivatives D_j,
// D_{j+1} and second derivatives M_j, M_{j+1}:
//   A = (dp - D_j h - M_j h^2 / 2) / h^3, B = (D_{j+1} - D_j - M_j h) / h^2,
//   C = (M_{j+1} - M_j) / h,
//   c3 = 10 A - 4 B + C / 2, c4 = (7 B - 15 A - C) / h, c5 = (6 A - 3 B + C / 2) / h^2.
template <typename T>
__device__ __forceinline__ void make_poly(SegPoly<T>& P, const T* __restrict__ hseg, const T* __restrict__ dp,
                                          const T* __restrict__ Mm, int j, int jn, const T drift[3],
                                          const T* __restrict__ Dd = nullptr)
{
    const T h = hseg[j];
    P.h = h;
    const T ih = (T)1 / h;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const T Mj = Mm[3 * j + c], Mn = Mm[3 * jn + c];
        P.m[c] = Mj;
        P.drift[c] = drift[c];
        if (Dd) {
            const T Dj = Dd[3 * j + c], Dn = Dd[3 * jn + c];
            const T A = (dp[3 * j + c] - Dj * h - (T)0.5 * Mj * h * h) * ih * ih * ih;
            const T B = (Dn - Dj - Mj * h) * ih * ih;
            const T C = (Mn - Mj) * ih;
            P.b[c] = Dj;
            P.c3[c] = (T)10 * A - (T)4 * B + (T)0.5 * C;
            P.c4[c] = ((T)7 * B - (T)15 * A - C) * ih;
            P.c5[c] = ((T)6 * A - (T)3 * B + (T)0.5 * C) * ih * ih;
        } else {
            P.b[c] = dp[3 * j + c] * ih - h * ((T)2 * Mj + Mn) / (T)6;
            P.c3[c] = (Mn - Mj) * ih / (T)6;
            P.c4[c] = 0;
            P.c5[c] = 0;
        }
    }
}

// Accumulate the self terms of one C_0 point: r from the node, charge q.
template <typename T>
__device__ __forceinline__ void self_add(const T r[3], const T q[3], T alpha, T* vs, T* ps)
{
    const T rr = tsqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    const T x = alpha * rr;
    const T fv = g_far(x) / (rr * rr * rr);
    const T fp = erf(x) / rr;
    vs[0] += fv * (r[1] * q[2] - r[2] * q[1]);
    vs[1] += fv * (r[2] * q[0] - r[0] * q[2]);
    vs[2] += fv * (r[0] * q[1] - r[1] * q[0]);
    ps[0] += fp * q[0];
    ps[1] += fp * q[1];
    ps[2] += fp * q[2];
}

template <typename T>
__device__ __forceinline__ void k_nodes_body(const GeomP& P, const double* __restrict__ nodes,
                                             const int* __restrict__ fil_of, const int* __restrict__ prev,
                                             const int64_t* __restrict__ off, const double* __restrict__ shift,
                                             const T* __restrict__ hseg, const T* __restrict__ dp,
                                             const T* __restrict__ ds, const T* __restrict__ Mm,
                                             const T* __restrict__ Tper, SrRec<T>* __restrict__ sr_rec,
                                             int* __restrict__ sr_key, LrRec<T>* __restrict__ lr_rec,
                                             int* __restrict__ lr_key, SrTgt<T>* __restrict__ tgt,
                                             double* __restrict__ vls, double* __restrict__ pls,
                                             double* __restrict__ part_local, double* __restrict__ part_self,
                                             double* __restrict__ psi_local, double* __restrict__ psi_self,
                                             int* __restrict__ status, const T* __restrict__ Dd, int bid)
{
    const int j = bid * blockDim.x + threadIdx.x;
    if (j >= P.N) return;
    const int f = fil_of[j];
    const int jp = prev[j];
    const int jn = (j + 1 < (int)off[f + 1]) ? j + 1 : (int)off[f];
    const T Tp = Tper[f];
    const T drift[3] = { (T)shift[3 * f] / Tp, (T)shift[3 * f + 1] / Tp, (T)shift[3 * f + 2] / Tp };
    const double sj[3] = { nodes[3 * j], nodes[3 * j + 1], nodes[3 * j + 2] };
    bool bad = false, bad_node = false;
    int flags = 0;
    double sw[3];  // the node wrapped into the box
#pragma unroll
    for (int c = 0; c < 3; ++c) sw[c] = wrap_box(sj[c], P.L[c], P.iL[c], bad_node);

    SegPoly<T> S;
    make_poly(S, hseg, dp, Mm, j, jn, drift, Dd);
    if ((double)S.h > P.seg_max || !(S.h > (T)0)) flags |= ST_GEOMETRY;

    T vs[3] = { 0, 0, 0 }, ps[3] = { 0, 0, 0 };
    T lp = 0, lm = 0;
    const T alpha = (T)P.alpha;

    // Outgoing segment j: sources for both ranges, self term, l^+.
    for (int i = 0; i < P.Q; ++i) {
        const T u = (T)P.gh[i] * S.h;
        T del[3], sd[3];
        S.eval(u, del, sd);
        const T wq = (T)P.gw[i] * S.h;
        T q[3] = { wq * sd[0], wq * sd[1], wq * sd[2] };
        lp += wq * tsqrt(sd[0] * sd[0] + sd[1] * sd[1] + sd[2] * sd[2]);
        self_add(del, q, alpha, vs, ps);

        // the point is near the wrapped node: it is mostly in the box already
        bool b2 = false;
        double xw[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double x = sw[c] + (double)del[c];
            if (!(x >= 0.0 && x < P.L[c])) x = wrap_box(x, P.L[c], P.iL[c], b2);
            xw[c] = x;
        }
        if (b2 || bad_node) {
            bad = true;
            q[0] = q[1] = q[2] = 0;
        }
        const int p = j * P.Q + i;
        // short-range record
        SrRec<T> R;
        int ci[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            int k = (int)(xw[c] * P.ihc[c]);
            k = k < 0 ? 0 : (k >= P.nc[c] ? P.nc[c] - 1 : k);
            ci[c] = k;
            R.o[c] = (T)(xw[c] - (k + 0.5) * P.hc[c]);  // from the cell centre: half the magnitude
            R.q[c] = q[c];
        }
        R.cx = ci[0];
        R.seg = j;
        sr_rec[p] = R;
        sr_key[p] = ci[0] + P.nc[0] * (ci[1] + P.nc[1] * ci[2]);
        // long-range record
        LrRec<T> G;
        int ib[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double g = xw[c] * P.ihg[c];
            int k = (int)floor(g);
            k = k < 0 ? 0 : (k >= P.ng[c] ? P.ng[c] - 1 : k);
            ib[c] = k;
            T fr = (T)(g - (double)k);
            fr = fr < (T)0 ? (T)0 : (fr > (T)1 ? (T)1 : fr);
            G.f[c] = fr;
            G.q[c] = q[c];
        }
        G.base = ib[0] | (ib[1] << 10) | (ib[2] << 20);
        lr_rec[p] = G;
        lr_key[p] = ib[0] / P.tile[0] + P.ntile[0] * (ib[1] / P.tile[1] + P.ntile[1] * (ib[2] / P.tile[2]));
    }

    // Incoming segment jp -> j: self term and l^-.
    {
        SegPoly<T> R;
        make_poly(R, hseg, dp, Mm, jp, j, drift, Dd);
        const T dsx = ds[3 * jp], dsy = ds[3 * jp + 1], dsz = ds[3 * jp + 2];
        for (int i = 0; i < P.Q; ++i) {
            const T u = (T)P.gh[i] * R.h;
            T del[3], sd[3];
            R.eval(u, del, sd);
            const T wq = (T)P.gw[i] * R.h;
            const T q[3] = { wq * sd[0], wq * sd[1], wq * sd[2] };
            lm += wq * tsqrt(sd[0] * sd[0] + sd[1] * sd[1] + sd[2] * sd[2]);
            const T r[3] = { del[0] - dsx, del[1] - dsy, del[2] - dsz };
            self_add(r, q, alpha, vs, ps);
        }
    }

    // Subdivided local segments (Sec. 5.2): l^+- cover the fraction f of each
    // local segment next to the node; the rest of both segments, cut into the
    // pieces [f, 2f], [2f, 4f], ..., [2^m f, 1] (fractions from the node), is
    // summed with the plain Biot-Savart kernel, Q-point Gauss-Legendre each.
    T vd[3] = { 0, 0, 0 }, pd[3] = { 0, 0, 0 };
    if (P.local_frac > 0.0) {
        const T fr = (T)P.local_frac;
        SegPoly<T> R;
        make_poly(R, hseg, dp, Mm, jp, j, drift, Dd);
        const T dsp[3] = { ds[3 * jp], ds[3 * jp + 1], ds[3 * jp + 2] };
        lp = 0;
        lm = 0;
        for (int i = 0; i < P.Q; ++i) {
            const T gh = (T)P.gh[i], gw = (T)P.gw[i];
            T del[3], sd[3];
            S.eval(gh * fr * S.h, del, sd);
            lp += gw * fr * S.h * tsqrt(sd[0] * sd[0] + sd[1] * sd[1] + sd[2] * sd[2]);
            R.eval(((T)1 - fr + gh * fr) * R.h, del, sd);
            lm += gw * fr * R.h * tsqrt(sd[0] * sd[0] + sd[1] * sd[1] + sd[2] * sd[2]);
        }
        for (int side = 0; side < 2; ++side) {
            const SegPoly<T>& Gs = side == 0 ? S : R;
            T x0 = fr;
            for (int piece = 0; piece < 64 && x0 < (T)1; ++piece) {
                const T x1 = (T)2 * x0 < (T)1 ? (T)2 * x0 : (T)1;
                for (int i = 0; i < P.Q; ++i) {
                    const T x = x0 + (x1 - x0) * (T)P.gh[i];  // fraction from the node
                    const T u = side == 0 ? x * Gs.h : ((T)1 - x) * Gs.h;
                    const T wt = (x1 - x0) * Gs.h * (T)P.gw[i];
                    T del[3], sd[3];
                    Gs.eval(u, del, sd);
                    T r[3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) r[c] = side == 0 ? del[c] : del[c] - dsp[c];
                    const T q[3] = { wt * sd[0], wt * sd[1], wt * sd[2] };
                    const T rr = tsqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
                    const T ir3 = (T)1 / (rr * rr * rr);
                    vd[0] += (r[1] * q[2] - r[2] * q[1]) * ir3;
                    vd[1] += (r[2] * q[0] - r[0] * q[2]) * ir3;
                    vd[2] += (r[0] * q[1] - r[1] * q[0]) * ir3;
                    pd[0] += q[0] / rr;
                    pd[1] += q[1] / rr;
                    pd[2] += q[2] / rr;
                }
                x0 = x1;
            }
        }
    }

    // Node geometry: sdot = b + drift, sddot = M_j; s' x s'' = (sdot x sddot)/|sdot|^3.
    const T d0 = S.b[0] + drift[0], d1 = S.b[1] + drift[1], d2 = S.b[2] + drift[2];
    const T sn = tsqrt(d0 * d0 + d1 * d1 + d2 * d2);
    const T is3 = (T)1 / (sn * sn * sn);
    const T bx = (d1 * S.m[2] - d2 * S.m[1]) * is3;
    const T by = (d2 * S.m[0] - d0 * S.m[2]) * is3;
    const T bz = (d0 * S.m[1] - d1 * S.m[0]) * is3;
    // log(2 sqrt(l- l+) / a): the l-dependent half in the kernel precision
    const double lg = (double)((T)0.5 * log(lm * lp)) + P.log2a;
    const double pv = P.kappa / (4.0 * kPi);
    const double vl[3] = { pv * ((double)bx * (lg - P.delta) + (double)vd[0]),
                           pv * ((double)by * (lg - P.delta) + (double)vd[1]),
                           pv * ((double)bz * (lg - P.delta) + (double)vd[2]) };
    const double vx[3] = { pv * (double)vs[0], pv * (double)vs[1], pv * (double)vs[2] };
#pragma unroll
    for (int c = 0; c < 3; ++c) vls[3 * j + c] = vl[c] - vx[c];
    if (part_local) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            part_local[3 * j + c] = vl[c];
            part_self[3 * j + c] = vx[c];
        }
    }
    if (P.want_psi) {
        const double pp = P.kappa / (2.0 * kPi);
        const double ip = 1.0 / (double)sn;
        const double pl[3] = { pp * (double)d0 * ip * (lg - (P.delta - 1.0)) + pv * (double)pd[0],
                               pp * (double)d1 * ip * (lg - (P.delta - 1.0)) + pv * (double)pd[1],
                               pp * (double)d2 * ip * (lg - (P.delta - 1.0)) + pv * (double)pd[2] };
        const double px[3] = { pv * (double)ps[0], pv * (double)ps[1], pv * (double)ps[2] };
#pragma unroll
        for (int c = 0; c < 3; ++c) pls[3 * j + c] = pl[c] - px[c];
        if (psi_local) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                psi_local[3 * j + c] = pl[c];
                psi_self[3 * j + c] = px[c];
            }
        }
    }

    // Target record of the node for the short range.
    {
        SrTgt<T> tg;
        int ci[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double xw = sw[c];
            int k = (int)(xw * P.ihc[c]);
            k = k < 0 ? 0 : (k >= P.nc[c] ? P.nc[c] - 1 : k);
            ci[c] = k;
            tg.o[c] = (T)(xw - (k + 0.5) * P.hc[c]);
        }
        tg.cell = ci[0] + P.nc[0] * (ci[1] + P.nc[1] * ci[2]);
        tgt[j] = tg;
        if (bad_node) bad = true;
    }
    if (bad) flags |= ST_NONFINITE;
    if (flags) atomicOr(status, flags);
}

template <typename T>
__global__ void k_nodes(GeomP P, const double* __restrict__ nodes, const int* __restrict__ fil_of,
                        const int* __restrict__ prev, const int64_t* __restrict__ off, const double* __restrict__ shift,
                        const T* __restrict__ hseg, const T* __restrict__ dp, const T* __restrict__ ds,
                        const T* __restrict__ Mm, const T* __restrict__ Tper, SrRec<T>* __restrict__ sr_rec,
                        int* __restrict__ sr_key, LrRec<T>* __restrict__ lr_rec, int* __restrict__ lr_key,
                        SrTgt<T>* __restrict__ tgt, double* __restrict__ vls, double* __restrict__ pls,
                        double* __restrict__ part_local, double* __restrict__ part_self,
                        double* __restrict__ psi_local, double* __restrict__ psi_self, int* __restrict__ status,
                        const T* __restrict__ Dd)
{
    k_nodes_body<T>(P, nodes, fil_of, prev, off, shift, hseg, dp, ds, Mm, Tper, sr_rec, sr_key, lr_rec, lr_key, tgt,
        vls, pls, part_local, part_self, psi_local, psi_self, status, Dd, blockIdx.x);
}

// Batched forms: every member of a batch in one launch.
template <typename T>
__global__ void k_spline_warp_b(const SplineD<T>* __restrict__ d, const int* __restrict__ bs, int n)
{
    int bid, nb;
    const SplineD<T>& a = d[batch_member(bs, n, bid, nb)];
    k_spline_warp_body<T>(a.nodes, a.off, a.shift, a.nfil, a.nmax, a.hseg, a.dp, a.ds, a.Mm, a.Tper, bid);
}

template <typename T>
__global__ void __launch_bounds__(128) k_nodes_b(const NodesD<T>* __restrict__ d, const int* __restrict__ bs, int n)
{
    int bid, nb;
    const NodesD<T>& a = d[batch_member(bs, n, bid, nb)];
    k_nodes_body<T>(a.P, a.nodes, a.fil_of, a.prev, a.off, a.shift, a.hseg, a.dp, a.ds, a.Mm, a.Tper, a.sr_rec,
                    a.sr_key, a.lr_rec, a.lr_key, a.tgt, a.vls, a.pls, nullptr, nullptr, nullptr, nullptr, a.status,
                    a.Dd, bid);
}

template <typename T>
size_t spline_smem(int nmax)
{
    return 9 * (size_t)nmax * sizeof(T);
}

template <typename T>
cudaError_t launch_spline_b(const BatchL& L, cudaStream_t s)
{
    if (L.total <= 0) return cudaSuccess;
    if (L.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_spline_warp_b<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)L.smem);
        if (e != cudaSuccess) return e;
    }
    k_spline_warp_b<T><<<L.total, 32, L.smem, s>>>((const SplineD<T>*)L.desc, L.bstart, L.n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_nodes_b(const BatchL& L, cudaStream_t s)
{
    if (L.total > 0) k_nodes_b<T><<<L.total, 128, 0, s>>>((const NodesD<T>*)L.desc, L.bstart, L.n);
    return cudaGetLastError();
}

template size_t spline_smem<float>(int);
template size_t spline_smem<double>(int);
template cudaError_t launch_spline_b<float>(const BatchL&, cudaStream_t);
template cudaError_t launch_spline_b<double>(const BatchL&, cudaStream_t);
template cudaError_t launch_nodes_b<float>(const BatchL&, cudaStream_t);
template cudaError_t launch_nodes_b<double>(const BatchL&, cudaStream_t);

// Energy line integral (Sec. 2.4, Eq. kinetic_energy_streamfunction): per
// filament, f_j = (psi_local + psi^(n) - psi^(f)_self)(s_j) . sdot(tau_j) at
// the nodes, interpolated by the periodic cubic spline with the same knots
// (float64 moments m_j from the cyclic tridiagonal system), integrated exactly:
// int f dtau = sum_j [h_j (f_j + f_{j+1}) / 2 - h_j^3 (m_j + m_{j+1}) / 24].
// One warp per filament; smem 5 * nmax doubles; the sum over filaments is
// added to *acc.
template <typename T>
__global__ void k_energy_line(const int64_t* __restrict__ off, const double* __restrict__ shift, int nfil, int nmax,
                              const T* __restrict__ hseg, const T* __restrict__ dp, const T* __restrict__ Mm,
                              const T* __restrict__ Tper, const double* __restrict__ pls, const double* __restrict__ psr,
                              double* __restrict__ acc, double* __restrict__ per_fil)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    double* sh_h = reinterpret_cast<double*>(sm_raw);
    double* sh_f = sh_h + nmax;   // values f_j
    double* sh_r = sh_f + nmax;   // right-hand side, then moments
    double* sh_z = sh_r + nmax;   // Sherman-Morrison vector
    double* sh_c = sh_z + nmax;   // modified super-diagonal
    const int f = blockIdx.x;
    if (f >= nfil) return;
    const int lane = threadIdx.x;
    const int64_t o = off[f];
    const int n = (int)(off[f + 1] - o);
    const double Tp = (double)Tper[f];
    const double dr0 = shift[3 * f] / Tp, dr1 = shift[3 * f + 1] / Tp, dr2 = shift[3 * f + 2] / Tp;
    for (int j = lane; j < n; j += 32) {
        const int jn = (j + 1 < n) ? j + 1 : 0;
        const double h = (double)hseg[o + j];
        sh_h[j] = h;
        double fj = 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double Mj = (double)Mm[3 * (o + j) + c], Mn = (double)Mm[3 * (o + jn) + c];
            const double drc = c == 0 ? dr0 : (c == 1 ? dr1 : dr2);
            const double sdot = (double)dp[3 * (o + j) + c] / h - h * (2.0 * Mj + Mn) / 6.0 + drc;
            const double psi = pls[3 * (o + j) + c] + psr[3 * (o + j) + c];
            fj += psi * sdot;
        }
        sh_f[j] = fj;
    }
    __syncwarp();
    for (int j = lane; j < n; j += 32) {
        const int jm = j == 0 ? n - 1 : j - 1, jn = (j + 1 < n) ? j + 1 : 0;
        sh_r[j] = 6.0 * ((sh_f[jn] - sh_f[j]) / sh_h[j] - (sh_f[j] - sh_f[jm]) / sh_h[jm]);
        sh_z[j] = 0.0;
    }
    __syncwarp();
    const double hl = sh_h[n - 1];
    const double gamma = -2.0 * (hl + sh_h[0]);
    if (lane == 0) {
        sh_z[0] = gamma;
        sh_z[n - 1] = hl;
    }
    __syncwarp();
    if (lane < 2) {  // lane 0: the right-hand side, lane 1: the Sherman-Morrison vector
        double* r = lane == 0 ? sh_r : sh_z;
        double cprev = 0, dprev = 0, hm = hl;
        for (int j = 0; j < n; ++j) {
            const double hj = sh_h[j];
            const double a = (j == 0) ? 0.0 : hm;
            double bb = 2.0 * (hm + hj);
            if (j == 0) bb -= gamma;
            if (j == n - 1) bb -= hl * hl / gamma;
            const double c = (j == n - 1) ? 0.0 : hj;
            const double im = 1.0 / (bb - a * cprev);
            cprev = c * im;
            dprev = (r[j] - a * dprev) * im;
            if (lane == 0) sh_c[j] = cprev;
            r[j] = dprev;
            hm = hj;
        }
        __syncwarp(0x3u);
        double x = r[n - 1];
        for (int j = n - 2; j >= 0; --j) {
            x = r[j] - sh_c[j] * x;
            r[j] = x;
        }
    }
    __syncwarp();
    const double vfac = hl / gamma;
    const double fac = (sh_r[0] + vfac * sh_r[n - 1]) / (1.0 + sh_z[0] + vfac * sh_z[n - 1]);
    double part = 0.0;
    for (int j = lane; j < n; j += 32) {
        const int jn = (j + 1 < n) ? j + 1 : 0;
        const double mj = sh_r[j] - fac * sh_z[j], mn = sh_r[jn] - fac * sh_z[jn];
        const double h = sh_h[j];
        part += 0.5 * h * (sh_f[j] + sh_f[jn]) - h * h * h * (mj + mn) / 24.0;
    }
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) part += __shfl_xor_sync(0xffffffffu, part, k);
    if (lane == 0) {
        if (per_fil)
            per_fil[f] = part;  // deterministic: summed in filament order on the host
        else
            atomicAdd(acc, part);
    }
}

// The periodic quintic spline solve of the curve fit below (k_spline_quintic).
__device__ void q_solve(int n, double* __restrict__ t, double xlast[6]);
__device__ __forceinline__ void q_node(const double* __restrict__ t, int m, const double xlast[6], int j, int c,
                                       double& D, double& M);

// The same line integral on a quintic curve (order 6): f_j = psi_j .
// sdot(tau_j), with sdot = D_j + n_l L / T the first derivative of the
// quintic at the node, is interpolated by the periodic quintic spline with
// the same knots (q_solve on the increments f_{j+1} - f_j, no drift) and
// integrated exactly, segment by segment (the Hermite quintic's integral):
//   int f dtau = h (f_j + f_{j+1}) / 2 + h^2 (F'_j - F'_{j+1}) / 10 + h^3 (F''_j + F''_{j+1}) / 120.
// One thread per filament; ftmp holds 19 float64 per node (the solver's 18
// and f_j).
template <typename T>
__global__ void k_energy_line_quintic(const int64_t* __restrict__ off, const double* __restrict__ shift, int nfil,
                                      const T* __restrict__ hseg, const T* __restrict__ Dd,
                                      const T* __restrict__ Tper, const double* __restrict__ pls,
                                      const double* __restrict__ psr, double* __restrict__ ftmp,
                                      double* __restrict__ acc, double* __restrict__ per_fil)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfil) return;
    const int64_t o = off[f];
    const int n = (int)(off[f + 1] - o);
    double* t = ftmp + 19 * (size_t)o;
    double* fv = t + 18 * (size_t)n;  // f_j after the solver's scratch
    const double Tp = (double)Tper[f];
    const double dr[3] = { shift[3 * f] / Tp, shift[3 * f + 1] / Tp, shift[3 * f + 2] / Tp };
    for (int j = 0; j < n; ++j) {
        double fj = 0.0;
        for (int c = 0; c < 3; ++c)
            fj += (pls[3 * (o + j) + c] + psr[3 * (o + j) + c]) * ((double)Dd[3 * (o + j) + c] + dr[c]);
        fv[j] = fj;
    }
    for (int j = 0; j < n; ++j) {
        t[18 * j] = (double)hseg[o + j];
        t[18 * j + 1] = fv[j + 1 < n ? j + 1 : 0] - fv[j];
        t[18 * j + 2] = 0.0;
        t[18 * j + 3] = 0.0;
    }
    double xlast[6];
    q_solve(n, t, xlast);
    const int m = n - 1;
    double part = 0.0;
    double Dj, Mj;
    q_node(t, m, xlast, 0, 0, Dj, Mj);
    const double D0 = Dj, M0 = Mj;
    for (int j = 0; j < n; ++j) {
        const int jn = j + 1 < n ? j + 1 : 0;
        double Dn, Mn;
        if (jn == 0) {
            Dn = D0;
            Mn = M0;
        } else {
            q_node(t, m, xlast, jn, 0, Dn, Mn);
        }
        const double h = t[18 * j];
        part += 0.5 * h * (fv[j] + fv[jn]) + h * h * (Dj - Dn) / 10.0 + h * h * h * (Mj + Mn) / 120.0;
        Dj = Dn;
        Mj = Mn;
    }
    if (per_fil)
        per_fil[f] = part;  // deterministic: summed in filament order on the host
    else
        atomicAdd(acc, part);
}

template <typename T>
cudaError_t launch_energy_line(const double* nodes, const Work& w, int nfil, int nmax, cudaStream_t s, bool det)
{
    (void)nodes;
    if (nfil <= 0) return cudaSuccess;
    if (w.Dd) {  // quintic curves
        const int tb = 64;
        k_energy_line_quintic<T><<<(nfil + tb - 1) / tb, tb, 0, s>>>(w.off, w.shift, nfil, (const T*)w.hseg,
                                                                     (const T*)w.Dd, (const T*)w.Tper, w.pls, w.psr,
                                                                     w.qtmp, w.energy_acc + 1, det ? w.lpart : nullptr);
        return cudaGetLastError();
    }
    const size_t sm = 5 * (size_t)nmax * sizeof(double);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_energy_line<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_energy_line<T><<<nfil, 32, sm, s>>>(w.off, w.shift, nfil, nmax, (const T*)w.hseg, (const T*)w.dp,
                                          (const T*)w.Mm, (const T*)w.Tper, w.pls, w.psr,
                                          w.energy_acc + 1, det ? w.lpart : nullptr);
    return cudaGetLastError();
}

template cudaError_t launch_energy_line<float>(const double*, const Work&, int, int, cudaStream_t, bool);
template cudaError_t launch_energy_line<double>(const double*, const Work&, int, int, cudaStream_t, bool);

// Quadrature export for bs_get_quadrature (float64, wrapped positions).
template <typename T>
__global__ void k_export_quad(GeomP P, const double* __restrict__ nodes, const int* __restrict__ fil_of,
                              const int64_t* __restrict__ off, const double* __restrict__ shift,
                              const T* __restrict__ hseg, const T* __restrict__ dp, const T* __restrict__ Mm,
                              const T* __restrict__ Tper, double* __restrict__ qX, double* __restrict__ qq,
                              const T* __restrict__ Dd)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.N) return;
    const int f = fil_of[j];
    const int jn = (j + 1 < (int)off[f + 1]) ? j + 1 : (int)off[f];
    const T Tp = Tper[f];
    const T drift[3] = { (T)shift[3 * f] / Tp, (T)shift[3 * f + 1] / Tp, (T)shift[3 * f + 2] / Tp };
    SegPoly<T> S;
    make_poly(S, hseg, dp, Mm, j, jn, drift, Dd);
    for (int i = 0; i < P.Q; ++i) {
        const T u = (T)P.gh[i] * S.h;
        T del[3], sd[3];
        S.eval(u, del, sd);
        const T wq = (T)P.gw[i] * S.h;
        const int p = j * P.Q + i;
        bool b = false;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            qX[3 * p + c] = wrap_box(nodes[3 * j + c] + (double)del[c], P.L[c], P.iL[c], b);
            qq[3 * p + c] = (double)(wq * sd[c]);
        }
    }
}


// ---------------------------------------------------------------------------
// Quintic spline fit (order 6, Appendix B): one thread per filament, float64.
// The periodic C4 quintic through the nodes at the chord-length knots is
// written per segment as the Hermite quintic of its end values, first
// derivatives D and second derivatives M (make_poly).  Continuity of the
// third and fourth derivatives at node j gives, per component,
//   L_j X_{j-1} + B_j X_j + U_j X_{j+1} = R_j,   X_j = (D_j, M_j),
//   L_j = [[-24/a^2, -3/a], [-168/a^3, -24/a^2]]
//   B_j = [[36/h^2 - 36/a^2, 9/a + 9/h], [-192/a^3 - 192/h^3, 36/a^2 - 36/h^2]]
//   U_j = [[24/h^2, -3/h], [-168/h^3, 24/h^2]]
//   R_j = (60 dp_j/h^3 - 60 dp_{j-1}/a^3, -360 dp_j/h^4 - 360 dp_{j-1}/a^4)
// with a = h_{j-1}, h = h_j (cyclic in j).  Solved by block elimination on
// X_0..X_{n-2} with X_{n-1} as a border: X_j = Y_j + Z_j X_{n-1}, then the
// last equation gives X_{n-1} (a 2 x 2 system).  The three components share
// the matrix: every right-hand side is a 2 x 5 block (3 components + 2
// border columns).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void q_blocks(double a, double h, double L[4], double B[4], double U[4])
{
    const double a2 = a * a, a3 = a2 * a, h2 = h * h, h3 = h2 * h;
    L[0] = -24.0 / a2; L[1] = -3.0 / a; L[2] = -168.0 / a3; L[3] = -24.0 / a2;
    B[0] = 36.0 / h2 - 36.0 / a2; B[1] = 9.0 / a + 9.0 / h;
    B[2] = -192.0 / a3 - 192.0 / h3; B[3] = 36.0 / a2 - 36.0 / h2;
    U[0] = 24.0 / h2; U[1] = -3.0 / h; U[2] = -168.0 / h3; U[3] = 24.0 / h2;
}

// inverse of the 2 x 2 matrix m (row major)
__device__ __forceinline__ void inv2(const double m[4], double r[4])
{
    const double id = 1.0 / (m[0] * m[3] - m[1] * m[2]);
    r[0] = m[3] * id; r[1] = -m[1] * id; r[2] = -m[2] * id; r[3] = m[0] * id;
}

// c (2 x 5) = a (2 x 2) * b (2 x 5)
__device__ __forceinline__ void mul25(const double a[4], const double b[10], double c[10])
{
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        c[k] = a[0] * b[k] + a[1] * b[5 + k];
        c[5 + k] = a[2] * b[k] + a[3] * b[5 + k];
    }
}

// Solves the cyclic block system above for the node lengths t[18 j] and
// the three increments t[18 j + 1 + c] of every node j of one filament (18
// float64 per node of scratch; n >= 3).  On return (D_j, M_j) of component c
// are q_node(t, m, xlast, j, c, D, M), m = n - 1.
__device__ void q_solve(int n, double* __restrict__ t, double xlast[6])
{
    const int m = n - 1;
    double L[4], B[4], U[4], Wm[4], iv[4], Bp[10], tmp10[10];
    // forward elimination over j = 0..m-1
    for (int j = 0; j < m; ++j) {
        const int jm = j == 0 ? n - 1 : j - 1;
        const double a = t[18 * jm], h = t[18 * j];
        q_blocks(a, h, L, B, U);
        double rhs[10];
        for (int c = 0; c < 3; ++c) {
            const double dj = t[18 * j + 1 + c], dm = t[18 * jm + 1 + c];
            rhs[c] = 60.0 * dj / (h * h * h) - 60.0 * dm / (a * a * a);
            rhs[5 + c] = -360.0 * dj / (h * h * h * h) - 360.0 * dm / (a * a * a * a);
        }
        rhs[3] = rhs[4] = rhs[8] = rhs[9] = 0.0;
        if (j == 0) {  // border column: -L_0 X_{n-1}
            rhs[3] -= L[0]; rhs[4] -= L[1]; rhs[8] -= L[2]; rhs[9] -= L[3];
        }
        if (j == m - 1) {  // border column: -U_{m-1} X_{n-1}
            rhs[3] -= U[0]; rhs[4] -= U[1]; rhs[8] -= U[2]; rhs[9] -= U[3];
        }
        double Bj[4] = { B[0], B[1], B[2], B[3] };
        if (j > 0) {
            // W = L_j Bp_{j-1}^{-1}; B'_j = B_j - W U_{j-1}; rhs'_j = rhs_j - W rhs'_{j-1}
            const double* pb = t + 18 * (j - 1) + 4;
            double Bprev[4] = { pb[0], pb[1], pb[2], pb[3] };
            inv2(Bprev, iv);
            Wm[0] = L[0] * iv[0] + L[1] * iv[2]; Wm[1] = L[0] * iv[1] + L[1] * iv[3];
            Wm[2] = L[2] * iv[0] + L[3] * iv[2]; Wm[3] = L[2] * iv[1] + L[3] * iv[3];
            double Lq[4], Bq[4], Uq[4];
            const int jmm = j - 2 < 0 ? n - 1 : j - 2;  // U_{j-1} uses h_{j-2}, h_{j-1}
            q_blocks(t[18 * jmm], t[18 * (j - 1)], Lq, Bq, Uq);
            Bj[0] -= Wm[0] * Uq[0] + Wm[1] * Uq[2]; Bj[1] -= Wm[0] * Uq[1] + Wm[1] * Uq[3];
            Bj[2] -= Wm[2] * Uq[0] + Wm[3] * Uq[2]; Bj[3] -= Wm[2] * Uq[1] + Wm[3] * Uq[3];
            const double* pr = t + 18 * (j - 1) + 8;
            for (int k = 0; k < 10; ++k) Bp[k] = pr[k];
            mul25(Wm, Bp, tmp10);
            for (int k = 0; k < 10; ++k) rhs[k] -= tmp10[k];
        }
        for (int k = 0; k < 4; ++k) t[18 * j + 4 + k] = Bj[k];
        for (int k = 0; k < 10; ++k) t[18 * j + 8 + k] = rhs[k];
    }
    // back substitution: X_j = B'_j^{-1} (rhs'_j - U_j X_{j+1}), stored over rhs'_j
    for (int j = m - 1; j >= 0; --j) {
        double rhs[10];
        for (int k = 0; k < 10; ++k) rhs[k] = t[18 * j + 8 + k];
        if (j < m - 1) {
            const int jm = j == 0 ? n - 1 : j - 1;
            q_blocks(t[18 * jm], t[18 * j], L, B, U);
            const double* xn = t + 18 * (j + 1) + 8;
            for (int k = 0; k < 10; ++k) Bp[k] = xn[k];
            mul25(U, Bp, tmp10);
            for (int k = 0; k < 10; ++k) rhs[k] -= tmp10[k];
        }
        double Bj[4] = { t[18 * j + 4], t[18 * j + 5], t[18 * j + 6], t[18 * j + 7] };
        inv2(Bj, iv);
        mul25(iv, rhs, tmp10);
        for (int k = 0; k < 10; ++k) t[18 * j + 8 + k] = tmp10[k];
    }
    // last equation: (L_{n-1} Z_{n-2} + B_{n-1} + U_{n-1} Z_0) X_{n-1} = R_{n-1} - L_{n-1} Y_{n-2} - U_{n-1} Y_0
    const double a = t[18 * (m - 1)], h = t[18 * m];
    q_blocks(a, h, L, B, U);
    const double* x0 = t + 8;                 // X_0 (Y | Z)
    const double* xl = t + 18 * (m - 1) + 8;  // X_{n-2}
    double Sm[4];
    // Z columns are entries 3, 4 (row 0) and 8, 9 (row 1)
    Sm[0] = B[0] + L[0] * xl[3] + L[1] * xl[8] + U[0] * x0[3] + U[1] * x0[8];
    Sm[1] = B[1] + L[0] * xl[4] + L[1] * xl[9] + U[0] * x0[4] + U[1] * x0[9];
    Sm[2] = B[2] + L[2] * xl[3] + L[3] * xl[8] + U[2] * x0[3] + U[3] * x0[8];
    Sm[3] = B[3] + L[2] * xl[4] + L[3] * xl[9] + U[2] * x0[4] + U[3] * x0[9];
    inv2(Sm, iv);
    for (int c = 0; c < 3; ++c) {
        const double dj = t[18 * m + 1 + c], dm = t[18 * (m - 1) + 1 + c];
        const double r0 = 60.0 * dj / (h * h * h) - 60.0 * dm / (a * a * a) - (L[0] * xl[c] + L[1] * xl[5 + c]) -
                          (U[0] * x0[c] + U[1] * x0[5 + c]);
        const double r1 = -360.0 * dj / (h * h * h * h) - 360.0 * dm / (a * a * a * a) -
                          (L[2] * xl[c] + L[3] * xl[5 + c]) - (U[2] * x0[c] + U[3] * x0[5 + c]);
        xlast[c] = iv[0] * r0 + iv[1] * r1;
        xlast[3 + c] = iv[2] * r0 + iv[3] * r1;
    }
}

// First and second derivative of component c at node j after q_solve.
__device__ __forceinline__ void q_node(const double* __restrict__ t, int m, const double xlast[6], int j, int c,
                                       double& D, double& M)
{
    if (j == m) {
        D = xlast[c];
        M = xlast[3 + c];
        return;
    }
    const double* x = t + 18 * j + 8;
    D = x[c] + x[3] * xlast[c] + x[4] * xlast[3 + c];
    M = x[5 + c] + x[8] * xlast[c] + x[9] * xlast[3 + c];
}

template <typename T>
__global__ void k_spline_quintic(const double* __restrict__ nodes, const int64_t* __restrict__ off,
                                 const double* __restrict__ shift, int nfil, T* __restrict__ hseg, T* __restrict__ dp,
                                 T* __restrict__ ds, T* __restrict__ Mm, T* __restrict__ Dd, T* __restrict__ Tper,
                                 double* __restrict__ tmp)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nfil) return;
    const int64_t o = off[f];
    const int n = (int)(off[f + 1] - o);
    const double sh[3] = { shift[3 * f], shift[3 * f + 1], shift[3 * f + 2] };
    // per node in tmp: h, dp[3] (float64), then the eliminated block (4) and right sides (10)
    double* t = tmp + 18 * (size_t)o;
    double Tsum = 0.0;
    for (int j = 0; j < n; ++j) {
        const double* a = nodes + 3 * (o + j);
        const double* b = nodes + 3 * (j + 1 < n ? o + j + 1 : o);
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = b[c] + (j + 1 < n ? 0.0 : sh[c]) - a[c];
        const double h = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        Tsum += h;
        t[18 * j] = h;
        for (int c = 0; c < 3; ++c) t[18 * j + 1 + c] = d[c];
        hseg[o + j] = (T)h;
        for (int c = 0; c < 3; ++c) ds[3 * (o + j) + c] = (T)d[c];
    }
    Tper[f] = (T)Tsum;
    const double invT = 1.0 / Tsum;
    for (int j = 0; j < n; ++j)
        for (int c = 0; c < 3; ++c) {
            t[18 * j + 1 + c] -= sh[c] * t[18 * j] * invT;  // periodic increments
            dp[3 * (o + j) + c] = (T)t[18 * j + 1 + c];
        }
    double xlast[6];
    q_solve(n, t, xlast);
    const int m = n - 1;
    for (int j = 0; j < n; ++j)
        for (int c = 0; c < 3; ++c) {
            double D, M;
            q_node(t, m, xlast, j, c, D, M);
            Dd[3 * (o + j) + c] = (T)D;
            Mm[3 * (o + j) + c] = (T)M;
        }
}

template <typename T>
cudaError_t launch_spline(const double* nodes, const Work& w, int nfil, cudaStream_t s)
{
    if (nfil <= 0) return cudaSuccess;
    if (w.Dd) {  // quintic
        const int tb = 64;
        k_spline_quintic<T><<<(nfil + tb - 1) / tb, tb, 0, s>>>(nodes, w.off, w.shift, nfil, (T*)w.hseg, (T*)w.dp,
                                                                (T*)w.ds, (T*)w.Mm, (T*)w.Dd, (T*)w.Tper, w.qtmp);
        return cudaGetLastError();
    }
    const size_t sm = 9 * (size_t)w.nmax_fil * sizeof(T);
    if (sm <= kSplineSmemMax) {
        if (sm > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k_spline_warp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            if (e != cudaSuccess) return e;
        }
        k_spline_warp<T><<<nfil, 32, sm, s>>>(nodes, w.off, w.shift, nfil, w.nmax_fil, (T*)w.hseg, (T*)w.dp,
                                               (T*)w.ds, (T*)w.Mm, (T*)w.Tper);
        return cudaGetLastError();
    }
    // filaments too long for shared memory: one thread per filament, in global memory
    const int tb = 64;
    k_spline<T><<<(nfil + tb - 1) / tb, tb, 0, s>>>(nodes, w.off, w.shift, nfil, (T*)w.hseg, (T*)w.dp, (T*)w.ds,
                                                    (T*)w.Mm, (T*)w.cpr, (T*)w.zz, (T*)w.Tper);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_nodes(const GeomP& P, const double* nodes, const Work& w, double* part_local, double* part_self,
                         double* psi_local, double* psi_self, cudaStream_t s)
{
    if (P.N <= 0) return cudaSuccess;
    const int tb = 128;
    k_nodes<T><<<(P.N + tb - 1) / tb, tb, 0, s>>>(
        P, nodes, w.fil_of, w.prev, w.off, w.shift, (const T*)w.hseg, (const T*)w.dp, (const T*)w.ds,
        (const T*)w.Mm, (const T*)w.Tper, (SrRec<T>*)w.sr_rec, w.sr_key, (LrRec<T>*)w.lr_rec, w.lr_key,
        (SrTgt<T>*)w.tgt, w.vls, w.pls, part_local, part_self, psi_local, psi_self, w.status, (const T*)w.Dd);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_export_quadrature(const GeomP& P, const double* nodes, const Work& w, double* qX, double* qq,
                                     cudaStream_t s)
{
    if (P.N <= 0) return cudaSuccess;
    const int tb = 128;
    k_export_quad<T><<<(P.N + tb - 1) / tb, tb, 0, s>>>(P, nodes, w.fil_of, w.off, w.shift, (const T*)w.hseg,
                                                         (const T*)w.dp, (const T*)w.Mm, (const T*)w.Tper, qX, qq,
                                                         (const T*)w.Dd);
    return cudaGetLastError();
}

template cudaError_t launch_spline<float>(const double*, const Work&, int, cudaStream_t);
template cudaError_t launch_spline<double>(const double*, const Work&, int, cudaStream_t);
template cudaError_t launch_nodes<float>(const GeomP&, const double*, const Work&, double*, double*, double*, double*,
                                         cudaStream_t);
template cudaError_t launch_nodes<double>(const GeomP&, const double*, const Work&, double*, double*, double*, double*,
                                          cudaStream_t);
template cudaError_t launch_export_quadrature<float>(const GeomP&, const double*, const Work&, double*, double*,
                                                     cudaStream_t);
template cudaError_t launch_export_quadrature<double>(const GeomP&, const double*, const Work&, double*, double*,
                                                      cudaStream_t);

}  // namespace bsw
