// Short-range velocity and streamfunction (Sec. 3.2, Eqs.
// velocity_shortrange and streamfunction_shortrange) at every node:
//   v^(n)(s_j)   = kappa/4pi sum_{q not in C_0(j), |r| < r_c} g^(n)(alpha r) (r x q) / r^3,
//   psi^(n)(s_j) = kappa/4pi sum_{same} erfc(alpha r) q / r,
// r the minimum image of (source - node), g^(n)(x) = erfc(x) + 2x/sqrt(pi) e^{-x^2}.
//
// Sources are binned in cells of edge >= r_c/m (m = 3 in Sec. 5.3) and
// sorted by cell with x fastest, so the 2m+1 cells of a row along x form one
// contiguous range of the sorted array (two when the row wraps).  One warp
// per node walks the (2m+1)^2 rows around its cell.  Positions are cell
// index + offset from the cell origin: the separation is
// (integer cell difference) * h + (offset difference), which keeps T
// precision relative to r instead of relative to L.
#include <math.h>

#include "bs_internal.cuh"

namespace bsw {

__device__ __forceinline__ int imod(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

// Signed periodic difference of two cell indices in [-n/2, n/2).
__device__ __forceinline__ int cdiff(int a, int b, int n)
{
    int d = a - b;
    if (d >= (n + 1) / 2) d -= n;
    if (d < -(n / 2)) d += n;
    return d;
}

// erfc(x) exp(x^2), x >= 0, in float32: a least-squares fit (weighted for
// relative error, degree 10 in t = 1 / (1 + x / 2), on [0, 8]) written by
// gen_erfcx_fit.py; 3.4e-7 relative error evaluated in float32.  Beyond
// x = 8 the factor exp(-x^2) it multiplies is below 2e-28.
__device__ __forceinline__ float erfcx_f(float x)
{
    constexpr float c[11] = { 1.441113045e-05f, 2.817091850e-01f, 2.866406861e-01f, 2.157398867e-01f,
                              3.128657818e-01f, -3.176314365e-01f, 7.893466267e-01f, -1.078447950e+00f,
                              7.163310796e-01f, -2.393311398e-01f, 3.276285984e-02f };
    const float t = 1.0f / (1.0f + 0.5f * x);
    float v = c[10];
#pragma unroll
    for (int k = 9; k >= 0; --k) v = fmaf(v, t, c[k]);
    return v;
}

// erfc(x) given e = exp(-x^2): float32 through the fit above, float64 exact.
template <typename T>
__device__ __forceinline__ T erfc_e(T x, T e);
template <>
__device__ __forceinline__ float erfc_e<float>(float x, float e) { return e * erfcx_f(x); }
template <>
__device__ __forceinline__ double erfc_e<double>(double x, double) { return erfc(x); }

// One warp per target node.  The lanes first list the source ranges of the
// (2m+1)^2 neighbour rows (32 rows at a time; a row wrapping around the box
// gives two ranges; rows and row ends beyond r_c are cut), prefix-sum their
// lengths, then stride through the flattened candidate list, so every lane
// has work however short the rows are.  Each lane finds the row of its candidate by a binary search over the
// lanes' inclusive sums.  The per-lane partial sums are reduced at the end.
template <typename T>
__global__ void __launch_bounds__(256) k_short(ShortP P, const SrTgt<T>* __restrict__ tgt, const int* __restrict__ prev,
                                               const int* __restrict__ start, const SrRec<T>* __restrict__ src,
                                               T* __restrict__ vsr, T* __restrict__ psr)
{
    const int lane = threadIdx.x & 31;
    const int j = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (j >= P.N) return;  // whole warps exit together
    const SrTgt<T> t = tgt[j];
    const int jp = prev[j];
    const int nc0 = P.nc[0], nc1 = P.nc[1], nc2 = P.nc[2];
    const int cx = t.cell % nc0;
    const int cy = (t.cell / nc0) % nc1;
    const int cz = t.cell / (nc0 * nc1);
    const T h0 = (T)P.hc[0], h1 = (T)P.hc[1], h2 = (T)P.hc[2];
    const T L0 = (T)P.L[0], L1 = (T)P.L[1], L2 = (T)P.L[2];
    const T rc2 = (T)P.rc2;
    const T alpha = (T)P.alpha;
    const T two_over_sqrtpi = (T)1.12837916709551257390;
    const int m = P.m;
    // neighbour ranges per axis: all cells when 2m+1 >= n
    const bool fullx = (2 * m + 1 >= nc0), fully = (2 * m + 1 >= nc1), fullz = (2 * m + 1 >= nc2);
    const int ny = fully ? nc1 : 2 * m + 1, nz = fullz ? nc2 : 2 * m + 1;
    const int nrows = ny * nz;
    // Rows whose y-z slab lies wholly beyond r_c of the node are skipped, and
    // a row's x cells are cut to those meeting the chord of the r_c sphere
    // at the slab's distance.  The pair test below stays exact; the margin
    // keeps the cut conservative under rounding.
    const T rcm2 = rc2 * (T)1.0001;
    const T ih0 = (T)1 / h0;

    T v0 = 0, v1 = 0, v2 = 0, p0 = 0, p1 = 0, p2 = 0;
    for (int rb = 0; rb < nrows; rb += 32) {
        // this lane's row
        const int r = rb + lane;
        int s0 = 0, n0 = 0, s1 = 0, n1r = 0, dyi = 0, dzi = 0;
        if (r < nrows) {
            const int iz = r / ny, iy = r - iz * ny;
            const int zc = fullz ? iz : imod(cz - m + iz, nc2);
            const int yc = fully ? iy : imod(cy - m + iy, nc1);
            dzi = cdiff(zc, cz, nc2);
            dyi = cdiff(yc, cy, nc1);
            // gaps between the node and the row's y and z slabs
            T gy = (T)0, gz = (T)0;
            if (!fully) gy = dyi > 0 ? dyi * h1 - t.o[1] : (dyi < 0 ? t.o[1] - (dyi + 1) * h1 : (T)0);
            if (!fullz) gz = dzi > 0 ? dzi * h2 - t.o[2] : (dzi < 0 ? t.o[2] - (dzi + 1) * h2 : (T)0);
            gy = gy > (T)0 ? gy : (T)0;
            gz = gz > (T)0 ? gz : (T)0;
            const T d2 = gy * gy + gz * gz;
            if (d2 < rcm2) {
                // x-ranges of the row: one or two contiguous runs [xa0, xb0], [xa1, xb1]
                int xa0, xb0, xa1 = 0, xb1 = -1;
                if (fullx) {
                    xa0 = 0;
                    xb0 = nc0 - 1;
                } else {
                    const T ext = sqrt(rcm2 - d2);
                    int lo = (int)floor((t.o[0] - ext) * ih0), hi = (int)floor((t.o[0] + ext) * ih0);
                    lo = cx + (lo < -m ? -m : lo);
                    hi = cx + (hi > m ? m : hi);
                    if (lo < 0) {
                        xa0 = lo + nc0; xb0 = nc0 - 1; xa1 = 0; xb1 = hi;
                    } else if (hi >= nc0) {
                        xa0 = lo; xb0 = nc0 - 1; xa1 = 0; xb1 = hi - nc0;
                    } else {
                        xa0 = lo; xb0 = hi;
                    }
                }
                const int row = (zc * nc1 + yc) * nc0;
                s0 = start[row + xa0];
                n0 = start[row + xb0 + 1] - s0;
                if (xb1 >= xa1) {
                    s1 = start[row + xa1];
                    n1r = start[row + xb1 + 1] - s1;
                }
            }
        }
        // inclusive prefix sum of the lanes' candidate counts
        int inc = n0 + n1r;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        const int total = __shfl_sync(0xffffffffu, inc, 31);
        for (int cb = 0; cb < total; cb += 32) {  // warp-uniform trip count: every shuffle has all lanes
            const int c = cb + lane;
            // owner lane: the first lane whose inclusive sum exceeds c
            int lo = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int probe = __shfl_sync(0xffffffffu, inc, lo + step - 1);
                if (probe <= c) lo += step;
            }
            lo = lo > 31 ? 31 : lo;
            const int own_inc = __shfl_sync(0xffffffffu, inc, lo);
            const int own_n0 = __shfl_sync(0xffffffffu, n0, lo);
            const int own_n1 = __shfl_sync(0xffffffffu, n1r, lo);
            const int own_s0 = __shfl_sync(0xffffffffu, s0, lo);
            const int own_s1 = __shfl_sync(0xffffffffu, s1, lo);
            const int own_dy = __shfl_sync(0xffffffffu, dyi, lo);
            const int own_dz = __shfl_sync(0xffffffffu, dzi, lo);
            if (c >= total) continue;
            const int local = c - (own_inc - own_n0 - own_n1);
            const int k = local < own_n0 ? own_s0 + local : own_s1 + (local - own_n0);
            const SrRec<T> S = src[k];
            if (S.seg == j || S.seg == jp) continue;  // C_0 of the node (Eq. BS_on_vortex)
            T rx = (T)cdiff(S.cx, cx, nc0) * h0 + (S.o[0] - t.o[0]);
            T ry = (T)own_dy * h1 + (S.o[1] - t.o[1]);
            T rz = (T)own_dz * h2 + (S.o[2] - t.o[2]);
            // exact minimum image when a cell difference sits at n/2
            rx = rx > (T)0.5 * L0 ? rx - L0 : (rx < (T)-0.5 * L0 ? rx + L0 : rx);
            ry = ry > (T)0.5 * L1 ? ry - L1 : (ry < (T)-0.5 * L1 ? ry + L1 : ry);
            rz = rz > (T)0.5 * L2 ? rz - L2 : (rz < (T)-0.5 * L2 ? rz + L2 : rz);
            const T r2 = rx * rx + ry * ry + rz * rz;
            if (r2 >= rc2 || r2 == (T)0) continue;
            const T rr = sqrt(r2);
            const T x = alpha * rr;
            const T e = exp(-x * x);
            const T ec = erfc_e(x, e);
            const T g = ec + two_over_sqrtpi * x * e;
            const T ir = (T)1 / rr;
            const T fv = g * ir * ir * ir;
            v0 += fv * (ry * S.q[2] - rz * S.q[1]);
            v1 += fv * (rz * S.q[0] - rx * S.q[2]);
            v2 += fv * (rx * S.q[1] - ry * S.q[0]);
            if (P.want_psi) {
                const T fp = ec * ir;
                p0 += fp * S.q[0];
                p1 += fp * S.q[1];
                p2 += fp * S.q[2];
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
        v2 += __shfl_xor_sync(0xffffffffu, v2, o);
        if (P.want_psi) {
            p0 += __shfl_xor_sync(0xffffffffu, p0, o);
            p1 += __shfl_xor_sync(0xffffffffu, p1, o);
            p2 += __shfl_xor_sync(0xffffffffu, p2, o);
        }
    }
    if (lane == 0) {
        const T pref = (T)P.pref;
        vsr[3 * j + 0] = pref * v0;
        vsr[3 * j + 1] = pref * v1;
        vsr[3 * j + 2] = pref * v2;
        if (P.want_psi) {
            psr[3 * j + 0] = pref * p0;
            psr[3 * j + 1] = pref * p1;
            psr[3 * j + 2] = pref * p2;
        }
    }
}

template <typename T>
cudaError_t launch_short(const ShortP& P, const Work& w, cudaStream_t s)
{
    if (P.N <= 0) return cudaSuccess;
    const int tb = 256;  // 8 targets per block, one warp each
    const long long threads = 32LL * P.N;
    k_short<T><<<(unsigned)((threads + tb - 1) / tb), tb, 0, s>>>(P, (const SrTgt<T>*)w.tgt, w.prev, w.cell_cnt,
                                                   (const SrRec<T>*)w.sr_sorted, (T*)w.vsr, (T*)w.psr);
    return cudaGetLastError();
}

template cudaError_t launch_short<float>(const ShortP&, const Work&, cudaStream_t);
template cudaError_t launch_short<double>(const ShortP&, const Work&, cudaStream_t);

// The float32 complementary error function as the short-range kernels take
// it (erfc_e with e = expf(-x^2)), one thread per argument.
__global__ void k_erfc_f32(int n, const float* __restrict__ x, float* __restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const float xi = x[i];
        out[i] = erfc_e<float>(xi, expf(-xi * xi));
    }
}

}  // namespace bsw

extern "C" int bs_erfc_f32(int n, const float* x, float* out, void* stream)
{
    if (n < 0 || (n > 0 && (!x || !out))) {
        bsw::set_last_error("bs_erfc_f32: bad arguments");
        return BS_ERR_ARG;
    }
    if (n == 0) return BS_OK;
    bsw::k_erfc_f32<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(n, x, out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        bsw::set_last_error(cudaGetErrorString(e));
        return BS_ERR_CUDA;
    }
    return BS_OK;
}
