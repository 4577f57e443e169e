// Short-range velocity and streamfunction (Sec. 3.2, Eqs.
// velocity_shortrange and streamfunction_shortrange) at every node:
//   v^(n)(s_j)   = kappa/4pi sum_{q not in C_0(j), |r| < r_c} g^(n)(alpha r) (r x q) / r^3,
//   psi^(n)(s_j) = kappa/4pi sum_{same} erfc(alpha r) q / r,
// r the minimum image of (source - node), g^(n)(x) = erfc(x) + 2x/sqrt(pi) e^{-x^2}.
//
// Sources are binned in cells of edge >= r_c/m (m = 3 in Sec. 5.3) and
// sorted by cell with x fastest, so the 2m+1 cells of a row along x form one
// contiguous range of the sorted array (two when the row wraps).  One thread
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

template <typename T>
__device__ __forceinline__ T erfc_t(T x) { return erfc(x); }

template <typename T>
__global__ void __launch_bounds__(128) k_short(ShortP P, const SrTgt<T>* __restrict__ tgt, const int* __restrict__ prev,
                                               const int* __restrict__ start, const SrRec<T>* __restrict__ src,
                                               T* __restrict__ vsr, T* __restrict__ psr)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.N) return;
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

    T v0 = 0, v1 = 0, v2 = 0, p0 = 0, p1 = 0, p2 = 0;
    for (int iz = 0; iz < nz; ++iz) {
        const int zc = fullz ? iz : imod(cz - m + iz, nc2);
        const T dzc = (T)cdiff(zc, cz, nc2) * h2;
        for (int iy = 0; iy < ny; ++iy) {
            const int yc = fully ? iy : imod(cy - m + iy, nc1);
            const T dyc = (T)cdiff(yc, cy, nc1) * h1;
            const int row = (zc * nc1 + yc) * nc0;
            // one or two contiguous x-ranges [xa0, xb0], [xa1, xb1]
            int xa0, xb0, xa1 = 0, xb1 = -1;
            if (fullx) {
                xa0 = 0; xb0 = nc0 - 1;
            } else {
                const int lo = cx - m, hi = cx + m;
                if (lo < 0) {
                    xa0 = lo + nc0; xb0 = nc0 - 1; xa1 = 0; xb1 = hi;
                } else if (hi >= nc0) {
                    xa0 = lo; xb0 = nc0 - 1; xa1 = 0; xb1 = hi - nc0;
                } else {
                    xa0 = lo; xb0 = hi;
                }
            }
            const int nr = (xb1 >= xa1) ? 2 : 1;
            for (int r = 0; r < nr; ++r) {
                const int s0 = start[row + (r ? xa1 : xa0)], s1 = start[row + (r ? xb1 : xb0) + 1];
                for (int k = s0; k < s1; ++k) {
                    const SrRec<T> S = src[k];
                    if (S.seg == j || S.seg == jp) continue;  // C_0 of the node (Eq. BS_on_vortex)
                    T rx = (T)cdiff(S.cx, cx, nc0) * h0 + (S.o[0] - t.o[0]);
                    T ry = dyc + (S.o[1] - t.o[1]);
                    T rz = dzc + (S.o[2] - t.o[2]);
                    // exact minimum image when a cell difference sits at n/2
                    rx = rx > (T)0.5 * L0 ? rx - L0 : (rx < (T)-0.5 * L0 ? rx + L0 : rx);
                    ry = ry > (T)0.5 * L1 ? ry - L1 : (ry < (T)-0.5 * L1 ? ry + L1 : ry);
                    rz = rz > (T)0.5 * L2 ? rz - L2 : (rz < (T)-0.5 * L2 ? rz + L2 : rz);
                    const T r2 = rx * rx + ry * ry + rz * rz;
                    if (r2 >= rc2 || r2 == (T)0) continue;
                    const T rr = sqrt(r2);
                    const T x = alpha * rr;
                    const T ec = erfc_t(x);
                    const T g = ec + two_over_sqrtpi * x * exp(-x * x);
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
        }
    }
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

template <typename T>
cudaError_t launch_short(const ShortP& P, const Work& w, cudaStream_t s)
{
    if (P.N <= 0) return cudaSuccess;
    const int tb = 128;
    k_short<T><<<(P.N + tb - 1) / tb, tb, 0, s>>>(P, (const SrTgt<T>*)w.tgt, w.prev, w.cell_cnt,
                                                   (const SrRec<T>*)w.sr_sorted, (T*)w.vsr, (T*)w.psr);
    return cudaGetLastError();
}

template cudaError_t launch_short<float>(const ShortP&, const Work&, cudaStream_t);
template cudaError_t launch_short<double>(const ShortP&, const Work&, cudaStream_t);

}  // namespace bsw
