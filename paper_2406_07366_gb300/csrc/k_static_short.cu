// Short-range velocity sum that allocates nothing: the cell list it needs
// lives in one fixed scratch array compiled into the library.
//
// Some callers cannot call cudaMalloc: an application that hands out all
// device memory through its own allocator or a fixed memory budget, or a
// latency-critical loop that must not hit the implicit device
// synchronisation a cudaMalloc / cudaFree can cause.  They can still use the
// short-range part of the method through bs_short_range_static: they pass
// their inputs and outputs, and the binning scratch comes from g_scratch.
//
// The arithmetic is that of the library's short-range kernel in float64
// (Sec. 3.2, Eq. velocity_shortrange): minimum image, cut-off r_c, cells of
// edge >= r_c / m sorted with x fastest so that a row of 2m+1 cells is one
// contiguous range.
#include <math.h>
#include <stddef.h>


#include "bs_internal.cuh"

namespace {

constexpr int kStaticMaxSources = 1 << 17;  // 131072 sources
constexpr int kStaticMaxCells = 1 << 16;    // 65536 cells

struct __align__(16) StRec {
    double o[3];  // offset from the cell origin
    double q[3];  // charge
    int cx;       // x-cell index
    int seg;      // segment id, compared with the targets' omitted ids
    int pad[2];
};

struct StScratch {
    StRec rec[kStaticMaxSources];     // 8 MiB: sources sorted by cell
    int key[kStaticMaxSources];       // cell of each source, input order
    int start[kStaticMaxCells + 1];   // counts, then exclusive offsets
    int cursor[kStaticMaxCells];      // scatter positions
};

// The scratch area: about 9 MiB on every device that loads the library,
// held until the process exits.
static __device__ __align__(256) unsigned char g_scratch[sizeof(StScratch)];

struct StP {
    double L[3];
    int nc[3];
    double hc[3];
    int m;
    double rc2, alpha, pref;
    int nsrc, ntgt;
};

__device__ __forceinline__ double st_wrap(double x, double L)
{
    if (!isfinite(x)) return 0.0;
    double y = x - L * floor(x / L);
    if (y >= L) y -= L;
    if (y < 0.0) y = 0.0;
    return y;
}

__device__ __forceinline__ int st_cell(double xw, double h, int n)
{
    int k = (int)(xw / h);
    return k < 0 ? 0 : (k >= n ? n - 1 : k);
}

__device__ __forceinline__ int st_imod(int a, int n)
{
    int r = a % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ int st_cdiff(int a, int b, int n)
{
    int d = a - b;
    if (d >= (n + 1) / 2) d -= n;
    if (d < -(n / 2)) d += n;
    return d;
}

__global__ void k_st_count(StP P, const double* __restrict__ pos, StScratch* __restrict__ S)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.nsrc) return;
    int c[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) c[d] = st_cell(st_wrap(pos[3 * i + d], P.L[d]), P.hc[d], P.nc[d]);
    const int key = c[0] + P.nc[0] * (c[1] + P.nc[1] * c[2]);
    S->key[i] = key;
    atomicAdd(&S->start[key], 1);
}

// Exclusive scan of start[0..n] in one block (n <= kStaticMaxCells); also
// copies the offsets to cursor.
__global__ void k_st_scan(int n, StScratch* __restrict__ S)
{
    __shared__ int warp_tot[32];
    const int per = (n + 1 + blockDim.x - 1) / blockDim.x;
    const int b = threadIdx.x * per;
    int s = 0;
    for (int k = 0; k < per; ++k)
        if (b + k <= n) s += (b + k < n) ? S->start[b + k] : 0;
    // block exclusive scan of s
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int v = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int w = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    int run = v - s + (wid > 0 ? warp_tot[wid - 1] : 0);
    for (int k = 0; k < per; ++k) {
        const int i = b + k;
        if (i > n) break;
        const int cnt = (i < n) ? S->start[i] : 0;
        S->start[i] = run;
        if (i < n) S->cursor[i] = run;
        run += cnt;
    }
}

__global__ void k_st_scatter(StP P, const double* __restrict__ pos, const double* __restrict__ q,
                             const int* __restrict__ seg, StScratch* __restrict__ S)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.nsrc) return;
    StRec R;
    int c0 = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double xw = st_wrap(pos[3 * i + d], P.L[d]);
        const int c = st_cell(xw, P.hc[d], P.nc[d]);
        if (d == 0) c0 = c;
        R.o[d] = xw - c * P.hc[d];
        R.q[d] = q[3 * i + d];
    }
    R.cx = c0;
    R.seg = seg[i];
    R.pad[0] = R.pad[1] = 0;
    const int p = atomicAdd(&S->cursor[S->key[i]], 1);
    S->rec[p] = R;
}

__global__ void k_st_pairs(StP P, const double* __restrict__ tpos, const int* __restrict__ excl,
                           const StScratch* __restrict__ S, double* __restrict__ vel)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.ntgt) return;
    const int nc0 = P.nc[0], nc1 = P.nc[1], nc2 = P.nc[2];
    double to[3];
    int tc[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double xw = st_wrap(tpos[3 * j + d], P.L[d]);
        tc[d] = st_cell(xw, P.hc[d], P.nc[d]);
        to[d] = xw - tc[d] * P.hc[d];
    }
    const int e0 = excl[2 * j], e1 = excl[2 * j + 1];
    const int m = P.m;
    const bool fullx = (2 * m + 1 >= nc0), fully = (2 * m + 1 >= nc1), fullz = (2 * m + 1 >= nc2);
    const int ny = fully ? nc1 : 2 * m + 1, nz = fullz ? nc2 : 2 * m + 1;
    const double two_over_sqrtpi = 1.12837916709551257390;
    double v0 = 0, v1 = 0, v2 = 0;
    for (int iz = 0; iz < nz; ++iz) {
        const int zc = fullz ? iz : st_imod(tc[2] - m + iz, nc2);
        const double dzc = st_cdiff(zc, tc[2], nc2) * P.hc[2];
        for (int iy = 0; iy < ny; ++iy) {
            const int yc = fully ? iy : st_imod(tc[1] - m + iy, nc1);
            const double dyc = st_cdiff(yc, tc[1], nc1) * P.hc[1];
            const int row = (zc * nc1 + yc) * nc0;
            int xa[2], xb[2], nr;
            if (fullx) {
                xa[0] = 0; xb[0] = nc0 - 1; nr = 1;
            } else {
                const int lo = tc[0] - m, hi = tc[0] + m;
                if (lo < 0) {
                    xa[0] = lo + nc0; xb[0] = nc0 - 1; xa[1] = 0; xb[1] = hi; nr = 2;
                } else if (hi >= nc0) {
                    xa[0] = lo; xb[0] = nc0 - 1; xa[1] = 0; xb[1] = hi - nc0; nr = 2;
                } else {
                    xa[0] = lo; xb[0] = hi; nr = 1;
                }
            }
            for (int r = 0; r < nr; ++r) {
                const int s0 = S->start[row + xa[r]], s1 = S->start[row + xb[r] + 1];
                for (int k = s0; k < s1; ++k) {
                    const StRec& R = S->rec[k];
                    if (R.seg == e0 || R.seg == e1) continue;
                    double rx = st_cdiff(R.cx, tc[0], nc0) * P.hc[0] + (R.o[0] - to[0]);
                    double ry = dyc + (R.o[1] - to[1]);
                    double rz = dzc + (R.o[2] - to[2]);
                    rx = rx > 0.5 * P.L[0] ? rx - P.L[0] : (rx < -0.5 * P.L[0] ? rx + P.L[0] : rx);
                    ry = ry > 0.5 * P.L[1] ? ry - P.L[1] : (ry < -0.5 * P.L[1] ? ry + P.L[1] : ry);
                    rz = rz > 0.5 * P.L[2] ? rz - P.L[2] : (rz < -0.5 * P.L[2] ? rz + P.L[2] : rz);
                    const double r2 = rx * rx + ry * ry + rz * rz;
                    if (r2 >= P.rc2 || r2 == 0.0) continue;
                    const double rr = sqrt(r2);
                    const double x = P.alpha * rr;
                    const double g = erfc(x) + two_over_sqrtpi * x * exp(-x * x);
                    const double fv = g / (rr * r2);
                    v0 += fv * (ry * R.q[2] - rz * R.q[1]);
                    v1 += fv * (rz * R.q[0] - rx * R.q[2]);
                    v2 += fv * (rx * R.q[1] - ry * R.q[0]);
                }
            }
        }
    }
    vel[3 * j + 0] = P.pref * v0;
    vel[3 * j + 1] = P.pref * v1;
    vel[3 * j + 2] = P.pref * v2;
}

// Device address of g_scratch, looked up once per device (with that device
// current) on the first call made on it.
int st_fail(int code, const char* msg)
{
    bsw::set_last_error(msg);
    return code;
}

}  // namespace

extern "C" int bs_short_range_static(const double L[3], double kappa, double alpha, double rc, int nsrc,
                                     const double* src_pos, const double* src_q, const int* src_seg, int ntgt,
                                     const double* tgt_pos, const int* tgt_omit, double* vel, void* stream)
{
    if (!L) return st_fail(BS_ERR_ARG, "null L");
    const double Lmin = fmin(L[0], fmin(L[1], L[2]));
    for (int d = 0; d < 3; ++d)
        if (!(L[d] > 0) || !isfinite(L[d])) return st_fail(BS_ERR_ARG, "L must be positive and finite");
    if (!(alpha > 0) || !(rc > 0) || !isfinite(alpha) || !isfinite(rc) || !isfinite(kappa))
        return st_fail(BS_ERR_ARG, "alpha and rc must be positive and finite");
    if (rc > 0.5 * Lmin * (1 + 1e-12)) return st_fail(BS_ERR_RC_GT_HALF_L, "rc exceeds min(L)/2");
    if (nsrc < 0 || ntgt < 0) return st_fail(BS_ERR_ARG, "negative count");
    if (nsrc > kStaticMaxSources)
        return st_fail(BS_ERR_ARG, "bs_short_range_static: more than 131072 sources (static scratch limit)");
    if ((nsrc > 0 && (!src_pos || !src_q || !src_seg)) || (ntgt > 0 && (!tgt_pos || !tgt_omit || !vel)))
        return st_fail(BS_ERR_ARG, "null array");
    if (ntgt == 0) return BS_OK;

    StP P;
    P.m = 3;
    for (;;) {
        // the cell counts are formed in double and clamped before the int
        // conversion, so that a strongly anisotropic box (one axis many
        // times r_c) cannot overflow them
        double tot = 1.0;
        for (int d = 0; d < 3; ++d) {
            double nd = floor(L[d] * P.m / rc);
            nd = nd < 1.0 ? 1.0 : (nd > (double)kStaticMaxCells + 1.0 ? (double)kStaticMaxCells + 1.0 : nd);
            const int n = (int)nd;
            P.nc[d] = n;
            P.hc[d] = L[d] / n;
            P.L[d] = L[d];
            tot *= nd;
        }
        if (tot <= (double)kStaticMaxCells) break;
        if (P.m == 1)
            return st_fail(BS_ERR_ARG, "bs_short_range_static: rc too small for the 65536-cell static scratch");
        P.m -= 1;
    }
    const int ncells = P.nc[0] * P.nc[1] * P.nc[2];
    P.rc2 = rc * rc;
    P.alpha = alpha;
    P.pref = kappa / (4.0 * bsw::kPi);
    P.nsrc = nsrc;
    P.ntgt = ntgt;

    // The scratch address is looked up on every call, with the caller's
    // device current: in host code g_scratch names a host-side stand-in,
    // and the device copy can move when the context is torn down and made
    // again (cudaDeviceReset, a released primary context).  The lookup
    // allocates nothing.
    void* base = nullptr;
    {
        cudaError_t e = cudaGetSymbolAddress(&base, g_scratch);
        if (e != cudaSuccess || !base) return st_fail(BS_ERR_CUDA, cudaGetErrorString(e));
    }
    StScratch* S = (StScratch*)base;
    int* start = (int*)((char*)base + offsetof(StScratch, start));
    cudaStream_t s = (cudaStream_t)stream;
    // counts start at zero on every call (the array keeps the last call's contents)
    cudaError_t e = cudaMemsetAsync(start, 0, sizeof(int) * (size_t)(ncells + 1), s);
    if (e != cudaSuccess) return st_fail(BS_ERR_CUDA, cudaGetErrorString(e));
    const int tb = 256;
    if (nsrc > 0) k_st_count<<<(nsrc + tb - 1) / tb, tb, 0, s>>>(P, src_pos, S);
    k_st_scan<<<1, 1024, 0, s>>>(ncells, S);
    if (nsrc > 0) k_st_scatter<<<(nsrc + tb - 1) / tb, tb, 0, s>>>(P, src_pos, src_q, src_seg, S);
    k_st_pairs<<<(ntgt + 127) / 128, 128, 0, s>>>(P, tgt_pos, tgt_omit, S, vel);
    e = cudaGetLastError();
    if (e != cudaSuccess) return st_fail(BS_ERR_CUDA, cudaGetErrorString(e));
    return BS_OK;
}
