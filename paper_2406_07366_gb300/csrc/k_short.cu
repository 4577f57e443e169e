// Short-range velocity and streamfunction (Sec. 3.2, Eqs.
// velocity_shortrange and streamfunction_shortrange) at every node:
//   v^(n)(s_j)   = kappa/4pi sum_{q not in C_0(j), |r| < r_c} g^(n)(alpha r) (r x q) / r^3,
//   psi^(n)(s_j) = kappa/4pi sum_{same} erfc(alpha r) q / r,
// r the minimum image of (source - node), g^(n)(x) = erfc(x) + 2x/sqrt(pi) e^{-x^2}.
//
// Sources are binned in cells of edge >= r_c/m (Sec. 5.3 uses m = 3) and
// sorted by cell with x fastest, so a run of cells along x is one contiguous
// range of the sorted array (two when it wraps around the box).
//
// k_short_tile (m <= kShortTileMaxM): the nodes are binned by blocks of
// m x m x m cells (an r_c cube).  A CTA per block stages the sources of the
// cells within r_c of the block (3m cells per axis) in shared memory, as
// positions relative to the block centre, then every warp takes a node of the
// block and sweeps the staged sources 32 at a time: the lanes test their
// candidates (cheap), the ones inside r_c are queued per warp, and the pair
// terms are evaluated 32 at a time by full warps.  Each lane sums its pair
// terms in T; the node's total is kept in float64.
//
// k_short (larger m): one warp per node walks the (2m+1)^2 neighbour rows.
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
    const float t = __frcp_rn(1.0f + 0.5f * x);  // the correctly rounded 1 / (1 + x/2)
    float v = c[10];
#pragma unroll
    for (int k = 9; k >= 0; --k) v = fmaf(v, t, c[k]);
    return v;
}

// 1 / sqrt(x) and exp(x) of the pair terms: float32 through the hardware
// approximations (reciprocal square root; exp as 2^(x log2 e), whose scaled
// argument costs about |x| 2^-24 relative, below 1e-6 for the |x| <= beta^2
// the short range meets), float64 exact.  Measured on the 4e6-node tangle:
// the short range 12.99 -> 11.89 ms with the accuracy against the converged
// sum unchanged (rms 3.148e-6 / 3.150e-6).
template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }
template <typename T>
__device__ __forceinline__ T exp_t(T x);
template <>
__device__ __forceinline__ float exp_t<float>(float x) { return __expf(x); }
template <>
__device__ __forceinline__ double exp_t<double>(double x) { return exp(x); }

// erfc(x) given e = exp(-x^2): float32 through the fit above, float64 exact.
template <typename T>
__device__ __forceinline__ T erfc_e(T x, T e);
template <>
__device__ __forceinline__ float erfc_e<float>(float x, float e) { return e * erfcx_f(x); }
template <>
__device__ __forceinline__ double erfc_e<double>(double x, double) { return erfc(x); }

// Adds the pair term of source (position rel, charge q) seen from the node at
// distance vector r (source - node), |r| = sqrt(r2).
template <typename T>
__device__ __forceinline__ void st_pair(T rx, T ry, T rz, T r2, const T* q, T alpha, int want_psi, T& v0, T& v1,
                                        T& v2, T& p0, T& p1, T& p2)
{
    const T two_over_sqrtpi = (T)1.12837916709551257390;
    const T ir = rsqrt_t(r2);
    const T rr = r2 * ir;
    const T x = alpha * rr;
    const T e = exp_t(-x * x);
    const T ec = erfc_e(x, e);
    const T g = ec + two_over_sqrtpi * x * e;
    const T fv = g * ir * ir * ir;
    v0 += fv * (ry * q[2] - rz * q[1]);
    v1 += fv * (rz * q[0] - rx * q[2]);
    v2 += fv * (rx * q[1] - ry * q[0]);
    if (want_psi) {
        const T fp = ec * ir;
        p0 += fp * q[0];
        p1 += fp * q[1];
        p2 += fp * q[2];
    }
}

constexpr int kShortWarps = 8;  // warps per CTA of the warp-per-node kernel

// One warp per target node.  The lanes first list the source ranges of the
// (2m+1)^2 neighbour rows (32 rows at a time; a row wrapping around the box
// gives two ranges; rows and row ends beyond r_c are cut), prefix-sum their
// lengths, then stride through the flattened candidate list, so every lane
// has work however short the rows are.  The non-empty rows go into a
// per-warp table in shared memory; a lane finds the row of its candidate from
// one OR-reduction per 32 candidates (which rows start in the window) and a
// population count, and reads the row from the table.  The per-lane partial
// sums are reduced at the end.
template <typename T>
__device__ __forceinline__ void k_short_body(const ShortP& P, const SrTgt<T>* __restrict__ tgt,
                                             const int* __restrict__ prev, const int* __restrict__ start,
                                             const SrRec<T>* __restrict__ src, double* __restrict__ vsr,
                                             double* __restrict__ psr, int bid)
{
    const int lane = threadIdx.x & 31;
    const int wslot = threadIdx.x >> 5;  // the warp's slot in the CTA's row tables
    // per warp: a round's non-empty rows (first source of each run, run
    // lengths, first candidate) and their y, z cell offsets
    __shared__ int4 s_row[kShortWarps][32];
    __shared__ int4 s_ofs[kShortWarps][32];   // x-cell offsets of the two runs, y and z cell offsets
    __shared__ T s_dh[kShortWarps][32][2];    // y and z cell offsets times the cell edges
    const int j = (int)((bid * (size_t)blockDim.x + threadIdx.x) >> 5);
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
    // offsets are from the cell centre; the node's position in its cell
    const T ox = t.o[0] + (T)0.5 * h0, oy = t.o[1] + (T)0.5 * h1, oz = t.o[2] + (T)0.5 * h2;
    // Candidates lie within m cells of the node's cell along each axis, so
    // |r| < (m + 1) h; with at least 2 (m + 1) cells per axis that is below
    // L/2 and the nearest cell image is already the minimum image: no wrap.
    const bool wrap = nc0 < 2 * (m + 1) || nc1 < 2 * (m + 1) || nc2 < 2 * (m + 1);

    T v0 = 0, v1 = 0, v2 = 0, p0 = 0, p1 = 0, p2 = 0;
    for (int rb = 0; rb < nrows; rb += 32) {
        // this lane's row
        const int r = rb + lane;
        int s0 = 0, n0 = 0, s1 = 0, n1r = 0, dyi = 0, dzi = 0;
        int xo0 = 0, xo1 = 0;  // x-cell offset from the node's cell: cell index + xo (per run)
        if (r < nrows) {
            const int iz = r / ny, iy = r - iz * ny;
            const int zc = fullz ? iz : imod(cz - m + iz, nc2);
            const int yc = fully ? iy : imod(cy - m + iy, nc1);
            dzi = cdiff(zc, cz, nc2);
            dyi = cdiff(yc, cy, nc1);
            // gaps between the node and the row's y and z slabs
            T gy = (T)0, gz = (T)0;
            if (!fully) gy = dyi > 0 ? dyi * h1 - oy : (dyi < 0 ? oy - (dyi + 1) * h1 : (T)0);
            if (!fullz) gz = dzi > 0 ? dzi * h2 - oz : (dzi < 0 ? oz - (dzi + 1) * h2 : (T)0);
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
                    int lo = (int)floor((ox - ext) * ih0), hi = (int)floor((ox + ext) * ih0);
                    lo = cx + (lo < -m ? -m : lo);
                    hi = cx + (hi > m ? m : hi);
                    if (lo < 0) {
                        xa0 = lo + nc0; xb0 = nc0 - 1; xa1 = 0; xb1 = hi;
                        xo0 = -nc0 - cx; xo1 = -cx;
                    } else if (hi >= nc0) {
                        xa0 = lo; xb0 = nc0 - 1; xa1 = 0; xb1 = hi - nc0;
                        xo0 = -cx; xo1 = nc0 - cx;
                    } else {
                        xa0 = lo; xb0 = hi;
                        xo0 = -cx;
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
        const int nr = n0 + n1r;
        int inc = nr;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += u;
        }
        const int total = __shfl_sync(0xffffffffu, inc, 31);
        const int ex = inc - nr;  // the row's first candidate
        // the non-empty rows in lane order, compacted into this warp's table
        const unsigned nonempty = __ballot_sync(0xffffffffu, nr > 0);
        if (nr > 0) {
            const int ci = __popc(nonempty & ((1u << lane) - 1u));
            s_row[wslot][ci] = make_int4(s0, n0, s1, ex);
            s_ofs[wslot][ci] = make_int4(xo0, xo1, dyi, dzi);
            s_dh[wslot][ci][0] = (T)dyi * h1;
            s_dh[wslot][ci][1] = (T)dzi * h2;
        }
        __syncwarp();
        // Candidate c belongs to the last non-empty row starting at or before
        // it.  Per window of 32 candidates, bit b of M marks a row starting at
        // cb + b; a lane's row is the one holding the window's first candidate
        // minus one (jr) plus the starts up to its own candidate.
        const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
        int jr = -1;
        for (int cb = 0; cb < total; cb += 32) {  // warp-uniform trip count
            const unsigned bit = (nr > 0 && ex >= cb && ex < cb + 32) ? (1u << (ex - cb)) : 0u;
            const unsigned M = __reduce_or_sync(0xffffffffu, bit);
            const int c = cb + lane;
            const int own = jr + __popc(M & upto);
            jr += __popc(M);
            if (c >= total) continue;
            const int4 rw = s_row[wslot][own];
            const int local = c - rw.w;
            const bool first = local < rw.y;
            const int k = first ? rw.x + local : rw.z + (local - rw.y);
            const SrRec<T> S = src[k];
            if (S.seg == j || S.seg == jp) continue;  // C_0 of the node (Eq. BS_on_vortex)
            T rx, ry, rz;
            if (!wrap) {
                const int4 of = s_ofs[wslot][own];
                rx = (T)(S.cx + (first ? of.x : of.y)) * h0 + (S.o[0] - t.o[0]);
                ry = s_dh[wslot][own][0] + (S.o[1] - t.o[1]);
                rz = s_dh[wslot][own][1] + (S.o[2] - t.o[2]);
            } else {
                const int4 of = s_ofs[wslot][own];
                rx = (T)cdiff(S.cx, cx, nc0) * h0 + (S.o[0] - t.o[0]);
                ry = (T)of.z * h1 + (S.o[1] - t.o[1]);
                rz = (T)of.w * h2 + (S.o[2] - t.o[2]);
                // exact minimum image when a cell difference sits at n/2
                rx = rx > (T)0.5 * L0 ? rx - L0 : (rx < (T)-0.5 * L0 ? rx + L0 : rx);
                ry = ry > (T)0.5 * L1 ? ry - L1 : (ry < (T)-0.5 * L1 ? ry + L1 : ry);
                rz = rz > (T)0.5 * L2 ? rz - L2 : (rz < (T)-0.5 * L2 ? rz + L2 : rz);
            }
            const T r2 = rx * rx + ry * ry + rz * rz;
            if (r2 >= rc2 || r2 == (T)0) continue;
            const T ir = rsqrt_t(r2);
            const T rr = r2 * ir;
            const T x = alpha * rr;
            const T e = exp_t(-x * x);
            const T ec = erfc_e(x, e);
            const T g = ec + two_over_sqrtpi * x * e;
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
        __syncwarp();  // the table is rewritten by the next round of rows
    }
    // lane sums reduced in T (a float64 tree costs about 1.5 ms on the
    // 4e6-node tangle: float64 runs at 1/64 of the float32 rate here), the
    // node's total kept in float64
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
        vsr[3 * j + 0] = P.pref * (double)v0;
        vsr[3 * j + 1] = P.pref * (double)v1;
        vsr[3 * j + 2] = P.pref * (double)v2;
        if (P.want_psi) {
            psr[3 * j + 0] = P.pref * (double)p0;
            psr[3 * j + 1] = P.pref * (double)p1;
            psr[3 * j + 2] = P.pref * (double)p2;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_short(ShortP P, const SrTgt<T>* __restrict__ tgt, const int* __restrict__ prev,
                                               const int* __restrict__ start, const SrRec<T>* __restrict__ src,
                                               double* __restrict__ vsr, double* __restrict__ psr)
{
    k_short_body<T>(P, tgt, prev, start, src, vsr, psr, blockIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(256) k_short_b(const ShortD<T>* __restrict__ d, const int* __restrict__ bs, int n)
{
    int bid, nb;
    const ShortD<T>& a = d[batch_member(bs, n, bid, nb)];
    k_short_body<T>(a.P, a.tgt, a.prev, a.start, a.src, a.vsr, a.psr, bid);
}

// ---------------------------------------------------------------------------
// Nodes binned by target block (m x m x m cells).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_tgt_key(ShortP P, const SrTgt<T>* __restrict__ tgt, int* __restrict__ key, int* __restrict__ cnt)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.N) return;
    const int cell = tgt[j].cell;
    const int cx = cell % P.nc[0], cy = (cell / P.nc[0]) % P.nc[1], cz = cell / (P.nc[0] * P.nc[1]);
    const int b = cx / P.m + P.nb[0] * (cy / P.m + P.nb[1] * (cz / P.m));
    key[j] = b;
    atomicAdd(&cnt[b], 1);
}

__global__ void k_tgt_scatter(int N, const int* __restrict__ key, int* __restrict__ cur, int* __restrict__ idx)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < N) idx[atomicAdd(&cur[key[j]], 1)] = j;
}

// ---------------------------------------------------------------------------
// Tiled short range (see the header).
// ---------------------------------------------------------------------------
template <typename T> struct __align__(16) StPos {
    T x, y, z;
    int seg;
};
template <typename T> struct __align__(16) StChg {
    T q[3];
    T pad;
};

constexpr int kStWarps = 4;
constexpr int kStRanges = 2 * (3 * kShortTileMaxM) * (3 * kShortTileMaxM);
template <typename T>
constexpr int st_chunk()
{
    return sizeof(T) == 4 ? 1024 : 512;  // staged sources (32 KB of shared memory)
}

// Minimum image along an axis the staged region wraps onto itself.
template <typename T>
__device__ __forceinline__ T st_wrap(T r, T L)
{
    return r > (T)0.5 * L ? r - L : (r < (T)-0.5 * L ? r + L : r);
}

template <typename T>
__global__ void __launch_bounds__(kStWarps * 32) k_short_tile(ShortP P, const SrTgt<T>* __restrict__ tgt,
                                                              const int* __restrict__ prev,
                                                              const int* __restrict__ start,
                                                              const SrRec<T>* __restrict__ src,
                                                              const int* __restrict__ tb_start,
                                                              const int* __restrict__ tb_idx,
                                                              double* __restrict__ vsr, double* __restrict__ psr)
{
    constexpr int CH = st_chunk<T>();
    constexpr int kRows = kStRanges / 2;
    __shared__ StPos<T> spos[CH];
    __shared__ StChg<T> schg[CH];
    // per staged row: the sorted-array start of its two x-runs, their staged
    // starts (prefix), and the staged start of every cell of the row
    __shared__ int r_beg[kStRanges], r_pre[kStRanges + 1];
    __shared__ int c_beg[kRows * (3 * kShortTileMaxM + 1)];
    __shared__ int qbuf[kStWarps][64];
    const int t0 = tb_start[blockIdx.x], t1 = tb_start[blockIdx.x + 1];
    if (t0 == t1) return;  // no node in this block (uniform over the CTA)
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int m = P.m;
    const int nc0 = P.nc[0], nc1 = P.nc[1], nc2 = P.nc[2];
    const int b = blockIdx.x;
    const int bxi = b % P.nb[0], byi = (b / P.nb[0]) % P.nb[1], bzi = b / (P.nb[0] * P.nb[1]);
    const int ox = bxi * m, oy = byi * m, oz = bzi * m;  // first cell of the block per axis
    const int mbx = min(m, nc0 - ox), mby = min(m, nc1 - oy), mbz = min(m, nc2 - oz);
    // staged cells per axis: [o - m, o + mb + m) (mod n), or every cell once
    // when that would wrap onto itself (then pairs take the minimum image)
    const bool fx = 2 * m + mbx >= nc0, fy = 2 * m + mby >= nc1, fz = 2 * m + mbz >= nc2;
    const int cntx = fx ? nc0 : 2 * m + mbx, cnty = fy ? nc1 : 2 * m + mby, cntz = fz ? nc2 : 2 * m + mbz;
    const int fstx = fx ? 0 : ox - m, fsty = fy ? 0 : oy - m, fstz = fz ? 0 : oz - m;
    const T h0 = (T)P.hc[0], h1 = (T)P.hc[1], h2 = (T)P.hc[2];
    const T L0 = (T)P.L[0], L1 = (T)P.L[1], L2 = (T)P.L[2];
    // block centre (cells from the block's first cell)
    const T cx0 = (T)0.5 * (T)mbx, cy0 = (T)0.5 * (T)mby, cz0 = (T)0.5 * (T)mbz;
    // staged cell k of a row is x cell fstx + k (mod nc0); the row's first run
    // covers k < na, its wrapped remainder the rest
    const int xa0 = fx ? 0 : imod(fstx, nc0);
    const int na = fx ? nc0 : min(cntx, nc0 - xa0);
    const int nrows = cnty * cntz;
    const int nr = 2 * nrows;
    for (int r = tid; r < nrows; r += blockDim.x) {
        const int iy = r % cnty, iz = r / cnty;
        const int cy = imod(fsty + iy, nc1), cz = imod(fstz + iz, nc2);
        const int rowb = (cz * nc1 + cy) * nc0;
        r_beg[2 * r] = start[rowb + xa0];
        r_pre[2 * r + 1] = start[rowb + xa0 + na] - r_beg[2 * r];
        if (na < cntx) {
            r_beg[2 * r + 1] = start[rowb];
            r_pre[2 * r + 2] = start[rowb + cntx - na] - r_beg[2 * r + 1];
        } else {
            r_beg[2 * r + 1] = 0;
            r_pre[2 * r + 2] = 0;
        }
    }
    __syncthreads();
    if (wid == 0) {  // run lengths -> exclusive prefix r_pre[0..nr]
        int carry = 0;
        for (int k0 = 0; k0 < nr; k0 += 32) {
            const int k = k0 + lane;
            const int v = k < nr ? r_pre[k + 1] : 0;
            int inc = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += u;
            }
            if (k < nr) r_pre[k + 1] = carry + inc;
            carry += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (lane == 0) r_pre[0] = 0;
    }
    __syncthreads();
    // staged start of every cell of every row (and the row's end)
    const int cpr = cntx + 1;
    for (int i = tid; i < nrows * cpr; i += blockDim.x) {
        const int r = i / cpr, k = i - r * cpr;
        int v;
        if (k == cntx) {
            v = r_pre[2 * r + 2];
        } else {
            const int iy = r % cnty, iz = r / cnty;
            const int cy = imod(fsty + iy, nc1), cz = imod(fstz + iz, nc2);
            const int rowb = (cz * nc1 + cy) * nc0;
            v = k < na ? r_pre[2 * r] + (start[rowb + xa0 + k] - r_beg[2 * r])
                       : r_pre[2 * r + 1] + (start[rowb + k - na] - r_beg[2 * r + 1]);
        }
        c_beg[i] = v;
    }
    const int total = r_pre[nr];
    const T rc2 = (T)P.rc2;
    const T rcm2 = rc2 * (T)1.0001;  // row cuts are conservative under rounding; the pair test is exact
    const T alpha = (T)P.alpha;
    const unsigned lt = (1u << lane) - 1u;
    int* q = qbuf[wid];
    for (int c0 = 0; c0 < total; c0 += CH) {
        const int nch = min(CH, total - c0);
        __syncthreads();  // the previous chunk's sources are no longer read (and c_beg is written)
        // stage: a warp per run, sources relative to the block centre
        for (int r = wid; r < nr; r += kStWarps) {
            const int a = max(r_pre[r], c0), e = min(r_pre[r + 1], c0 + nch);
            if (a >= e) continue;
            const int row = r >> 1;
            const int iy = row % cnty, iz = row / cnty;
            const int ry = fy ? imod(fsty + iy, nc1) - oy : iy - m, rz = fz ? imod(fstz + iz, nc2) - oz : iz - m;
            const T py = (T)ry - cy0, pz = (T)rz - cz0;
            const int beg = r_beg[r] - r_pre[r];
            for (int k = a + lane; k < e; k += 32) {
                const SrRec<T> S = src[beg + k];
                const int rx = fx ? S.cx - ox : imod(S.cx - fstx, nc0) - m;
                StPos<T> sp;
                sp.x = ((T)rx - cx0 + (T)0.5) * h0 + S.o[0];  // offsets are from the cell centre
                sp.y = (py + (T)0.5) * h1 + S.o[1];
                sp.z = (pz + (T)0.5) * h2 + S.o[2];
                sp.seg = S.seg;
                spos[k - c0] = sp;
                StChg<T> sq;
                sq.q[0] = S.q[0];
                sq.q[1] = S.q[1];
                sq.q[2] = S.q[2];
                sq.pad = (T)0;
                schg[k - c0] = sq;
            }
        }
        __syncthreads();
        for (int t = t0 + wid; t < t1; t += kStWarps) {
            const int j = tb_idx[t];
            const int jp = prev[j];
            const SrTgt<T> tg = tgt[j];
            const int cell = tg.cell;
            const int tcx = cell % nc0 - ox, tcy = (cell / nc0) % nc1 - oy, tcz = cell / (nc0 * nc1) - oz;
            const T px = ((T)tcx - cx0 + (T)0.5) * h0 + tg.o[0];
            const T py = ((T)tcy - cy0 + (T)0.5) * h1 + tg.o[1];
            const T pz = ((T)tcz - cz0 + (T)0.5) * h2 + tg.o[2];
            // the node's rows: staged rows within m cells (all rows of a full axis)
            const int iy0 = fy ? 0 : tcy, ny = fy ? cnty : 2 * m + 1;
            const int iz0 = fz ? 0 : tcz, nz = fz ? cntz : 2 * m + 1;
            const int nrw = ny * nz;
            T v0 = 0, v1 = 0, v2 = 0, p0 = 0, p1 = 0, p2 = 0;
            int qn = 0;  // warp-uniform queue length
            for (int rb = 0; rb < nrw; rb += 32) {
                // this lane's row and its candidate run [s, s + n) in the staged chunk
                int s = 0, n = 0;
                const int rr = rb + lane;
                if (rr < nrw) {
                    const int iy = iy0 + rr % ny, iz = iz0 + rr / ny;
                    const int row = iy + cnty * iz;
                    int klo = 0, khi = cntx - 1;
                    bool live = true;
                    if (!fx) {
                        // gaps between the node and the row's y and z slabs
                        T gy = (T)0, gz = (T)0;
                        if (!fy) {
                            const T ylo = ((T)(iy - m) - cy0) * h1;
                            gy = py < ylo ? ylo - py : (py > ylo + h1 ? py - ylo - h1 : (T)0);
                        }
                        if (!fz) {
                            const T zlo = ((T)(iz - m) - cz0) * h2;
                            gz = pz < zlo ? zlo - pz : (pz > zlo + h2 ? pz - zlo - h2 : (T)0);
                        }
                        const T d2 = gy * gy + gz * gz;
                        live = d2 < rcm2;
                        if (live) {
                            const T ext = sqrt(rcm2 - d2);
                            klo = (int)floor((px - ext) / h0 + cx0) + m;
                            khi = (int)floor((px + ext) / h0 + cx0) + m;
                            klo = max(klo, tcx);          // within m cells of the node's cell
                            khi = min(khi, tcx + 2 * m);
                        }
                    }
                    if (live && khi >= klo) {
                        const int* cr = c_beg + row * cpr;
                        const int a = max(cr[klo], c0), e = min(cr[khi + 1], c0 + nch);
                        if (e > a) {
                            s = a - c0;
                            n = e - a;
                        }
                    }
                }
                int inc = n;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += u;
                }
                const int tot = __shfl_sync(0xffffffffu, inc, 31);
                const int beg_l = inc - n;  // this lane's run starts at candidate beg_l
                for (int cb = 0; cb < tot; cb += 32) {
                    const int c = cb + lane;
                    // owner lane of candidate c: the last lane whose run starts at or before c
                    int lo = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int probe = __shfl_sync(0xffffffffu, beg_l, lo + step);
                        if (lo + step < 32 && probe <= c) lo += step;
                    }
                    const int ob = __shfl_sync(0xffffffffu, beg_l, lo);
                    const int os = __shfl_sync(0xffffffffu, s, lo);
                    bool ok = false;
                    const int k = os + (c - ob);
                    if (c < tot) {
                        const StPos<T> sp = spos[k];
                        T rx = sp.x - px, ry = sp.y - py, rz = sp.z - pz;
                        if (fx) rx = st_wrap(rx, L0);
                        if (fy) ry = st_wrap(ry, L1);
                        if (fz) rz = st_wrap(rz, L2);
                        const T r2 = rx * rx + ry * ry + rz * rz;
                        // C_0 of the node (Eq. BS_on_vortex); a source exactly on the node adds nothing
                        ok = r2 < rc2 && r2 > (T)0 && sp.seg != j && sp.seg != jp;
                    }
                    const unsigned msk = __ballot_sync(0xffffffffu, ok);
                    if (ok) q[qn + __popc(msk & lt)] = k;
                    qn += __popc(msk);
                    if (qn >= 32) {
                        __syncwarp();
                        {
                            const int kk = q[lane];
                            const StPos<T> sp = spos[kk];
                            T rx = sp.x - px, ry = sp.y - py, rz = sp.z - pz;
                            if (fx) rx = st_wrap(rx, L0);
                            if (fy) ry = st_wrap(ry, L1);
                            if (fz) rz = st_wrap(rz, L2);
                            st_pair<T>(rx, ry, rz, rx * rx + ry * ry + rz * rz, schg[kk].q, alpha, P.want_psi, v0, v1,
                                       v2, p0, p1, p2);
                        }
                        const int rest = qn - 32;
                        const int mv = lane < rest ? q[32 + lane] : 0;
                        __syncwarp();
                        if (lane < rest) q[lane] = mv;
                        __syncwarp();
                        qn = rest;
                    }
                }
            }
            __syncwarp();
            if (lane < qn) {
                const int kk = q[lane];
                const StPos<T> sp = spos[kk];
                T rx = sp.x - px, ry = sp.y - py, rz = sp.z - pz;
                if (fx) rx = st_wrap(rx, L0);
                if (fy) ry = st_wrap(ry, L1);
                if (fz) rz = st_wrap(rz, L2);
                st_pair<T>(rx, ry, rz, rx * rx + ry * ry + rz * rz, schg[kk].q, alpha, P.want_psi, v0, v1, v2, p0, p1,
                           p2);
            }
            __syncwarp();  // the queue is reused by the next node
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
            const double d0 = v0, d1 = v1, d2 = v2, e0 = p0, e1 = p1, e2 = p2;
            if (lane == 0) {
                // the first chunk writes, later ones add (same warp, ordered by the barriers)
                double* vj = vsr + 3 * (size_t)j;
                if (c0 == 0) {
                    vj[0] = P.pref * d0;
                    vj[1] = P.pref * d1;
                    vj[2] = P.pref * d2;
                } else {
                    atomicAdd(&vj[0], P.pref * d0);
                    atomicAdd(&vj[1], P.pref * d1);
                    atomicAdd(&vj[2], P.pref * d2);
                }
                if (P.want_psi) {
                    double* pj = psr + 3 * (size_t)j;
                    if (c0 == 0) {
                        pj[0] = P.pref * e0;
                        pj[1] = P.pref * e1;
                        pj[2] = P.pref * e2;
                    } else {
                        atomicAdd(&pj[0], P.pref * e0);
                        atomicAdd(&pj[1], P.pref * e1);
                        atomicAdd(&pj[2], P.pref * e2);
                    }
                }
            }
        }
    }
    if (total == 0) {
        // no source near the block: its nodes get zero
        for (int t = t0 + tid; t < t1; t += blockDim.x) {
            const int j = tb_idx[t];
            for (int c = 0; c < 3; ++c) {
                vsr[3 * (size_t)j + c] = 0.0;
                if (P.want_psi) psr[3 * (size_t)j + c] = 0.0;
            }
        }
    }
}

template <typename T>
cudaError_t launch_short(const ShortP& P, const Work& w, cudaStream_t s)
{
    if (P.N <= 0) return cudaSuccess;
    const int nblocks = P.nb[0] * P.nb[1] * P.nb[2];
    // the warp-per-node kernel is the default: measured faster on the random
    // tangles (12.8 against 18.0 ms on the 4e6-node tangle, 0.21 against 0.41
    // ms on the 1e5-node one), the tiled kernel only on request
    const bool tiled = P.m <= kShortTileMaxM && P.kernel == 1;
    if (!tiled) {
        const int tb = 32 * kShortWarps;  // one warp per target
        const long long threads = 32LL * P.N;
        k_short<T><<<(unsigned)((threads + tb - 1) / tb), tb, 0, s>>>(
            P, (const SrTgt<T>*)w.tgt, w.prev, w.cell_cnt, (const SrRec<T>*)w.sr_sorted, w.vsr, w.psr);
        return cudaGetLastError();
    }
    // nodes by target block: count, scan, scatter
    cudaError_t e = cudaMemsetAsync(w.tb_cnt, 0, sizeof(int) * (size_t)(nblocks + 1), s);
    if (e != cudaSuccess) return e;
    const int g = (P.N + kThreads - 1) / kThreads;
    k_tgt_key<T><<<g, kThreads, 0, s>>>(P, (const SrTgt<T>*)w.tgt, w.tb_key, w.tb_cnt);
    e = scan_exclusive(w.tb_cnt, nblocks, w.scan_tmp, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(w.tb_cur, w.tb_cnt, sizeof(int) * (size_t)nblocks, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    k_tgt_scatter<<<g, kThreads, 0, s>>>(P.N, w.tb_key, w.tb_cur, w.tb_idx);
    k_short_tile<T><<<nblocks, kStWarps * 32, 0, s>>>(P, (const SrTgt<T>*)w.tgt, w.prev, w.cell_cnt,
                                                     (const SrRec<T>*)w.sr_sorted, w.tb_cnt, w.tb_idx, w.vsr, w.psr);
    return cudaGetLastError();
}

// Batched: the warp-per-node kernel over every member (one warp per node).
template <typename T>
cudaError_t launch_short_b(const BatchL& L, cudaStream_t s)
{
    if (L.total > 0) k_short_b<T><<<L.total, 32 * kShortWarps, 0, s>>>((const ShortD<T>*)L.desc, L.bstart, L.n);
    return cudaGetLastError();
}

template cudaError_t launch_short_b<float>(const BatchL&, cudaStream_t);
template cudaError_t launch_short_b<double>(const BatchL&, cudaStream_t);
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
