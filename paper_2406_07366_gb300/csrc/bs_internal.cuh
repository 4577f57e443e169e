// Internal declarations of the bsewald CUDA library (not part of the ABI).
#pragma once

#include <cuda.h>  // CUtensorMap (tensor-copy descriptors; encoded through the runtime's driver entry point)
#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include "bsewald.h"

namespace bsw {

constexpr int kMaxQ = 8;
constexpr int kMaxW = 16;
constexpr int kThreads = 256;
constexpr size_t kSplineSmemMax = 96 * 1024;  // warp-per-filament spline fit up to this smem
constexpr double kPi = 3.14159265358979323846264338327950288;

// Device status bits (bs_status).
enum : int { ST_NONFINITE = 1, ST_GEOMETRY = 2, ST_TIMEOUT = 4 };

// Short-range source: offset from its cell origin, charge, x-cell index and
// the global index of its segment (the node at the segment start).
template <typename T> struct SrRec;
template <> struct __align__(16) SrRec<float> {
    float o[3];
    int cx;
    float q[3];
    int seg;
};
template <> struct __align__(16) SrRec<double> {
    double o[3];
    double q[3];
    int cx;
    int seg;
    int pad[2];
};

// Short-range target: node offset from its cell origin and packed cell.
template <typename T> struct __align__(16) SrTgt {
    T o[3];
    int cell;
};

// Long-range source: fractional grid position, charge, packed base index
// (10 bits per axis).
// Spread source with its charge and kernel weights along the three axes
// (support point t of axis d at grid index ib_d - W/2 + 1 + t), written
// once; every block of z-columns its support reaches holds its index.
template <typename T, int W> struct __align__(16) SpPt {
    int base;  // ib0 | ib1 << 10 | ib2 << 20
    T q[3];
    T wx[W];
    T wy[W];
    T wz[W];
};

// Interpolation target with its kernel weights along the three axes
// (support point t of axis d at grid index ib_d - W/2 + 1 + t), binned once
// by the z-column block that holds its grid cell.
template <typename T, int W> struct __align__(16) NdW {
    int base;  // ib0 | ib1 << 10 | ib2 << 20
    int j;     // node index
    T wx[W];
    T wy[W];
    T wz[W];
};

template <typename T> struct LrRec;
template <> struct __align__(16) LrRec<float> {
    float f[3];
    int base;
    float q[3];
    int pad;
};
template <> struct __align__(16) LrRec<double> {
    double f[3];
    double q[3];
    int base;
    int pad[3];
};

// Parameters of the geometry / node kernel.
struct GeomP {
    double L[3];
    int N;
    int nfil;
    int Q;
    double gh[kMaxQ];   // Gauss-Legendre nodes on [0,1]
    double gw[kMaxQ];   // weights, sum 1
    double kappa, a, delta, alpha;
    int nc[3];          // short-range cells per axis
    double hc[3];       // cell edge
    int ng[3];          // spread grid
    double hg[3];       // grid spacing
    int w;              // kernel width (even)
    int tile[3];        // spread tile edge
    int ntile[3];
    double seg_max;     // longest allowed segment chord (min L / 4)
    double iL[3], ihc[3], ihg[3];  // reciprocals of L, hc, hg (binning multiplies: float64 division is slow here)
    int want_psi;
    double local_frac;  // subdivided local segments (0: off)
    double log2a;       // log(2 / a): the local term's logarithm is log(l- l+) / 2 + log(2 / a)
};

struct ShortP {
    int N;
    int nc[3];
    double hc[3];
    double L[3];
    int m;              // cells per cut-off
    double rc2;
    double alpha;
    double pref;        // kappa / 4 pi
    int want_psi;
    int nb[3];          // target blocks of m x m x m cells per axis, ceil(nc / m)
    int kernel;         // 0: by size, 1: tiled, 2: warp per node (BS_SHORT_TILED / BS_SHORT_PER_NODE)
};

// The tiled short range takes cells per cut-off up to this (larger m: the
// warp-per-node kernel).
constexpr int kShortTileMaxM = 4;

struct SpreadP {
    int ng[3];
    int tile[3];
    int ntile[3];
    int w;
    double zeta, inorm;
};

struct KspaceP {
    int ng[3];
    int nh;             // ng[2]/2 + 1
    int K[3];           // mode cube
    double kk[3];       // 2 pi / L
    double scale;       // kappa / V
    int want_psi;
    double* energy;     // if non-null: += (1/2) sum_k e^{-k^2/4a^2} |omega_k|^2 / k^2
    double* epart;      // if non-null (deterministic): the CTA's share written to epart[blockIdx.x]
    // Spectrum mode (spectrum non-null): after the forward x transform, add
    // |k x F_k|^2 e^{s k^2 / 4a^2} prod tab_d / k^4 (s = +1 unsmoothed, -1
    // smoothed; both halves of the spectrum) to shell round(|k| / dk) of
    // spectrum[0..nbins), then stop (no k-space pass, no inverse).
    double* spectrum;
    int nbins;
    int smoothed;
    double dk;
    double inv4a2;      // 1 / (4 alpha^2)
    int single_decon;   // k-space tables with the spread's deconvolution only (grid field)
};

// Exact unsigned division by a run-time constant d for 0 <= x < 2^31
// (Granlund & Montgomery): q = umulhi(x, m) >> s, or x >> s for powers of 2.
struct FastDiv {
    unsigned d, m;
    int s;
    int pow2;
};

inline FastDiv make_fastdiv(unsigned d)
{
    FastDiv f;
    f.d = d;
    int l = 0;
    while ((1ull << l) < d) ++l;  // ceil(log2 d)
    if ((d & (d - 1)) == 0) {
        f.m = 0;
        f.s = l;
        f.pow2 = 1;
    } else {
        f.m = (unsigned)((1ull << (31 + l)) / d + 1);
        f.s = l - 1;
        f.pow2 = 0;
    }
    return f;
}

__device__ __forceinline__ int fdiv(int x, const FastDiv& f)
{
    return f.pow2 ? (int)((unsigned)x >> f.s) : (int)(__umulhi((unsigned)x, f.m) >> f.s);
}

// Radix sequence of one in-place 1-D transform of length n = r[0] ... r[nr-1].
// Pass s works on spans L_s = st[s] r[s] with butterfly stride st[s] =
// n / (r[0] ... r[s]); tws[s] = n / L_s is its twiddle step; sd[s] divides by
// st[s].  Decimation in frequency runs the passes forward and leaves
// frequency k at position rev(k) = sum_s d_s st[s] (k = d_0 + r[0] d_1 +
// r[0] r[1] d_2 + ...); decimation in time runs them backward and takes its
// input at those positions.
struct FftPlan {
    int n;
    int nr;
    int r[16];
    int st[16];
    int tws[16];
    FastDiv sd[16];
};

// Column binning of the spread records (blocks of tx x ty full z-columns).
struct ColP {
    int tx, ty, nbx, nby, ncols, w;
    int nzb;  // z-buckets per block (1: the copies of a block are not sorted by z)
    int n2;   // grid points along z
    double zeta;   // kernel shape parameter
    double inorm;  // 1 / (1 - e^{-2 zeta}), the kernel's normalisation
};

struct SpZP {
    int det;  // deterministic accumulation: each warp owns a z-range and adds in record order
    int nthreads;  // threads per CTA (256, or 512 for float32 on large grids)
    int ng[3];
    int K[3];
    int tx, ty, nbx, nby;
    int w;
    int nzb;            // z-buckets per block: > 1 selects the bucketed record loop
    int ls;             // padded stride of the real z-lines in shared memory
    int cls;            // complex line stride of the z FFT buffers
    double zeta;
    FftPlan plan2;
    const int* rev;  // position of frequency k after the forward transform, k < n
    FastDiv d_nbx, d_n2, d_nk, d_txy, d_ty, d_ncl;
};

struct FftYP {
    int ng[3];
    int K[3];
    int lmc;            // log2 of the chunk of z-modes per CTA
    int ls;             // line stride in shared memory
    int tby, tnb;       // tensor copies of F1 (tnb > 0): rows per box, boxes per CTA
    FftPlan plan1;
    const int* rev;
    FastDiv d_nch, d_lines;
};

struct FftXP {
    int ng[3];
    int K[3];
    int lmc;            // log2 of the chunk of z-modes per CTA
    int nthreads;       // threads per CTA (256, or 512 for float32 on large grids)
    int ls;             // line stride in shared memory
    int tbx, tnbx;      // tensor copies of F2 (tnbx > 0): x rows per box, boxes per CTA
    const int* irev;    // frequency at each position of an x line after the forward transform
    double kk[3];
    double scale;
    FftPlan plan0;
    const int* rev;
    FastDiv d_nch, d_n0, d_lines, d_lines_psi;
    double* energy;     // if non-null: += (1/2) sum_k e^{-k^2/4a^2} |omega_k|^2 / k^2
    double* epart;      // if non-null (deterministic): the CTA's share written to epart[blockIdx.x]
    // Spectrum mode (spectrum non-null): after the forward x transform, add
    // |k x F_k|^2 e^{s k^2 / 4a^2} prod tab_d / k^4 (s = +1 unsmoothed, -1
    // smoothed; both halves of the spectrum) to shell round(|k| / dk) of
    // spectrum[0..nbins), then stop (no k-space pass, no inverse).
    double* spectrum;
    int nbins;
    int smoothed;
    double dk;
    double inv4a2;      // 1 / (4 alpha^2)
    int single_decon;   // k-space tables with the spread's deconvolution only (grid field)
};

struct FftZP {
    int ng[3];
    int K[3];
    int yc;
    int cls;            // complex line stride in shared memory
    FftPlan plan2;
    const int* rev;  // position of frequency k after the forward transform, k < n
    FastDiv d_nch, d_n0, d_nk, d_n2, d_ncl;
};

struct InterpP {
    int N;
    int ng[3];
    double hg[3];
    double L[3];
    double iL[3], ihg[3];  // reciprocals of L and hg
    int w;
    double zeta, inorm;
    int want_psi;
};

// Workspace buffers (device) of one context; T-typed buffers are void*.
struct Work {
    // topology
    int64_t* off = nullptr;
    int* fil_of = nullptr;
    int* prev = nullptr;
    double* shift = nullptr;
    // spline
    void* hseg = nullptr;   // N
    void* dp = nullptr;     // N x 3 periodic increments
    void* ds = nullptr;     // N x 3 chord vectors
    void* Mm = nullptr;     // N x 3 moments (second derivatives at the nodes)
    void* Dd = nullptr;     // N x 3 first derivatives at the nodes (quintic splines only)
    double* qtmp = nullptr; // 19 N scratch of the quintic spline solve (and of the quintic energy integral)
    void* cpr = nullptr;    // N Thomas scratch
    void* zz = nullptr;     // N Sherman-Morrison vector
    void* Tper = nullptr;   // nfil
    int nmax_fil = 0;       // longest filament
    // node outputs
    double* vls = nullptr;  // N x 3  v_local - v_self
    double* pls = nullptr;  // N x 3  psi_local - psi_self
    double* vsr = nullptr;  // N x 3  short range (float64 sums of the pair terms)
    double* psr = nullptr;
    int* tb_key = nullptr;  // N  target block of every node (short range)
    int* tb_idx = nullptr;  // N  nodes sorted by target block
    int* tb_cnt = nullptr;  // nblocks + 1 block starts
    int* tb_cur = nullptr;  // nblocks scatter cursors
    void* tgt = nullptr;    // N SrTgt
    // sources
    void* sr_rec = nullptr;   // NQ
    void* sr_sorted = nullptr;
    int* sr_key = nullptr;
    void* lr_rec = nullptr;
    void* lr_sorted = nullptr;
    int* lr_key = nullptr;
    // counting sorts
    int* cell_cnt = nullptr;  // ncells + 1
    int* cell_cur = nullptr;
    int* tile_cnt = nullptr;  // ntiles + 1
    int* tile_cur = nullptr;
    int* scan_tmp = nullptr;   // short-range sort (side stream)
    int* scan_tmp2 = nullptr;  // long-range sort (main stream)
    // grids
    void* grid = nullptr;     // 3 x ng^3 real (allocated only where a path writes it)
    void* spec = nullptr;     // 3 x ng0 ng1 nh complex
    void* spec_psi = nullptr; // 3 x ... (psi)
    void* ktab = nullptr;     // per-axis k-space tables
    int* rev = nullptr;       // per-axis positions of frequency k after the forward transform (n0 + n1 + n2)
    double* shell = nullptr;  // energy-spectrum shell sums
    // BS_DETERMINISTIC: the source index of every binned copy (scatter order),
    // the copies re-ordered by it, and float64 partial sums reduced in order
    int* sr_idx = nullptr;
    void* sr_sorted2 = nullptr;
    int2* col_rec2 = nullptr; // the spread copies' entries in scatter order
    double* epart = nullptr;  // per-CTA energy partials of the x/k-space kernel
    double* lpart = nullptr;  // per-filament energy line integrals
    int nepart = 0;
    void* fft_work = nullptr;
    // pruned-FFT pipeline
    void* tw = nullptr;       // twiddles e^{-2 pi i j / n_d}, n0 + n1 + n2 complex
    void* f2 = nullptr;       // 3 x n0 x (2K1+1) x (K2+1) complex
    void* f2psi = nullptr;
    int2* col_rec = nullptr;  // every copy's (source index, relative support start), by z-column block
    void* col_pts = nullptr;  // SpPt per source (charge and kernel weights)
    int* col_cnt = nullptr;   // ncols + 1
    int* col_cur = nullptr;
    // fused inverse-z interpolation: the nodes with their weights, counting-
    // sorted by the z-column block of their grid cell
    void* nd_rec = nullptr;     // N NdW records, node order
    void* nd_sorted = nullptr;  // N NdW records, block order
    int* nd_key = nullptr;      // block of every node
    int* nd_rank = nullptr;     // rank of the node within its block
    int* ncol_cnt = nullptr;    // ncols + 1 block starts
    void* vacc = nullptr;       // N x 3 accumulated long-range velocity
    // host staging for bs_compute_host
    double* nodes_in = nullptr;
    double* vel_out = nullptr;
    double* psi_out = nullptr;
    int* status = nullptr;
    double* energy_acc = nullptr;  // [0] Fourier part, [1] line integral
};

// Launchers (explicit instantiations for float and double live in the .cu files).
template <typename T>
cudaError_t launch_spline(const double* nodes, const Work& w, int nfil, cudaStream_t s);
template <typename T>
cudaError_t launch_nodes(const GeomP& P, const double* nodes, const Work& w, double* part_local, double* part_self,
                         double* psi_local, double* psi_self, cudaStream_t s);
template <typename T>
cudaError_t launch_export_quadrature(const GeomP& P, const double* nodes, const Work& w, double* qX, double* qq,
                                     cudaStream_t s);
template <typename T>
cudaError_t launch_sort_sr(const Work& w, int NQ, int ncells, cudaStream_t s, bool det);
template <typename T>
cudaError_t launch_sort_lr(const Work& w, int NQ, int ntiles, cudaStream_t s);
template <typename T>
cudaError_t launch_short(const ShortP& P, const Work& w, cudaStream_t s);
template <typename T>
cudaError_t launch_spread(const SpreadP& P, const Work& w, int ntiles, cudaStream_t s);
template <typename T>
cudaError_t launch_kspace(const KspaceP& P, const Work& w, cudaStream_t s);
template <typename T>
cudaError_t launch_interp(const InterpP& P, const double* nodes, const Work& w, const void* grid, int what,
                          double* out, double* part_long, cudaStream_t s);

template <typename T>
cudaError_t launch_col_sort(const ColP& P, const Work& w, int NQ, cudaStream_t s, bool det);
template <typename T>
cudaError_t launch_spread_zfft(const SpZP& P, const Work& w, cudaStream_t s);
template <typename T>
size_t col_pt_bytes(int w);
cudaError_t set_fft_constants();
template <typename T>
cudaError_t launch_fft_y(const FftYP& P, const Work& w, void* f2, int sign, cudaStream_t s,
                         const CUtensorMap* tm_f1 = nullptr);
template <typename T>
cudaError_t launch_fft_x_kspace(const FftXP& P, const Work& w, bool want_psi, cudaStream_t s,
                                const CUtensorMap* tm_f2);
// Tensor-copy descriptor of F2 for the x pass: 4-D (2 nk reals, 3 components,
// n0 x rows, 2 K1 + 1 y modes), box (2 MC, 3, tbx, 1), which lands as x rows
// of the 3 MC lines' modes; false where the layout does not allow it.
template <typename T>
bool make_tmap_x(void* F2, const FftXP& P, CUtensorMap* tm);
// Tensor-copy descriptor of F1 for the y pass: 3-D (2 nk reals, n1 rows,
// 3 n0 lines), box (2 MC, tby, 1); false where the layout does not allow it
// (float32 with an odd nk: rows not 16-byte multiples; MC < 2).
template <typename T>
bool make_tmap_y(void* F1, const FftYP& P, CUtensorMap* tm);
template <typename T>
cudaError_t launch_fft_x_kspace(const FftXP& P, const Work& w, bool want_psi, cudaStream_t s);
// Inverse z transform into the real grid (w.grid), or, with out64, into a
// float64 grid of the same layout (the coarse-grained field).
template <typename T>
cudaError_t launch_fft_z_c2r(const FftZP& P, const Work& w, cudaStream_t s, double* out64 = nullptr);
// Blocks whose points are gathered from home-block lists (the points sorted
// once by the block of their grid cell): the home blocks a CTA gathers are
// distinct and at most 64, and one periodic image of a support meets a block
// (the grid wider than the support plus a block).
inline bool home_fits(int tx, int ty, int w, int n0, int n1, int nbx, int nby)
{
    const int nhx = (tx + w - 2) / tx + 2, nhy = (ty + w - 2) / ty + 2;
    return nhx * nhy <= 64 && nhx <= nbx && nhy <= nby && n0 >= w + tx && n1 >= w + ty;
}

// The fused inverse-z interpolation also pairs adjacent y rows into one
// complex line (Ty even).
inline bool zfft_interp_fits(int tx, int ty, int w, int n0, int n1, int nbx, int nby)
{
    return ty % 2 == 0 && home_fits(tx, ty, w, n0, n1, nbx, nby);
}
template <typename T>
cudaError_t launch_zfft_interp(const SpZP& P, const Work& w, cudaStream_t s);
template <typename T>
cudaError_t launch_node_bin(const ColP& P, const InterpP& I, const double* nodes, const Work& w, cudaStream_t s);
template <typename T>
size_t nd_rec_bytes(int w);
template <typename T>
cudaError_t launch_interp_sum(int N, const Work& w, int what, double* out, double* part_long, cudaStream_t s);
template <typename T>
size_t spread_zfft_smem(const SpZP& P);

template <typename T>
cudaError_t launch_energy_line(const double* nodes, const Work& w, int nfil, int nmax, cudaStream_t s, bool det);
// Warp per segment: out[start[s] + rank] = in[i] with rank the position of
// key[i] among the segment's keys (distinct within a segment).
template <typename R>
cudaError_t launch_segsort(const int* start, int nseg, const R* in, const int* key, R* out, cudaStream_t s);
cudaError_t launch_segsort_bytes(const int* start, int nseg, const void* in, const int* key, void* out,
                                 size_t rec_bytes, cudaStream_t s);
// Warp per segment: the segment's pairs in increasing order of .x (distinct).
cudaError_t launch_segsort_int2(const int* start, int nseg, const int2* in, int2* out, cudaStream_t s);

template <typename T>
cudaError_t launch_to_double(const void* in, double* out, int n, cudaStream_t s);

// Set the thread-local message returned by bs_last_error.
cudaError_t launch_rk4_stage(const double* x0, const double* k, double c, double* out, long long n, cudaStream_t s);
cudaError_t launch_rk4_final(double* x, const double* k1, const double* k2, const double* k3, const double* k4,
                             double h, long long n, cudaStream_t s);

void set_last_error(const char* msg);

// ---------------------------------------------------------------------------
// Batched stage launches.  One launch serves every member of a batch: member
// m owns the launch's CTAs [bstart[m], bstart[m + 1]) and runs them as its
// blocks 0 .. bstart[m + 1] - bstart[m] - 1, with its own arguments (a
// descriptor per member, in device memory).  No CTA waits on another.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int batch_member(const int* __restrict__ bstart, int n, int& bid, int& nb)
{
    const int b = (int)blockIdx.x;
    int lo = 0, hi = n;  // bstart[lo] <= b < bstart[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(bstart + mid) <= b) lo = mid;
        else hi = mid;
    }
    const int b0 = __ldg(bstart + lo);
    bid = b - b0;
    nb = __ldg(bstart + lo + 1) - b0;
    return lo;
}

// A member's parameter struct copied into shared memory by the CTA (the
// transform loops read the plan at every pass: shared memory instead of the
// descriptor in global memory).  Every thread calls it; it ends with a barrier.
template <typename PT>
__device__ __forceinline__ void batch_param_copy(PT& dst, const PT& src)
{
    static_assert(sizeof(PT) % 4 == 0, "parameter structs are copied as 4-byte words");
    const int* s = reinterpret_cast<const int*>(&src);
    int* d = reinterpret_cast<int*>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(PT) / 4); i += blockDim.x) d[i] = s[i];
    __syncthreads();
}

// A batched launch: descriptors and block starts in device memory.
struct BatchL {
    const void* desc;
    const int* bstart;
    int n;        // members
    int total;    // CTAs of the launch
    int threads;  // threads per CTA
    size_t smem;  // dynamic shared memory per CTA (the largest member's)
};

// Descriptors of the batched stages (one per member).
struct ZeroD { int* p; int n; };                  // p[0..n) = 0
struct CopyD { const int* src; int* dst; int n; };
struct CountD { const int* key; int n; int* cnt; };
struct ScanD { int* cnt; int n; int* part; int nb; };
template <typename R> struct ScatterD { const int* key; const R* in; int n; int* cur; R* out; };

template <typename T> struct SplineD {
    const double* nodes;
    const int64_t* off;
    const double* shift;
    int nfil, nmax;
    T *hseg, *dp, *ds, *Mm, *Tper;
};
template <typename T> struct NodesD {
    GeomP P;
    const double* nodes;
    const int* fil_of;
    const int* prev;
    const int64_t* off;
    const double* shift;
    const T *hseg, *dp, *ds, *Mm, *Tper, *Dd;
    SrRec<T>* sr_rec;
    int* sr_key;
    LrRec<T>* lr_rec;
    int* lr_key;
    SrTgt<T>* tgt;
    double *vls, *pls;
    int* status;
};
template <typename T> struct ShortD {
    ShortP P;
    const SrTgt<T>* tgt;
    const int* prev;
    const int* start;
    const SrRec<T>* src;
    double *vsr, *psr;
};
template <typename T> struct ColD {      // k_col_count (out unused) and k_col_scatter
    ColP P;
    const LrRec<T>* rec;
    int n;
    int* cnt;                             // counts (count) or cursors (scatter)
    void* out;                            // int2 (source index, relative start) per copy (scatter)
    void* pts;                            // SpPt<T, W>, one per source (scatter)
};
template <typename T> struct SpzD {      // k_spread_zfft and k_zfft_interp
    SpZP P;
    const int* cstart;
    const void* recs;                     // int2 copy entries (spread) or NdW<T, W> (interpolation)
    const void* pts;                      // SpPt<T, W> (spread)
    const void* tw2;
    void* F1;                             // written (spread) or read (interpolation)
    T* vacc;                              // interpolation sums
};
template <typename T> struct FftYD {
    FftYP P;
    void* F1;
    void* F2;
    const void* tw1;
    int sign;
};
template <typename T> struct FftXD {
    FftXP P;
    void* F2;
    const void* tw0;
    const T *tab0, *tab1, *tab2;
};
template <typename T> struct NodeWD {   // k_node_w and k_node_scatter
    InterpP P;
    int tx, ty, nbx;
    const double* nodes;
    void* rec;                            // NdW<T, W>, node order
    int* key;
    int* rank;
    int* cnt;                             // block counts, then starts
    void* sorted;                         // NdW<T, W>, block order
};
template <typename T> struct SumD {
    int n3;
    const T* acc;
    const double* add_d;
    const double* add_t;
    double* out;
};

template <typename T>
cudaError_t launch_spline_b(const BatchL& L, cudaStream_t s);
template <typename T>
cudaError_t launch_nodes_b(const BatchL& L, cudaStream_t s);
template <typename T>
cudaError_t launch_short_b(const BatchL& L, cudaStream_t s);
template <typename T>
cudaError_t launch_col_count_b(const BatchL& L, cudaStream_t s);
template <typename T>
cudaError_t launch_col_scatter_b(int w, const BatchL& L, cudaStream_t s);
template <typename T>
cudaError_t launch_spread_zfft_b(int w, const BatchL& L, cudaStream_t s);
template <typename T>
cudaError_t launch_fft_y_b(const BatchL& L, cudaStream_t s);
template <typename T>
cudaError_t launch_fft_x_kspace_b(const BatchL& L, cudaStream_t s);
template <typename T>
cudaError_t launch_node_w_b(int w, const BatchL& L, cudaStream_t s);
template <typename T>
cudaError_t launch_node_scatter_b(int w, const BatchL& L, cudaStream_t s);
template <typename T>
cudaError_t launch_zfft_interp_b(int w, const BatchL& L, cudaStream_t s);
template <typename T>
cudaError_t launch_interp_sum_b(const BatchL& L, cudaStream_t s);
// shared memory of one member's CTA in the launches above
template <typename T>
size_t spline_smem(int nmax);
template <typename T>
size_t fft_y_smem(const FftYP& P);
template <typename T>
size_t fft_x_smem(const FftXP& P);
template <typename T>
size_t zfft_interp_smem(const SpZP& P);

cudaError_t launch_zero_b(const BatchL& L, cudaStream_t s);
cudaError_t launch_copy_b(const BatchL& L, cudaStream_t s);
cudaError_t launch_count_b(const BatchL& L, cudaStream_t s);
// the three phases of the exclusive scan, per member: L1 over each member's
// scan tiles (scan_blocks(n)), L2 one CTA per member
cudaError_t launch_scan_b(const BatchL& L1, const BatchL& L2, cudaStream_t s);
template <typename R>
cudaError_t launch_scatter_b(const BatchL& L, cudaStream_t s);

// Exclusive scan of n ints in place (cnt[n] receives the total); tmp holds
// scan_blocks(n) ints.
cudaError_t scan_exclusive(int* cnt, int n, int* tmp, cudaStream_t s);
int scan_blocks(int n);

}  // namespace bsw
