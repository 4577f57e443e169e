// C ABI of the bsewald library: parameter helpers (Sec. 4, Sec. 5.3, Table
// tab:performance), NUFFT set-up (Appendix A), context lifecycle and the
// evaluation pipeline of Eq. ewald_velocity_splitting:
//
//   main stream : spline -> nodes (sources, local - self) --fork--+
//                 tile sort -> spread -> FFT -> k-space -> FFT^-1  |
//                 --join-- interpolation + sum                     |
//   side stream : cell sort -> short range  <---------------------+
//
// The compute calls allocate nothing: every buffer, the cuFFT plans and
// their work area are made in bs_create / bs_set_filaments.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "bs_internal.cuh"

using namespace bsw;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                                     \
    do {                                                                                                   \
        cudaError_t _e = (expr);                                                                           \
        if (_e != cudaSuccess) {                                                                           \
            return fail(_e == cudaErrorMemoryAllocation ? BS_ERR_OOM : BS_ERR_CUDA, "%s: %s", #expr,      \
                        cudaGetErrorString(_e));                                                           \
        }                                                                                                  \
    } while (0)

#define CUFFT_TRY(expr)                                                                                    \
    do {                                                                                                   \
        cufftResult _r = (expr);                                                                           \
        if (_r != CUFFT_SUCCESS) return fail(BS_ERR_CUFFT, "%s: cufft error %d", #expr, (int)_r);         \
    } while (0)

// ---------------------------------------------------------------- host numerics
// Gauss-Legendre nodes/weights on [-1, 1] (Newton on the Legendre recurrence).
void gauss_legendre(int n, double* x, double* w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(kPi * (i + 0.75) / (n + 0.5));
        double pp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int k = 1; k <= n; ++k) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double z1 = z;
            z = z1 - p1 / pp;
            if (fabs(z - z1) < 1e-16) break;
        }
        double p1 = 1.0, p2 = 0.0;
        for (int k = 1; k <= n; ++k) {
            double p3 = p2;
            p2 = p1;
            p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
        }
        pp = n * (z * p1 - p2) / (z * z - 1.0);
        x[i] = -z;  // ascending
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

// Smallest m >= n with m % 8 == 0 and m = 2^a 3^b (the lengths the
// library's transforms handle).
int fft_friendly(int n)
{
    for (int m = std::max(n, 8);; ++m) {
        if (m % 8) continue;
        int r = m;
        for (int p : { 2, 3 })
            while (r % p == 0) r /= p;
        if (r == 1) return m;
    }
}

// Line stride (in complex elements) of nl lines of length n in shared memory:
// with the line-fastest butterfly order, a group of `slots` threads (one
// shared-memory wavefront: 16 float2 or 8 double2) spans nl lines x slots/nl
// positions, which fall in distinct banks when stride = slots/nl (mod slots);
// for nl >= slots an odd stride suffices.
int line_stride(int n, int nl, int slots)
{
    const int target = nl >= slots ? 1 : (slots % nl == 0 ? slots / nl : 1);
    return n + (((target - n) % slots) + slots) % slots;
}

// Radices of a length-n transform: the fewest in-register passes, each of a
// size the kernels implement (up to maxr), and among those the most even
// split (largest smallest factor), largest factor first.
void plan_search(int n, int maxr, int start, std::vector<int>& cur, std::vector<int>& best)
{
    static const int kRadices[] = { 32, 24, 16, 12, 9, 8, 6, 4, 3, 2 };
    if (n == 1) {
        if (best.empty() || cur.size() < best.size() ||
            (cur.size() == best.size() && cur.back() > best.back()))
            best = cur;
        return;
    }
    if (!best.empty() && cur.size() + 1 > best.size()) return;
    for (int i = start; i < 10; ++i) {
        const int r = kRadices[i];
        if (r > maxr || n % r) continue;
        cur.push_back(r);
        plan_search(n / r, maxr, i, cur, best);
        cur.pop_back();
    }
}

FftPlan make_plan(int n, int maxr)
{
    FftPlan pl;
    pl.n = n;
    std::vector<int> cur, best;
    plan_search(n, maxr, 0, cur, best);
    pl.nr = (int)best.size();
    for (int s = 0; s < pl.nr; ++s) pl.r[s] = best[s];
    int L = n;
    for (int s = 0; s < pl.nr; ++s) {
        pl.st[s] = L / pl.r[s];
        pl.tws[s] = n / L;
        pl.sd[s] = make_fastdiv((unsigned)pl.st[s]);
        L = pl.st[s];
    }
    return pl;
}

// Position of frequency index k (0 <= k < n) after the forward (decimation
// in frequency) transform of plan pl: the mixed-radix digits of k, least
// significant first in the order of the passes, weighted by the pass strides.
int rev_pos_host(int k, const FftPlan& pl)
{
    int p = 0;
    for (int s = 0; s < pl.nr; ++s) {
        p += (k % pl.r[s]) * pl.st[s];
        k /= pl.r[s];
    }
    return p;
}

// Normalised backwards Kaiser-Bessel kernel psi(z) = sinh(zeta s)/(s sinh zeta).
double kb_host(double z, double zeta)
{
    double s2 = 1.0 - z * z;
    if (s2 < 0) s2 = 0;
    const double s = sqrt(s2);
    const double num = s > 1e-12 ? -expm1(-2.0 * zeta * s) / s : 2.0 * zeta;
    return exp(zeta * (s - 1.0)) * num / (1.0 - exp(-2.0 * zeta));
}

// F(m) = (w/2) int_{-1}^{1} psi(z) cos(kappa z) dz, kappa = pi m w / n_g: the
// continuous Fourier transform of the spreading kernel as used (width w grid
// points) divided by the grid spacing.  Gauss-Legendre with 400 points (the
// integrand is entire in z).
void kb_fourier(double zeta, int w, int ng, int K, double* F)
{
    const int nq = 400;
    std::vector<double> x(nq), wt(nq);
    gauss_legendre(nq, x.data(), wt.data());
    std::vector<double> pz(nq);
    for (int i = 0; i < nq; ++i) pz[i] = kb_host(x[i], zeta);
    for (int m = 0; m <= K; ++m) {
        const double kap = kPi * m * w / ng;
        double s = 0;
        for (int i = 0; i < nq; ++i) s += wt[i] * pz[i] * cos(kap * x[i]);
        F[m] = 0.5 * w * s;
    }
}

struct Derived {
    int ng[3], nh, K[3];
    double zeta;
    double hg[3];
    int tile[3], ntile[3], ntiles;
    int nc[3], m;
    long long ncells;
    double hc[3];
    // pruned-FFT pipeline
    FftPlan plan[3];
    int tx, ty, nbx, nby, ncols, colcap;  // z-column blocks; records per source at most
    int nzb, ncolb;                       // z-buckets per block; bins of the spread copies (ncols nzb)
    int nshell;                            // spectrum shells reaching the mode cube's corner
    int lmcy, lmcx, yc;                   // log2 chunk sizes of the y and x passes; inverse-z chunk
    int zthreads;                         // threads of a z-column-block CTA (256 or 512)
    int lsz;                              // padded stride of the real z-lines of the spread
    int fuse_interp;                      // inverse z fused with the interpolation (no real grid)
};

int derive(const bs_params* p, Derived* d)
{
    const double Lmin = std::min(p->L[0], std::min(p->L[1], p->L[2]));
    for (int c = 0; c < 3; ++c)
        if (!(p->L[c] > 0) || !isfinite(p->L[c])) return fail(BS_ERR_ARG, "L[%d] must be positive and finite", c);
    if (!isfinite(p->kappa)) return fail(BS_ERR_ARG, "kappa must be finite");
    if (!(p->a > 0) || !isfinite(p->a)) return fail(BS_ERR_ARG, "core radius a must be positive");
    if (!isfinite(p->delta)) return fail(BS_ERR_ARG, "delta must be finite");
    if (!(p->alpha > 0) || !isfinite(p->alpha)) return fail(BS_ERR_ARG, "alpha must be positive");
    if ((p->flags & BS_SHORT_TILED) && (p->flags & BS_SHORT_PER_NODE))
        return fail(BS_ERR_ARG, "BS_SHORT_TILED and BS_SHORT_PER_NODE exclude each other");
    if ((p->flags & BS_DETERMINISTIC) && (p->flags & BS_FFT_CUFFT))
        return fail(BS_ERR_ARG, "BS_DETERMINISTIC needs the default transform path, not BS_FFT_CUFFT");
    if (!(p->rc > 0) || !isfinite(p->rc)) return fail(BS_ERR_ARG, "rc must be positive");
    if (p->rc > 0.5 * Lmin * (1 + 1e-12))
        return fail(BS_ERR_RC_GT_HALF_L, "rc = %g exceeds min(L)/2 = %g", p->rc, 0.5 * Lmin);
    if (p->quad_Q < 1 || p->quad_Q > kMaxQ) return fail(BS_ERR_ARG, "quad_Q must be in 1..%d", kMaxQ);
    if (p->spline_order != 4 && p->spline_order != 6)
        return fail(BS_ERR_ARG, "spline_order %d not supported (4 = cubic, 6 = quintic)", p->spline_order);
    if (p->nufft_w < 2 || p->nufft_w > kMaxW || (p->nufft_w & 1))
        return fail(BS_ERR_ARG, "nufft_w must be even in 2..16");
    if (!(p->nufft_sigma > 1.0) || p->nufft_sigma > 4.0) return fail(BS_ERR_ARG, "nufft_sigma must be in (1, 4]");
    if (p->precision != BS_FP64 && p->precision != BS_MIXED) return fail(BS_ERR_ARG, "unknown precision");
    if (p->cell_div < 0 || p->cell_div > 8) return fail(BS_ERR_ARG, "cell_div must be in 0..8");
    if (!(p->local_frac >= 0.0 && p->local_frac < 1.0)) return fail(BS_ERR_ARG, "local_frac must be in [0, 1)");
    for (int c = 0; c < 3; ++c) {
        if (p->M[c] < 3) return fail(BS_ERR_ARG, "M[%d] must be >= 3", c);
        d->K[c] = (p->M[c] - 1) / 2;
        int n = fft_friendly((int)ceil(p->nufft_sigma * p->M[c]));
        n = std::max(n, fft_friendly(2 * p->nufft_w));
        if (n > 1024) return fail(BS_ERR_ARG, "spread grid %d > 1024 along axis %d", n, c);
        d->ng[c] = n;
        d->hg[c] = p->L[c] / n;
        d->tile[c] = 8;
        d->ntile[c] = n / 8;
    }
    if (d->ng[2] % 32 == 0) d->tile[2] = 32;
    else if (d->ng[2] % 16 == 0) d->tile[2] = 16;
    d->ntile[2] = d->ng[2] / d->tile[2];
    d->ntiles = d->ntile[0] * d->ntile[1] * d->ntile[2];
    d->nh = d->ng[2] / 2 + 1;
    // zeta = gamma w pi (1 - 1/(2 sigma)), gamma = 0.995 (Appendix A); with
    // the effective sigma of the rounded grid of the first axis.
    const double sig = (double)d->ng[0] / p->M[0];
    d->zeta = 0.995 * p->nufft_w * kPi * (1.0 - 1.0 / (2.0 * sig));
    d->m = p->cell_div > 0 ? p->cell_div : 2;
    for (;;) {
        long long tot = 1;
        for (int c = 0; c < 3; ++c) {
            int n = (int)floor(p->L[c] * d->m / p->rc);
            n = std::max(n, 1);
            d->nc[c] = n;
            d->hc[c] = p->L[c] / n;
            tot *= n;
        }
        d->ncells = tot;
        if (tot <= (1LL << 27) || d->m == 1) break;
        d->m -= 1;
    }
    if (d->ncells > (1LL << 28)) return fail(BS_ERR_ARG, "too many short-range cells (rc too small)");
    // pruned-FFT pipeline shapes: single-buffer in-place transforms, shared
    // memory per CTA near 50 KB (4-5 CTAs per SM)
    const size_t rb = p->precision == BS_FP64 ? 8 : 4;
    const size_t cb = 2 * rb;
    for (int c = 0; c < 3; ++c) d->plan[c] = make_plan(d->ng[c], 8);
    // Blocks of z-columns sized for about 50 KB of shared memory per CTA of
    // 256 threads; float32 blocks on grids of more than ~260 points per axis
    // are doubled and run by 512 threads at two CTAs per SM (about 85 KB
    // each).  Larger blocks mean fewer copies of each spread point (small
    // grids keep 256 threads: there the CTA count is what fills the GPU,
    // measured on the batch of 64 tangles).  Measured, on the
    // 384^3 grid of the 1e5-node tangle 4 x 4 blocks (5.6 copies) against
    // 2 x 4 (8.75 copies) take the spread binning, spread and fused
    // interpolation from 1.10 to 1.07 ms, and on the 768^3 grid of the
    // 4e6-node tangle 2 x 4 blocks against 1 x 4 take a whole evaluation
    // from 58.1 to 53.5 ms.
    int txy = (int)(50000 / (1.5 * (d->ng[2] + 1) * cb));
    txy = txy >= 16 ? 16 : (txy >= 8 ? 8 : (txy >= 4 ? 4 : 2));
    d->zthreads = 256;
    if (rb == 4 && txy < 16) {  // grids of more than ~260 points per axis
        txy *= 2;
        d->zthreads = 512;
    }
    d->ty = std::min(4, txy);
    d->tx = txy / d->ty;
    if (p->block_x > 0 || p->block_y > 0 || p->block_threads > 0) {
        // a chosen block (bs_autotune_tiles): shapes in {1, 2, 4}^2, 256 or
        // 512 threads (512 in float32 only), within the shared memory of a CTA
        const int bx = p->block_x > 0 ? p->block_x : d->tx, by = p->block_y > 0 ? p->block_y : d->ty;
        const int bt = p->block_threads > 0 ? p->block_threads : d->zthreads;
        auto ok = [](int v) { return v == 1 || v == 2 || v == 4; };
        if (!ok(bx) || !ok(by) || bx * by < 2) return fail(BS_ERR_ARG, "block_x, block_y must be in {1, 2, 4}");
        if (bt != 256 && !(bt == 512 && rb == 4)) return fail(BS_ERR_ARG, "block_threads must be 256 (or 512 in float32)");
        const size_t lines = (size_t)(3 * bx * by / 2) * (size_t)(d->ng[2] + 33) * cb;
        if (lines + 128 * (size_t)(16 + 24 * rb + 16 * (size_t)rb * p->nufft_w / 4) > 220 * 1024)
            return fail(BS_ERR_ARG, "block %d x %d does not fit in shared memory at %d points per line", bx, by,
                        d->ng[2]);
        d->tx = bx;
        d->ty = by;
        d->zthreads = bt;
    }
    d->nbx = d->ng[0] / d->tx;
    d->nby = d->ng[1] / d->ty;
    d->ncols = d->nbx * d->nby;
    // the bucketed spread (copies of a block sorted by the z-bucket of their
    // support start, partial sums in registers): even block height, a warp's
    // lanes over (y column, z offset), two buckets' planes distinct; the
    // deterministic mode keeps the record order of its own loop
    {
        const int W = p->nufft_w;
        const bool bucketed = !(p->flags & BS_DETERMINISTIC) && d->ty % 2 == 0 && d->ty * W <= 32 &&
                              d->ng[2] >= 2 * W;
        d->nzb = bucketed ? (d->ng[2] + W - 1) / W : 1;
        d->ncolb = d->ncols * d->nzb;
    }
    d->colcap = ((p->nufft_w - 1) / d->tx + 2) * ((p->nufft_w - 1) / d->ty + 2);
    {
        const double Lmin = std::min(p->L[0], std::min(p->L[1], p->L[2]));
        double r2 = 0.0;  // |k_corner| / dk, dk = 2 pi / min L
        for (int c = 0; c < 3; ++c) r2 += (d->K[c] * Lmin / p->L[c]) * (d->K[c] * Lmin / p->L[c]);
        d->nshell = (int)ceil(sqrt(r2)) + 2;
    }
    const size_t mcy = 50000 / ((size_t)(d->ng[1] + 1) * cb);
    d->lmcy = 0;
    while (d->lmcy < 4 && ((size_t)2 << d->lmcy) <= mcy) ++d->lmcy;
    const int lines_x = (p->flags & BS_WANT_PSI) ? 6 : 3;
    // the x pass gets the same larger CTAs as the z-column blocks (two
    // 512-thread CTAs per SM; measured on the 384^3 grid: 0.29 ms against
    // 0.32 ms for the x transforms with the k-space pass)
    const size_t mcx = (d->zthreads == 512 ? 100000 : 50000) / ((size_t)lines_x * (d->ng[0] + 1) * cb);
    d->lmcx = 0;
    while (d->lmcx < 4 && ((size_t)2 << d->lmcx) <= mcx) ++d->lmcx;
    // inverse z: 2 yc real lines per CTA as yc/2 complex ones; 16 complex
    // lines at an odd stride keep every transform pass free of bank conflicts
    d->yc = (rb == 4 && d->ng[1] % 32 == 0) ? 32 : ((d->ng[1] % 16 == 0) ? 16 : 8);
    d->lsz = d->ng[2] + 1;
    // the fused inverse z + interpolation gives every node copy one warp with
    // a lane per (y column, z offset); its float sums are added atomically,
    // so the deterministic mode keeps the grid and the gather kernel
    d->fuse_interp = !(p->flags & (BS_FFT_CUFFT | BS_DETERMINISTIC)) &&
                     zfft_interp_fits(d->tx, d->ty, p->nufft_w, d->ng[0], d->ng[1], d->nbx, d->nby);
    return BS_OK;
}

}  // namespace

void bsw::set_last_error(const char* msg) { g_err = msg ? msg : ""; }

struct bs_ctx {
    bs_params p;
    Derived d;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    static constexpr int kStages = 11;
    cudaEvent_t ev_t[kStages] = {};
    bool timed = false;
    int nfil = 0;
    long long N = 0, NQ = 0;
    bool have_fil = false;
    Work w;
    cufftHandle plan_fwd = 0, plan_inv = 0;
    bool plans = false;
    long long bytes = 0;
    std::vector<std::pair<void*, size_t>> alloc_n, alloc_g;
    int device = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    double* rk = nullptr;  // RK4 workspace: k1..k4 and the stage positions, 5 x N x 3
    cudaGraph_t rk_graph = nullptr;
    cudaGraphExec_t rk_exec = nullptr;
    // tensor-copy descriptor of F1 for the y pass, built for the buffer
    // tmy_for (rebuilt if the grids move)
    CUtensorMap tmy;
    const void* tmy_for = nullptr;
    bool tmy_ok = false;
    // the same for F2 in the x pass
    CUtensorMap tmx;
    const void* tmx_for = nullptr;
    bool tmx_ok = false;
};

namespace {

int dalloc(bs_ctx* c, std::vector<std::pair<void*, size_t>>& list, void** ptr, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return fail(BS_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    list.push_back({ *ptr, bytes });
    c->bytes += (long long)bytes;
    return BS_OK;
}

void free_list(bs_ctx* c, std::vector<std::pair<void*, size_t>>& list)
{
    for (auto& pr : list) {
        cudaFree(pr.first);
        c->bytes -= (long long)pr.second;
    }
    list.clear();
}

#define TRY(expr)                   \
    do {                            \
        int _rc = (expr);           \
        if (_rc != BS_OK) return _rc; \
    } while (0)

template <typename T>
int make_plans(bs_ctx* c)
{
    const Derived& d = c->d;
    int n[3] = { d.ng[0], d.ng[1], d.ng[2] };
    const long long rsz = (long long)d.ng[0] * d.ng[1] * d.ng[2];
    const long long csz = (long long)d.ng[0] * d.ng[1] * d.nh;
    CUFFT_TRY(cufftCreate(&c->plan_fwd));
    CUFFT_TRY(cufftCreate(&c->plan_inv));
    c->plans = true;
    CUFFT_TRY(cufftSetAutoAllocation(c->plan_fwd, 0));
    CUFFT_TRY(cufftSetAutoAllocation(c->plan_inv, 0));
    size_t ws1 = 0, ws2 = 0;
    const bool f32 = sizeof(T) == 4;
    CUFFT_TRY(cufftMakePlanMany(c->plan_fwd, 3, n, nullptr, 1, (int)rsz, nullptr, 1, (int)csz,
                                f32 ? CUFFT_R2C : CUFFT_D2Z, 3, &ws1));
    CUFFT_TRY(cufftMakePlanMany(c->plan_inv, 3, n, nullptr, 1, (int)csz, nullptr, 1, (int)rsz,
                                f32 ? CUFFT_C2R : CUFFT_Z2D, 3, &ws2));
    TRY(dalloc(c, c->alloc_g, &c->w.fft_work, std::max(ws1, ws2)));
    CUFFT_TRY(cufftSetWorkArea(c->plan_fwd, c->w.fft_work));
    CUFFT_TRY(cufftSetWorkArea(c->plan_inv, c->w.fft_work));
    return BS_OK;
}

template <typename T>
int alloc_grids(bs_ctx* c)
{
    const Derived& d = c->d;
    const size_t rsz = (size_t)d.ng[0] * d.ng[1] * d.ng[2];
    const size_t csz = (size_t)d.ng[0] * d.ng[1] * d.nh;
    // the real grid: written only for psi, the deterministic mode, the cuFFT
    // form and the unfused interpolation (1.4 GB at 384^3 float32, 5.4 GB at 768^3)
    const bool need_grid = (c->p.flags & (BS_WANT_PSI | BS_DETERMINISTIC | BS_FFT_CUFFT)) || !d.fuse_interp;
    if (need_grid) TRY(dalloc(c, c->alloc_g, &c->w.grid, 3 * rsz * sizeof(T)));
    TRY(dalloc(c, c->alloc_g, &c->w.spec, 3 * csz * 2 * sizeof(T)));
    if ((c->p.flags & BS_WANT_PSI) && (c->p.flags & BS_FFT_CUFFT))
        TRY(dalloc(c, c->alloc_g, &c->w.spec_psi, 3 * csz * 2 * sizeof(T)));
    TRY(dalloc(c, c->alloc_g, (void**)&c->w.tile_cnt, sizeof(int) * (size_t)(d.ntiles + 1)));
    TRY(dalloc(c, c->alloc_g, (void**)&c->w.tile_cur, sizeof(int) * (size_t)(d.ntiles + 1)));
    TRY(dalloc(c, c->alloc_g, (void**)&c->w.scan_tmp2,
               sizeof(int) * (size_t)std::max(scan_blocks(d.ntiles), scan_blocks(d.ncolb))));
    TRY(dalloc(c, c->alloc_g, (void**)&c->w.col_cnt, sizeof(int) * (size_t)(d.ncolb + 1)));
    TRY(dalloc(c, c->alloc_g, (void**)&c->w.col_cur, sizeof(int) * (size_t)(d.ncolb + 1)));
    {
        const size_t f2n = 3 * (size_t)d.ng[0] * (2 * d.K[1] + 1) * (d.K[2] + 1);
        TRY(dalloc(c, c->alloc_g, &c->w.f2, f2n * 2 * sizeof(T)));
        if (c->p.flags & BS_WANT_PSI) TRY(dalloc(c, c->alloc_g, &c->w.f2psi, f2n * 2 * sizeof(T)));
        const int ntw = d.ng[0] + d.ng[1] + d.ng[2];
        std::vector<T> tw(2 * (size_t)ntw);
        int o = 0;
        for (int ax = 0; ax < 3; ++ax)
            for (int j = 0; j < d.ng[ax]; ++j, ++o) {
                const double ph = -2.0 * kPi * j / d.ng[ax];
                tw[2 * o] = (T)cos(ph);
                tw[2 * o + 1] = (T)sin(ph);
            }
        TRY(dalloc(c, c->alloc_g, &c->w.tw, sizeof(T) * tw.size()));
        CUDA_TRY(cudaMemcpy(c->w.tw, tw.data(), sizeof(T) * tw.size(), cudaMemcpyHostToDevice));
        // positions of frequency k per axis, then the frequency at each
        // position of an x line (the inverse of the first table)
        std::vector<int> rev(ntw + d.ng[0]);
        o = 0;
        for (int ax = 0; ax < 3; ++ax)
            for (int k = 0; k < d.ng[ax]; ++k) rev[o++] = rev_pos_host(k, d.plan[ax]);
        for (int k = 0; k < d.ng[0]; ++k) rev[ntw + rev[k]] = k;
        TRY(dalloc(c, c->alloc_g, (void**)&c->w.rev, sizeof(int) * rev.size()));
        CUDA_TRY(cudaMemcpy(c->w.rev, rev.data(), sizeof(int) * rev.size(), cudaMemcpyHostToDevice));
    }
    {
        // nodes binned by target block (m x m x m cells) for the tiled short range
        long long nblk = 1;
        for (int k = 0; k < 3; ++k) nblk *= (d.nc[k] + d.m - 1) / d.m;
        TRY(dalloc(c, c->alloc_g, (void**)&c->w.tb_cnt, sizeof(int) * (size_t)(nblk + 1)));
        TRY(dalloc(c, c->alloc_g, (void**)&c->w.tb_cur, sizeof(int) * (size_t)(nblk + 1)));
    }
    TRY(dalloc(c, c->alloc_g, (void**)&c->w.cell_cnt, sizeof(int) * (size_t)(d.ncells + 1)));
    TRY(dalloc(c, c->alloc_g, (void**)&c->w.cell_cur, sizeof(int) * (size_t)(d.ncells + 1)));
    TRY(dalloc(c, c->alloc_g, (void**)&c->w.scan_tmp,
               sizeof(int) * (size_t)std::max(scan_blocks((int)d.ncells), scan_blocks(d.ncols))));
    if (d.fuse_interp) TRY(dalloc(c, c->alloc_g, (void**)&c->w.ncol_cnt, sizeof(int) * (size_t)(d.ncols + 1)));
    TRY(dalloc(c, c->alloc_g, (void**)&c->w.status, sizeof(int)));
    TRY(dalloc(c, c->alloc_g, (void**)&c->w.energy_acc, 2 * sizeof(double)));
    TRY(dalloc(c, c->alloc_g, (void**)&c->w.shell, sizeof(double) * (size_t)d.nshell));
    if (c->p.flags & BS_DETERMINISTIC) {
        const int mcx = 1 << d.lmcx;
        c->w.nepart = (2 * d.K[1] + 1) * ((d.K[2] + 1 + mcx - 1) / mcx);
        TRY(dalloc(c, c->alloc_g, (void**)&c->w.epart, sizeof(double) * (size_t)c->w.nepart));
    }
    CUDA_TRY(cudaMemset(c->w.status, 0, sizeof(int)));
    // k-space tables, m = 0..K_d: e^{-k_d^2 / 4 alpha^2} / F_d(m)^2 (deconvolved for
    // the spread and for the interpolation), then e^{-k_d^2 / 4 alpha^2} / F_d(m)
    // (the spread's deconvolution alone: the coarse-grained field on the grid)
    const int ntab = d.K[0] + d.K[1] + d.K[2] + 3;
    std::vector<T> tab(2 * (size_t)ntab);
    int o = 0;
    for (int ax = 0; ax < 3; ++ax) {
        std::vector<double> F(d.K[ax] + 1);
        kb_fourier(d.zeta, c->p.nufft_w, d.ng[ax], d.K[ax], F.data());
        for (int m = 0; m <= d.K[ax]; ++m, ++o) {
            const double k = 2.0 * kPi * m / c->p.L[ax];
            const double g = exp(-k * k / (4.0 * c->p.alpha * c->p.alpha));
            tab[o] = (T)(g / (F[m] * F[m]));
            tab[ntab + o] = (T)(g / F[m]);
        }
    }
    TRY(dalloc(c, c->alloc_g, &c->w.ktab, sizeof(T) * tab.size()));
    CUDA_TRY(cudaMemcpy(c->w.ktab, tab.data(), sizeof(T) * tab.size(), cudaMemcpyHostToDevice));
    // a copy from pageable memory may return before its DMA has landed, and
    // the kernels run on streams that do not wait for the legacy stream
    CUDA_TRY(cudaDeviceSynchronize());
    if (c->p.flags & BS_FFT_CUFFT) return make_plans<T>(c);
    return BS_OK;
}

template <typename T>
int alloc_filaments(bs_ctx* c, const std::vector<int64_t>& off, const std::vector<int>& fil_of,
                    const std::vector<int>& prev, const std::vector<double>& shift)
{
    const size_t N = (size_t)c->N, NQ = (size_t)c->NQ, nf = (size_t)c->nfil;
    Work& w = c->w;
    std::vector<std::pair<void*, size_t>>& L = c->alloc_n;
    TRY(dalloc(c, L, (void**)&w.off, sizeof(int64_t) * (nf + 1)));
    TRY(dalloc(c, L, (void**)&w.fil_of, sizeof(int) * N));
    TRY(dalloc(c, L, (void**)&w.prev, sizeof(int) * N));
    TRY(dalloc(c, L, (void**)&w.shift, sizeof(double) * 3 * nf));
    TRY(dalloc(c, L, &w.hseg, sizeof(T) * N));
    TRY(dalloc(c, L, &w.dp, sizeof(T) * 3 * N));
    TRY(dalloc(c, L, &w.ds, sizeof(T) * 3 * N));
    TRY(dalloc(c, L, &w.Mm, sizeof(T) * 3 * N));
    if (c->p.spline_order == 6) {
        TRY(dalloc(c, L, &w.Dd, sizeof(T) * 3 * N));
        // the quintic solver's scratch (18 per node), and f_j of the energy line integral
        TRY(dalloc(c, L, (void**)&w.qtmp, sizeof(double) * 19 * N));
    } else {
        w.Dd = nullptr;
        w.qtmp = nullptr;
    }
    TRY(dalloc(c, L, &w.cpr, sizeof(T) * N));
    TRY(dalloc(c, L, &w.zz, sizeof(T) * N));
    TRY(dalloc(c, L, &w.Tper, sizeof(T) * nf));
    TRY(dalloc(c, L, (void**)&w.vls, sizeof(double) * 3 * N));
    TRY(dalloc(c, L, (void**)&w.pls, sizeof(double) * 3 * N));
    TRY(dalloc(c, L, (void**)&w.vsr, sizeof(double) * 3 * N));
    TRY(dalloc(c, L, (void**)&w.psr, sizeof(double) * 3 * N));
    TRY(dalloc(c, L, (void**)&w.tb_key, sizeof(int) * N));
    TRY(dalloc(c, L, (void**)&w.tb_idx, sizeof(int) * N));
    TRY(dalloc(c, L, &w.tgt, sizeof(SrTgt<T>) * N));
    TRY(dalloc(c, L, &w.sr_rec, sizeof(SrRec<T>) * NQ));
    TRY(dalloc(c, L, &w.sr_sorted, sizeof(SrRec<T>) * NQ));
    TRY(dalloc(c, L, (void**)&w.sr_key, sizeof(int) * NQ));
    TRY(dalloc(c, L, &w.lr_rec, sizeof(LrRec<T>) * NQ));
    TRY(dalloc(c, L, &w.lr_sorted, sizeof(LrRec<T>) * NQ));
    TRY(dalloc(c, L, (void**)&w.lr_key, sizeof(int) * NQ));
    TRY(dalloc(c, L, (void**)&w.col_rec, sizeof(int2) * NQ * (size_t)c->d.colcap));
    TRY(dalloc(c, L, &w.col_pts, col_pt_bytes<T>(c->p.nufft_w) * NQ));
    if (c->d.fuse_interp) {
        TRY(dalloc(c, L, &w.nd_rec, nd_rec_bytes<T>(c->p.nufft_w) * N));
        TRY(dalloc(c, L, &w.nd_sorted, nd_rec_bytes<T>(c->p.nufft_w) * N));
        TRY(dalloc(c, L, (void**)&w.nd_key, sizeof(int) * N));
        TRY(dalloc(c, L, (void**)&w.nd_rank, sizeof(int) * N));
        TRY(dalloc(c, L, &w.vacc, sizeof(T) * 3 * N));
    }
    if (c->p.flags & BS_DETERMINISTIC) {
        TRY(dalloc(c, L, (void**)&w.sr_idx, sizeof(int) * NQ));
        TRY(dalloc(c, L, &w.sr_sorted2, sizeof(SrRec<T>) * NQ));
        TRY(dalloc(c, L, (void**)&w.col_rec2, sizeof(int2) * NQ * (size_t)c->d.colcap));
        TRY(dalloc(c, L, (void**)&w.lpart, sizeof(double) * std::max<size_t>(nf, 1)));
    }
    TRY(dalloc(c, L, (void**)&w.nodes_in, sizeof(double) * 3 * N));
    TRY(dalloc(c, L, (void**)&w.vel_out, sizeof(double) * 3 * N));
    TRY(dalloc(c, L, (void**)&w.psi_out, sizeof(double) * 3 * N));
    CUDA_TRY(cudaMemcpy(w.off, off.data(), sizeof(int64_t) * (nf + 1), cudaMemcpyHostToDevice));
    if (N) {
        CUDA_TRY(cudaMemcpy(w.fil_of, fil_of.data(), sizeof(int) * N, cudaMemcpyHostToDevice));
        CUDA_TRY(cudaMemcpy(w.prev, prev.data(), sizeof(int) * N, cudaMemcpyHostToDevice));
    }
    if (nf) CUDA_TRY(cudaMemcpy(w.shift, shift.data(), sizeof(double) * 3 * nf, cudaMemcpyHostToDevice));
    // the copies from pageable memory may return before their DMA has landed
    CUDA_TRY(cudaDeviceSynchronize());
    return BS_OK;
}

void fill_geom(const bs_ctx* c, GeomP& G)
{
    const bs_params& p = c->p;
    const Derived& d = c->d;
    memset(&G, 0, sizeof G);
    for (int k = 0; k < 3; ++k) {
        G.L[k] = p.L[k];
        G.nc[k] = d.nc[k];
        G.hc[k] = d.hc[k];
        G.ng[k] = d.ng[k];
        G.hg[k] = d.hg[k];
        G.tile[k] = d.tile[k];
        G.ntile[k] = d.ntile[k];
    }
    G.N = (int)c->N;
    G.nfil = c->nfil;
    G.Q = p.quad_Q;
    double x[kMaxQ], wq[kMaxQ];
    gauss_legendre(p.quad_Q, x, wq);
    for (int i = 0; i < p.quad_Q; ++i) {
        G.gh[i] = 0.5 * (x[i] + 1.0);
        G.gw[i] = 0.5 * wq[i];
    }
    G.kappa = p.kappa;
    G.a = p.a;
    G.log2a = std::log(2.0 / p.a);
    G.delta = p.delta;
    G.alpha = p.alpha;
    G.w = p.nufft_w;
    G.seg_max = 0.25 * std::min(p.L[0], std::min(p.L[1], p.L[2]));
    G.local_frac = p.local_frac;
    for (int k = 0; k < 3; ++k) {
        G.iL[k] = 1.0 / p.L[k];
        G.ihc[k] = 1.0 / d.hc[k];
        G.ihg[k] = 1.0 / d.hg[k];
    }
    G.want_psi = (p.flags & BS_WANT_PSI) ? 1 : 0;
}

void rec(bs_ctx* c, int i, cudaStream_t s)
{
    if (c->timed && i < bs_ctx::kStages) cudaEventRecord(c->ev_t[i], s);
}

#define CE(expr)                                                                                    \
    do {                                                                                            \
        cudaError_t _e = (expr);                                                                    \
        if (_e != cudaSuccess) return fail(BS_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(_e));   \
    } while (0)

template <typename T>
int fft_fwd(bs_ctx* c, cudaStream_t s)
{
    CUFFT_TRY(cufftSetStream(c->plan_fwd, s));
    if (sizeof(T) == 4)
        CUFFT_TRY(cufftExecR2C(c->plan_fwd, (cufftReal*)c->w.grid, (cufftComplex*)c->w.spec));
    else
        CUFFT_TRY(cufftExecD2Z(c->plan_fwd, (cufftDoubleReal*)c->w.grid, (cufftDoubleComplex*)c->w.spec));
    return BS_OK;
}

template <typename T>
int fft_inv(bs_ctx* c, void* spec, cudaStream_t s)
{
    CUFFT_TRY(cufftSetStream(c->plan_inv, s));
    if (sizeof(T) == 4)
        CUFFT_TRY(cufftExecC2R(c->plan_inv, (cufftComplex*)spec, (cufftReal*)c->w.grid));
    else
        CUFFT_TRY(cufftExecZ2D(c->plan_inv, (cufftDoubleComplex*)spec, (cufftDoubleReal*)c->w.grid));
    return BS_OK;
}

// Stage parameters of a context (shared by run() and the batched form).
void fill_interp(const bs_ctx* c, bool want_psi, InterpP& I)
{
    const bs_params& p = c->p;
    const Derived& d = c->d;
    I.N = (int)c->N;
    for (int k = 0; k < 3; ++k) {
        I.ng[k] = d.ng[k];
        I.hg[k] = d.hg[k];
        I.L[k] = p.L[k];
        I.iL[k] = 1.0 / p.L[k];
        I.ihg[k] = 1.0 / d.hg[k];
    }
    I.w = p.nufft_w;
    I.zeta = d.zeta;
    I.inorm = 1.0 / (1.0 - exp(-2.0 * d.zeta));
    I.want_psi = want_psi ? 1 : 0;
}

void fill_colp(const bs_ctx* c, ColP& CP)
{
    const Derived& d = c->d;
    CP.tx = d.tx;
    CP.ty = d.ty;
    CP.nbx = d.nbx;
    CP.nby = d.nby;
    CP.ncols = d.ncols;
    CP.w = c->p.nufft_w;
    CP.nzb = d.nzb;
    CP.n2 = d.ng[2];
    CP.zeta = d.zeta;
    CP.inorm = 1.0 / (1.0 - exp(-2.0 * d.zeta));
}

void fill_short(const bs_ctx* c, bool want_psi, ShortP& S)
{
    const bs_params& p = c->p;
    const Derived& d = c->d;
    memset(&S, 0, sizeof S);
    S.N = (int)c->N;
    for (int k = 0; k < 3; ++k) {
        S.nc[k] = d.nc[k];
        S.hc[k] = d.hc[k];
        S.L[k] = p.L[k];
    }
    S.m = d.m;
    for (int k = 0; k < 3; ++k) S.nb[k] = (d.nc[k] + d.m - 1) / d.m;
    S.kernel = (p.flags & BS_SHORT_TILED) ? 1 : ((p.flags & BS_SHORT_PER_NODE) ? 2 : 0);
    S.rc2 = p.rc * p.rc;
    S.alpha = p.alpha;
    S.pref = p.kappa / (4.0 * kPi);
    S.want_psi = want_psi ? 1 : 0;
}

template <typename T>
void fill_spzp(const bs_ctx* c, bool det, SpZP& SZ)
{
    const bs_params& p = c->p;
    const Derived& d = c->d;
    const Work& w = c->w;
    SZ.det = det ? 1 : 0;
    SZ.nthreads = d.zthreads;
    for (int k = 0; k < 3; ++k) {
        SZ.ng[k] = d.ng[k];
        SZ.K[k] = d.K[k];
    }
    SZ.tx = d.tx;
    SZ.ty = d.ty;
    SZ.nbx = d.nbx;
    SZ.nby = d.nby;
    SZ.w = p.nufft_w;
    SZ.nzb = d.nzb;
    // room for the interpolation's periodic halo of w - 1 positions
    SZ.cls = line_stride(d.ng[2] + p.nufft_w - 1, 3 * d.tx * d.ty / 2, 128 / (2 * (int)sizeof(T)));
    SZ.ls = d.lsz;
    while (SZ.ls < SZ.cls) SZ.ls += 32;  // the real region also holds the complex lines
    SZ.zeta = d.zeta;
    SZ.plan2 = d.plan[2];
    SZ.rev = w.rev + d.ng[0] + d.ng[1];
    SZ.d_nbx = make_fastdiv((unsigned)d.nbx);
    SZ.d_n2 = make_fastdiv((unsigned)d.ng[2]);
    SZ.d_nk = make_fastdiv((unsigned)(d.K[2] + 1));
    SZ.d_txy = make_fastdiv((unsigned)(d.tx * d.ty));
    SZ.d_ty = make_fastdiv((unsigned)d.ty);
    SZ.d_ncl = make_fastdiv((unsigned)(3 * d.tx * d.ty / 2));
}

template <typename T>
void fill_fftyp(const bs_ctx* c, FftYP& YP)
{
    const Derived& d = c->d;
    for (int k = 0; k < 3; ++k) {
        YP.ng[k] = d.ng[k];
        YP.K[k] = d.K[k];
    }
    YP.lmc = d.lmcy;
    YP.ls = line_stride(d.ng[1], 1 << d.lmcy, 128 / (2 * (int)sizeof(T)));
    YP.plan1 = d.plan[1];
    YP.rev = c->w.rev + d.ng[0];
    YP.d_nch = make_fastdiv((unsigned)((d.K[2] + 1 + (1 << d.lmcy) - 1) >> d.lmcy));
    YP.d_lines = make_fastdiv(1u << d.lmcy);
    // tensor-copy boxes of at most 256 rows, a multiple of 8 rows each (whole
    // 128-byte units in shared memory)
    YP.tnb = (d.ng[1] + 255) / 256;
    YP.tby = ((d.ng[1] + YP.tnb - 1) / YP.tnb + 7) & ~7;
}

// The x pass's descriptor of F2 (null: the per-element copy path).
template <typename T>
const CUtensorMap* tmap_x(bs_ctx* c, const FftXP& XP)
{
    if (c->tmx_for != c->w.f2) {
        c->tmx_ok = make_tmap_x<T>(c->w.f2, XP, &c->tmx);
        c->tmx_for = c->w.f2;
    }
    return c->tmx_ok ? &c->tmx : nullptr;
}

// The y pass's descriptor of F1 (null: the per-element copy path).
template <typename T>
const CUtensorMap* tmap_y(bs_ctx* c, const FftYP& YP)
{
    if (c->tmy_for != c->w.spec) {
        c->tmy_ok = make_tmap_y<T>(c->w.spec, YP, &c->tmy);
        c->tmy_for = c->w.spec;
    }
    return c->tmy_ok ? &c->tmy : nullptr;
}

// The x pass with the velocity's k-space pass (no energy, spectrum or psi).
template <typename T>
void fill_fftxp(const bs_ctx* c, FftXP& XP)
{
    const bs_params& p = c->p;
    const Derived& d = c->d;
    memset(&XP, 0, sizeof XP);
    for (int k = 0; k < 3; ++k) {
        XP.ng[k] = d.ng[k];
        XP.K[k] = d.K[k];
        XP.kk[k] = 2.0 * kPi / p.L[k];
    }
    XP.lmc = d.lmcx;
    XP.nthreads = d.zthreads;
    XP.ls = line_stride(d.ng[0], 3 << d.lmcx, 128 / (2 * (int)sizeof(T)));
    XP.scale = p.kappa / (p.L[0] * p.L[1] * p.L[2]);
    XP.plan0 = d.plan[0];
    XP.rev = c->w.rev;
    XP.irev = c->w.rev + d.ng[0] + d.ng[1] + d.ng[2];
    // tensor-copy boxes of at most 256 x rows, a multiple of 16 rows each
    XP.tnbx = (d.ng[0] + 255) / 256;
    XP.tbx = ((d.ng[0] + XP.tnbx - 1) / XP.tnbx + 15) & ~15;
    XP.d_nch = make_fastdiv((unsigned)((d.K[2] + 1 + (1 << d.lmcx) - 1) >> d.lmcx));
    XP.d_n0 = make_fastdiv((unsigned)d.ng[0]);
    XP.d_lines = make_fastdiv(3u << d.lmcx);
    XP.d_lines_psi = make_fastdiv(6u << d.lmcx);
    XP.dk = 2.0 * kPi / std::min(p.L[0], std::min(p.L[1], p.L[2]));
    XP.inv4a2 = 1.0 / (4.0 * p.alpha * p.alpha);
}

// The pipeline.  parts (4 x N x 3) / psi_parts switch the output to the
// separate parts of Eq. ewald_velocity_splitting.  With BS_TIMING, events
// are recorded on the stream each stage runs on (the two branches stay
// concurrent); stage i spans events [kStageBeg[i], kStageEnd[i]].
template <typename T>
int run(bs_ctx* c, const double* nodes, double* vel, double* psi, double* parts, double* psi_parts,
        bool want_energy = false, double* spectrum = nullptr, int smoothed = 0, int nbins = 0,
        double* coarse = nullptr)
{
    const bs_params& p = c->p;
    const Derived& d = c->d;
    const Work& w = c->w;
    cudaStream_t s = c->stream;
    const size_t N3 = (size_t)c->N * 3;
    const bool want_psi = (psi != nullptr) || (psi_parts != nullptr) || want_energy;
    c->timed = (p.flags & BS_TIMING) != 0;
    const bool det = (p.flags & BS_DETERMINISTIC) != 0;
    if (want_energy) CE(cudaMemsetAsync(w.energy_acc, 0, 2 * sizeof(double), s));

    GeomP G;
    fill_geom(c, G);
    G.want_psi = want_psi ? 1 : 0;

    InterpP I;
    fill_interp(c, want_psi, I);
    ColP CP;
    fill_colp(c, CP);
    const bool fused = d.fuse_interp && !spectrum && !coarse;

    rec(c, 0, s);
    CE(launch_spline<T>(nodes, w, c->nfil, s));
    CE(launch_nodes<T>(G, nodes, w, parts ? parts : nullptr, parts ? parts + 3 * N3 : nullptr,
                       psi_parts ? psi_parts : nullptr, psi_parts ? psi_parts + 3 * N3 : nullptr, s));
    rec(c, 1, s);

    // short range on the side stream (not for the spectrum or the grid field)
    if (!spectrum && !coarse) {
    CE(cudaEventRecord(c->ev_fork, s));
    CE(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    cudaStream_t ss = c->side;
    CE(launch_sort_sr<T>(w, (int)c->NQ, (int)d.ncells, ss, det));
    rec(c, 2, ss);
    ShortP S;
    fill_short(c, want_psi, S);
    CE(launch_short<T>(S, w, ss));
    rec(c, 3, ss);
    if (fused) CE(launch_node_bin<T>(CP, I, nodes, w, ss));
    CE(cudaEventRecord(c->ev_join, ss));
    }

    // long range on the main stream
    if (p.flags & BS_FFT_CUFFT) {
        CE(launch_sort_lr<T>(w, (int)c->NQ, d.ntiles, s));
        rec(c, 4, s);
        SpreadP SP;
        for (int k = 0; k < 3; ++k) {
            SP.ng[k] = d.ng[k];
            SP.tile[k] = d.tile[k];
            SP.ntile[k] = d.ntile[k];
        }
        SP.w = p.nufft_w;
        SP.zeta = d.zeta;
        SP.inorm = 1.0 / (1.0 - exp(-2.0 * d.zeta));
        CE(launch_spread<T>(SP, w, d.ntiles, s));
        rec(c, 5, s);
        TRY(fft_fwd<T>(c, s));
        rec(c, 6, s);
        KspaceP K;
        for (int k = 0; k < 3; ++k) {
            K.ng[k] = d.ng[k];
            K.K[k] = d.K[k];
            K.kk[k] = 2.0 * kPi / p.L[k];
        }
        K.nh = d.nh;
        K.scale = p.kappa / (p.L[0] * p.L[1] * p.L[2]);
        K.want_psi = want_psi ? 1 : 0;
        K.energy = want_energy ? w.energy_acc : nullptr;
        CE(launch_kspace<T>(K, w, s));
        rec(c, 7, s);
        TRY(fft_inv<T>(c, w.spec, s));
        rec(c, 8, s);
    } else {
        CE(launch_col_sort<T>(CP, w, (int)c->NQ, s, det));
        rec(c, 4, s);
        SpZP SZ;
        fill_spzp<T>(c, det, SZ);
        CE(launch_spread_zfft<T>(SZ, w, s));
        rec(c, 5, s);
        FftYP YP;
        fill_fftyp<T>(c, YP);
        CE(launch_fft_y<T>(YP, w, w.f2, -1, s, tmap_y<T>(c, YP)));
        rec(c, 6, s);
        FftXP XP;
        fill_fftxp<T>(c, XP);
        XP.epart = (want_energy && det) ? w.epart : nullptr;
        XP.energy = want_energy ? w.energy_acc : nullptr;
        XP.spectrum = spectrum;
        XP.nbins = nbins;
        XP.smoothed = smoothed;
        XP.single_decon = coarse ? 1 : 0;
        if (spectrum) return (int)launch_fft_x_kspace<T>(XP, w, false, s) == (int)cudaSuccess
                                 ? BS_OK
                                 : fail(BS_ERR_CUDA, "spectrum kernel launch failed");
        CE(launch_fft_x_kspace<T>(XP, w, want_psi, s, tmap_x<T>(c, XP)));
        rec(c, 7, s);
        CE(launch_fft_y<T>(YP, w, w.f2, +1, s, tmap_y<T>(c, YP)));
        if (fused) {
            rec(c, 8, s);
            CE(cudaStreamWaitEvent(s, c->ev_join, 0));
            rec(c, 9, s);
            CE(launch_zfft_interp<T>(SZ, w, s));
        } else {
        FftZP ZP;
        for (int k = 0; k < 3; ++k) {
            ZP.ng[k] = d.ng[k];
            ZP.K[k] = d.K[k];
        }
        ZP.yc = d.yc;
        ZP.cls = line_stride(d.ng[2], d.yc / 2, 128 / (2 * (int)sizeof(T)));
        ZP.plan2 = d.plan[2];
            ZP.rev = w.rev + d.ng[0] + d.ng[1];
        ZP.d_nch = make_fastdiv((unsigned)(d.ng[1] / d.yc));
        ZP.d_n0 = make_fastdiv((unsigned)d.ng[0]);
        ZP.d_nk = make_fastdiv((unsigned)(d.K[2] + 1));
        ZP.d_n2 = make_fastdiv((unsigned)d.ng[2]);
        ZP.d_ncl = make_fastdiv((unsigned)(d.yc / 2));
        if (coarse) {  // the coarse-grained field on the grid, written straight in float64; no interpolation
            CE(launch_fft_z_c2r<T>(ZP, w, s, coarse));
            return BS_OK;
        }
        CE(launch_fft_z_c2r<T>(ZP, w, s));
        rec(c, 8, s);
        }
    }
    if (!fused) {
        CE(cudaStreamWaitEvent(s, c->ev_join, 0));
        rec(c, 9, s);
    }
    if (want_energy) CE(launch_energy_line<T>(nodes, w, c->nfil, w.nmax_fil, s, det));

    if (fused) {
        CE(launch_interp_sum<T>((int)c->N, w, parts ? 2 : 0, vel, parts ? parts + 2 * N3 : nullptr, s));
        if (parts) CE(cudaMemcpyAsync(parts + N3, w.vsr, sizeof(double) * N3, cudaMemcpyDeviceToDevice, s));
    } else if (parts) {
        CE(launch_interp<T>(I, nodes, w, w.grid, 2, nullptr, parts + 2 * N3, s));
        CE(cudaMemcpyAsync(parts + N3, w.vsr, sizeof(double) * N3, cudaMemcpyDeviceToDevice, s));
    } else {
        CE(launch_interp<T>(I, nodes, w, w.grid, 0, vel, nullptr, s));
    }
    if (want_psi) {
        if (p.flags & BS_FFT_CUFFT) {
            TRY(fft_inv<T>(c, w.spec_psi, s));
        } else {
            FftYP YP;
            fill_fftyp<T>(c, YP);
            CE(launch_fft_y<T>(YP, w, w.f2psi, +1, s, tmap_y<T>(c, YP)));
            FftZP ZP;
            for (int k = 0; k < 3; ++k) {
                ZP.ng[k] = d.ng[k];
                ZP.K[k] = d.K[k];
            }
            ZP.yc = d.yc;
            ZP.cls = line_stride(d.ng[2], d.yc / 2, 128 / (2 * (int)sizeof(T)));
            ZP.plan2 = d.plan[2];
            ZP.rev = w.rev + d.ng[0] + d.ng[1];
            ZP.d_nch = make_fastdiv((unsigned)(d.ng[1] / d.yc));
            ZP.d_n0 = make_fastdiv((unsigned)d.ng[0]);
            ZP.d_nk = make_fastdiv((unsigned)(d.K[2] + 1));
            ZP.d_n2 = make_fastdiv((unsigned)d.ng[2]);
            ZP.d_ncl = make_fastdiv((unsigned)(d.yc / 2));
            CE(launch_fft_z_c2r<T>(ZP, w, s));
        }
        if (psi_parts) {
            CE(launch_interp<T>(I, nodes, w, w.grid, 2, nullptr, psi_parts + 2 * N3, s));
            CE(cudaMemcpyAsync(psi_parts + N3, w.psr, sizeof(double) * N3, cudaMemcpyDeviceToDevice, s));
        } else {
            CE(launch_interp<T>(I, nodes, w, w.grid, 1, psi, nullptr, s));
        }
    }
    rec(c, 10, s);
    return BS_OK;
}

int check_ctx(bs_ctx* c)
{
    if (!c) return fail(BS_ERR_ARG, "null context");
    if (!c->have_fil) return fail(BS_ERR_STATE, "bs_set_filaments has not been called");
    CUDA_TRY(cudaSetDevice(c->device));
    return BS_OK;
}


void rk4_drop_graph(bs_ctx* c)
{
    if (c->rk_exec) cudaGraphExecDestroy(c->rk_exec);
    if (c->rk_graph) cudaGraphDestroy(c->rk_graph);
    c->rk_exec = nullptr;
    c->rk_graph = nullptr;
}

int rk4_alloc(bs_ctx* c)
{
    if (!c->rk) TRY(dalloc(c, c->alloc_n, (void**)&c->rk, sizeof(double) * 15 * (size_t)c->N));
    return BS_OK;
}

// One RK4 step of the nodes in place: four evaluations on the stage
// positions, then the weighted update (Sec. 5.2).
int rk4_issue(bs_ctx* c, double* nodes, double dt)
{
    const long long n3 = 3 * (long long)c->N;
    double* k[4] = { c->rk, c->rk + n3, c->rk + 2 * n3, c->rk + 3 * n3 };
    double* xs = c->rk + 4 * n3;
    const double cs[3] = { 0.5 * dt, 0.5 * dt, dt };
    const double* x = nodes;
    for (int st = 0; st < 4; ++st) {
        const int rc = c->p.precision == BS_FP64 ? run<double>(c, x, k[st], nullptr, nullptr, nullptr)
                                                 : run<float>(c, x, k[st], nullptr, nullptr, nullptr);
        if (rc != BS_OK) return rc;
        if (st < 3) {
            CE(launch_rk4_stage(nodes, k[st], cs[st], xs, n3, c->stream));
            x = xs;
        }
    }
    CE(launch_rk4_final(nodes, k[0], k[1], k[2], k[3], dt, n3, c->stream));
    return BS_OK;
}

}  // namespace

extern "C" {

const char* bs_last_error(void) { return g_err.c_str(); }

int bs_params_from_beta(double beta, const double L[3], int M, long long N, bs_params* out)
{
    if (!out || !L) return fail(BS_ERR_ARG, "null argument");
    if (!(beta > 0)) return fail(BS_ERR_ARG, "beta must be positive");
    for (int c = 0; c < 3; ++c)
        if (!(L[c] > 0)) return fail(BS_ERR_ARG, "L must be positive");
    if (M <= 0 && N <= 0) return fail(BS_ERR_ARG, "need M > 0 or N > 0");
    // Table tab:performance: beta, C_beta, w (sigma = 1.5)
    static const double tb[7][3] = { { 2.0, 2.06, 4 }, { 2.5, 1.92, 6 }, { 3.5, 1.71, 8 }, { 4.0, 1.64, 10 },
                                     { 4.5, 1.57, 12 }, { 5.0, 1.52, 14 }, { 5.5, 1.47, 16 } };
    memset(out, 0, sizeof *out);
    const double Lmin = std::min(L[0], std::min(L[1], L[2]));
    int best = 0;
    for (int i = 1; i < 7; ++i)
        if (fabs(tb[i][0] - beta) < fabs(tb[best][0] - beta)) best = i;
    double Cb;
    if (beta < tb[0][0] || beta > tb[6][0]) {
        Cb = 2.6 * pow(beta, -1.0 / 3.0);  // empirical fit of Sec. 5.3
    } else {
        int i = 0;
        while (i < 5 && beta > tb[i + 1][0]) ++i;
        const double t = (beta - tb[i][0]) / (tb[i + 1][0] - tb[i][0]);
        Cb = tb[i][1] + t * (tb[i + 1][1] - tb[i][1]);
    }
    int Mv = M;
    if (M <= 0) {
        double alpha = Cb * cbrt((double)N) / Lmin;          // Eq. alpha_optimal_performance
        alpha = std::max(alpha, 2.0 * beta / Lmin);          // keeps rc <= L/2
        const int K = (int)ceil(beta * alpha * Lmin / kPi);  // k_max = 2 beta alpha
        Mv = 2 * K + 1;
    }
    const int K = (Mv - 1) / 2;
    const double kmax = 2.0 * kPi * K / Lmin;
    out->alpha = kmax / (2.0 * beta);
    out->rc = beta / out->alpha;
    for (int c = 0; c < 3; ++c) {
        out->L[c] = L[c];
        // the same k_max on every axis: K_c = floor(K L_c / min L)
        out->M[c] = (L[c] == Lmin) ? Mv : 2 * (int)floor(K * L[c] / Lmin + 1e-9) + 1;
    }
    out->kappa = 1.0;
    out->a = 1e-8;
    out->delta = 0.25;
    out->quad_Q = 3;
    out->spline_order = 4;
    out->nufft_sigma = 1.5;
    out->nufft_w = (int)tb[best][2];
    out->precision = BS_FP64;
    out->flags = 0;
    out->cell_div = 0;
    out->local_frac = 0.0;
    out->block_x = out->block_y = out->block_threads = 0;
    return BS_OK;
}

int bs_error_estimate(const bs_params* p, double total_length, double* eps_v, double* eps_psi)
{
    if (!p || !(total_length >= 0)) return fail(BS_ERR_ARG, "bad argument");
    const double V = p->L[0] * p->L[1] * p->L[2];
    const double beta = p->alpha * p->rc;
    const double k = p->kappa, a = p->alpha, Lt = total_length;
    const double g = sqrt(Lt / (8.0 * kPi * V));
    if (eps_v) *eps_v = k * (Lt / (sqrt(kPi) * a * V) + g / beta) * exp(-beta * beta);
    if (eps_psi) *eps_psi = k / (2.0 * a) * (Lt / (a * V) + g / sqrt(beta)) * exp(-beta * beta) / pow(beta, 1.5);
    return BS_OK;
}

int bs_nufft_setup(const bs_params* p, int n_g[3], double* table)
{
    if (!p || !n_g) return fail(BS_ERR_ARG, "null argument");
    Derived d;
    TRY(derive(p, &d));
    int o = 0;
    for (int c = 0; c < 3; ++c) {
        n_g[c] = d.ng[c];
        if (table) {
            kb_fourier(d.zeta, p->nufft_w, d.ng[c], d.K[c], table + o);
            o += d.K[c] + 1;
        }
    }
    return BS_OK;
}

int bs_create(bs_ctx** out, const bs_params* p, void* stream)
{
    if (!out || !p) return fail(BS_ERR_ARG, "null argument");
    *out = nullptr;
    bs_ctx* c = new bs_ctx();
    c->p = *p;
    int rc = derive(p, &c->d);
    if (rc != BS_OK) {
        delete c;
        return rc;
    }
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = set_fft_constants();
    // the short-range branch runs at the highest stream priority: its few
    // CTAs are dispatched ahead of the long-range kernels' waiting ones, so
    // the branch ends while the spread is still running
    int prio_lo = 0, prio_hi = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    for (int i = 0; i < bs_ctx::kStages && e == cudaSuccess; ++i) e = cudaEventCreate(&c->ev_t[i]);
    if (e != cudaSuccess) {
        rc = fail(BS_ERR_CUDA, "CUDA set-up failed: %s", cudaGetErrorString(e));
        bs_destroy(c);
        return rc;
    }
    c->stream = (cudaStream_t)stream;
    rc = (p->precision == BS_FP64) ? alloc_grids<double>(c) : alloc_grids<float>(c);
    if (rc != BS_OK) {
        std::string msg = g_err;
        bs_destroy(c);
        g_err = msg;
        return rc;
    }
    *out = c;
    return BS_OK;
}

int bs_set_stream(bs_ctx* c, void* stream)
{
    if (!c) return fail(BS_ERR_ARG, "null context");
    c->stream = (cudaStream_t)stream;
    return BS_OK;
}

int bs_set_filaments(bs_ctx* c, int nfil, const int64_t* offsets, const int32_t* closing)
{
    if (!c) return fail(BS_ERR_ARG, "null context");
    if (nfil < 0 || (nfil > 0 && !offsets)) return fail(BS_ERR_ARG, "bad filament count or offsets");
    std::vector<int64_t> off(nfil + 1, 0);
    if (nfil > 0) {
        if (offsets[0] != 0) return fail(BS_ERR_ARG, "offsets[0] must be 0");
        for (int l = 0; l <= nfil; ++l) off[l] = offsets[l];
    }
    long long sumn[3] = { 0, 0, 0 };
    for (int l = 0; l < nfil; ++l) {
        const int64_t n = off[l + 1] - off[l];
        if (n < c->p.spline_order)
            return fail(BS_ERR_SPLINE, "filament %d has %lld nodes < spline order %d", l, (long long)n,
                        c->p.spline_order);
        if (closing)
            for (int k = 0; k < 3; ++k) sumn[k] += closing[3 * l + k];
    }
    if (sumn[0] || sumn[1] || sumn[2])
        return fail(BS_ERR_NET_VORTICITY, "sum of closing offsets is (%lld,%lld,%lld), must be 0", sumn[0], sumn[1],
                    sumn[2]);
    const long long N = off[nfil];
    if (N * c->p.quad_Q > (1LL << 31) - 1) return fail(BS_ERR_ARG, "too many quadrature points");
    CUDA_TRY(cudaSetDevice(c->device));
    CUDA_TRY(cudaDeviceSynchronize());
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    if (c->graph) {
        cudaGraphDestroy(c->graph);
        c->graph = nullptr;
    }
    rk4_drop_graph(c);
    free_list(c, c->alloc_n);  // drop the buffers of a previous topology
    c->w.off = nullptr;
    c->rk = nullptr;
    std::vector<int> fil_of((size_t)N), prev((size_t)N);
    std::vector<double> shift(3 * (size_t)nfil, 0.0);
    for (int l = 0; l < nfil; ++l) {
        for (int64_t j = off[l]; j < off[l + 1]; ++j) {
            fil_of[(size_t)j] = l;
            prev[(size_t)j] = (int)(j == off[l] ? off[l + 1] - 1 : j - 1);
        }
        if (closing)
            for (int k = 0; k < 3; ++k) shift[3 * l + k] = closing[3 * l + k] * c->p.L[k];
    }
    c->nfil = nfil;
    c->N = N;
    c->w.nmax_fil = 0;
    for (int l = 0; l < nfil; ++l) c->w.nmax_fil = std::max(c->w.nmax_fil, (int)(off[l + 1] - off[l]));
    c->NQ = N * c->p.quad_Q;
    c->have_fil = false;
    int rc = (c->p.precision == BS_FP64) ? alloc_filaments<double>(c, off, fil_of, prev, shift)
                                         : alloc_filaments<float>(c, off, fil_of, prev, shift);
    if (rc != BS_OK) return rc;
    c->have_fil = true;
    return BS_OK;
}

int bs_compute(bs_ctx* c, const double* nodes, double* vel, double* psi)
{
    TRY(check_ctx(c));
    if (c->N == 0) return BS_OK;
    if (!nodes || !vel) return fail(BS_ERR_ARG, "null nodes or vel");
    if (psi && !(c->p.flags & BS_WANT_PSI)) return fail(BS_ERR_ARG, "psi requested without BS_WANT_PSI");
    return c->p.precision == BS_FP64 ? run<double>(c, nodes, vel, psi, nullptr, nullptr)
                                     : run<float>(c, nodes, vel, psi, nullptr, nullptr);
}

int bs_compute_host(bs_ctx* c, const double* nodes, double* vel, double* psi)
{
    TRY(check_ctx(c));
    if (c->N == 0) return BS_OK;
    if (!nodes || !vel) return fail(BS_ERR_ARG, "null nodes or vel");
    if (psi && !(c->p.flags & BS_WANT_PSI)) return fail(BS_ERR_ARG, "psi requested without BS_WANT_PSI");
    const size_t bytes = sizeof(double) * 3 * (size_t)c->N;
    CUDA_TRY(cudaMemcpyAsync(c->w.nodes_in, nodes, bytes, cudaMemcpyHostToDevice, c->stream));
    int rc = c->p.precision == BS_FP64
                 ? run<double>(c, c->w.nodes_in, c->w.vel_out, psi ? c->w.psi_out : nullptr, nullptr, nullptr)
                 : run<float>(c, c->w.nodes_in, c->w.vel_out, psi ? c->w.psi_out : nullptr, nullptr, nullptr);
    if (rc != BS_OK) return rc;
    CUDA_TRY(cudaMemcpyAsync(vel, c->w.vel_out, bytes, cudaMemcpyDeviceToHost, c->stream));
    if (psi) CUDA_TRY(cudaMemcpyAsync(psi, c->w.psi_out, bytes, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return BS_OK;
}

int bs_compute_parts(bs_ctx* c, const double* nodes, double* parts, double* psi_parts)
{
    TRY(check_ctx(c));
    if (c->N == 0) return BS_OK;
    if (!nodes || !parts) return fail(BS_ERR_ARG, "null nodes or parts");
    if (psi_parts && !(c->p.flags & BS_WANT_PSI)) return fail(BS_ERR_ARG, "psi requested without BS_WANT_PSI");
    return c->p.precision == BS_FP64 ? run<double>(c, nodes, nullptr, nullptr, parts, psi_parts)
                                     : run<float>(c, nodes, nullptr, nullptr, parts, psi_parts);
}

int bs_compute_energy(bs_ctx* c, const double* nodes, double* vel, double* psi, double* energy)
{
    TRY(check_ctx(c));
    if (!energy) return fail(BS_ERR_ARG, "null energy");
    *energy = 0.0;
    if (c->N == 0) return BS_OK;
    if (!nodes) return fail(BS_ERR_ARG, "null nodes");
    if (!(c->p.flags & BS_WANT_PSI)) return fail(BS_ERR_ARG, "the energy needs a context created with BS_WANT_PSI");
    if (c->p.spline_order == 4 && 5 * (size_t)c->w.nmax_fil * sizeof(double) > 200 * 1024)
        return fail(BS_ERR_ARG, "filament too long for the energy integral (%d nodes > 5120)", c->w.nmax_fil);
    double* v = vel ? vel : c->w.vel_out;
    double* ps = psi ? psi : c->w.psi_out;
    int rc = c->p.precision == BS_FP64 ? run<double>(c, nodes, v, ps, nullptr, nullptr, true)
                                       : run<float>(c, nodes, v, ps, nullptr, nullptr, true);
    if (rc != BS_OK) return rc;
    double acc[2];
    if (c->p.flags & BS_DETERMINISTIC) {
        // partial sums (per k-space CTA, per filament) added in a fixed order
        std::vector<double> ep((size_t)c->w.nepart), lp((size_t)c->nfil);
        CUDA_TRY(cudaMemcpyAsync(ep.data(), c->w.epart, sizeof(double) * ep.size(), cudaMemcpyDeviceToHost,
                                 c->stream));
        CUDA_TRY(cudaMemcpyAsync(lp.data(), c->w.lpart, sizeof(double) * lp.size(), cudaMemcpyDeviceToHost,
                                 c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        acc[0] = acc[1] = 0.0;
        for (double v : ep) acc[0] += v;
        for (double v : lp) acc[1] += v;
    } else {
        CUDA_TRY(cudaMemcpyAsync(acc, c->w.energy_acc, sizeof acc, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    const double V = c->p.L[0] * c->p.L[1] * c->p.L[2];
    *energy = acc[0] + c->p.kappa / (2.0 * V) * acc[1];
    return BS_OK;
}

int bs_energy_spectrum(bs_ctx* c, const double* nodes, int smoothed, int nbins, double* Ek, double* dk_out)
{
    TRY(check_ctx(c));
    if (!Ek || nbins <= 0) return fail(BS_ERR_ARG, "bad spectrum output");
    if (c->p.flags & BS_FFT_CUFFT) return fail(BS_ERR_STATE, "the spectrum needs the pruned transform path");
    const double dk = 2.0 * kPi / std::min(c->p.L[0], std::min(c->p.L[1], c->p.L[2]));
    if (dk_out) *dk_out = dk;
    for (int m = 0; m < nbins; ++m) Ek[m] = 0.0;
    if (c->N == 0) return BS_OK;
    if (!nodes) return fail(BS_ERR_ARG, "null nodes");
    // shells beyond the mode cube's corner stay zero
    const int nb = std::min(nbins, c->d.nshell);
    double* bins = c->w.shell;
    CUDA_TRY(cudaMemsetAsync(bins, 0, sizeof(double) * (size_t)nb, c->stream));
    const int rc = c->p.precision == BS_FP64
                       ? run<double>(c, nodes, nullptr, nullptr, nullptr, nullptr, false, bins, smoothed, nb)
                       : run<float>(c, nodes, nullptr, nullptr, nullptr, nullptr, false, bins, smoothed, nb);
    if (rc != BS_OK) return rc;
    CUDA_TRY(cudaMemcpyAsync(Ek, bins, sizeof(double) * (size_t)nb, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    const double sc = c->p.kappa / (c->p.L[0] * c->p.L[1] * c->p.L[2]);
    for (int m = 0; m < nb; ++m) Ek[m] *= sc * sc / (2.0 * dk);
    return BS_OK;
}

int bs_coarse_velocity(bs_ctx* c, const double* nodes, double* grid, int n_g[3])
{
    TRY(check_ctx(c));
    if (c->p.flags & BS_FFT_CUFFT) return fail(BS_ERR_STATE, "the grid field needs the pruned transform path");
    if (n_g)
        for (int k = 0; k < 3; ++k) n_g[k] = c->d.ng[k];
    if (!grid) return BS_OK;  // size query
    const double ng3 = (double)c->d.ng[0] * c->d.ng[1] * c->d.ng[2];
    if (3.0 * ng3 > 2147483647.0) return fail(BS_ERR_ARG, "grid too large for the copy-out");
    if (c->N == 0) {
        CUDA_TRY(cudaMemsetAsync(grid, 0, sizeof(double) * 3 * (size_t)ng3, c->stream));
        return BS_OK;
    }
    if (!nodes) return fail(BS_ERR_ARG, "null nodes");
    return c->p.precision == BS_FP64
               ? run<double>(c, nodes, nullptr, nullptr, nullptr, nullptr, false, nullptr, 0, 0, grid)
               : run<float>(c, nodes, nullptr, nullptr, nullptr, nullptr, false, nullptr, 0, 0, grid);
}

int bs_get_quadrature(bs_ctx* c, const double* nodes, double* qX, double* qq)
{
    TRY(check_ctx(c));
    if (c->N == 0) return BS_OK;
    if (!nodes || !qX || !qq) return fail(BS_ERR_ARG, "null argument");
    GeomP G;
    fill_geom(c, G);
    if (c->p.precision == BS_FP64) {
        CE(launch_spline<double>(nodes, c->w, c->nfil, c->stream));
        CE(launch_export_quadrature<double>(G, nodes, c->w, qX, qq, c->stream));
    } else {
        CE(launch_spline<float>(nodes, c->w, c->nfil, c->stream));
        CE(launch_export_quadrature<float>(G, nodes, c->w, qX, qq, c->stream));
    }
    return BS_OK;
}

int bs_graph_capture(bs_ctx* c, const double* nodes, double* vel, double* psi)
{
    TRY(check_ctx(c));
    if (!c->stream) return fail(BS_ERR_ARG, "graph capture needs a non-default stream");
    if (!nodes || !vel) return fail(BS_ERR_ARG, "null nodes or vel");
    if (psi && !(c->p.flags & BS_WANT_PSI)) return fail(BS_ERR_ARG, "psi requested without BS_WANT_PSI");
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    if (c->graph) {
        cudaGraphDestroy(c->graph);
        c->graph = nullptr;
    }
    if (c->N == 0) return BS_OK;
    CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = c->p.precision == BS_FP64 ? run<double>(c, nodes, vel, psi, nullptr, nullptr)
                                       : run<float>(c, nodes, vel, psi, nullptr, nullptr);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (rc != BS_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(BS_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
    c->graph = g;
    CUDA_TRY(cudaGraphInstantiate(&c->gexec, c->graph, cudaGraphInstantiateFlagUseNodePriority));
    return BS_OK;
}

int bs_graph_launch(bs_ctx* c)
{
    TRY(check_ctx(c));
    if (c->N == 0) return BS_OK;
    if (!c->gexec) return fail(BS_ERR_STATE, "no captured graph (call bs_graph_capture first)");
    CUDA_TRY(cudaGraphLaunch(c->gexec, c->stream));
    return BS_OK;
}

int bs_rk4_step(bs_ctx* c, double* nodes, double dt)
{
    TRY(check_ctx(c));
    if (c->N == 0) return BS_OK;
    if (!nodes) return fail(BS_ERR_ARG, "null nodes");
    if (!(dt > 0.0) || !isfinite(dt)) return fail(BS_ERR_ARG, "dt must be positive and finite");
    TRY(rk4_alloc(c));
    return rk4_issue(c, nodes, dt);
}

int bs_rk4_capture(bs_ctx* c, double* nodes, double dt)
{
    TRY(check_ctx(c));
    if (!c->stream) return fail(BS_ERR_ARG, "graph capture needs a non-default stream");
    if (!nodes) return fail(BS_ERR_ARG, "null nodes");
    if (!(dt > 0.0) || !isfinite(dt)) return fail(BS_ERR_ARG, "dt must be positive and finite");
    rk4_drop_graph(c);
    if (c->N == 0) return BS_OK;
    TRY(rk4_alloc(c));
    CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = rk4_issue(c, nodes, dt);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (rc != BS_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(BS_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
    c->rk_graph = g;
    CUDA_TRY(cudaGraphInstantiate(&c->rk_exec, c->rk_graph, cudaGraphInstantiateFlagUseNodePriority));
    return BS_OK;
}

int bs_rk4_launch(bs_ctx* c, int nsteps)
{
    TRY(check_ctx(c));
    if (nsteps < 0) return fail(BS_ERR_ARG, "negative step count");
    if (c->N == 0 || nsteps == 0) return BS_OK;
    if (!c->rk_exec) return fail(BS_ERR_STATE, "no captured RK4 step (call bs_rk4_capture first)");
    for (int i = 0; i < nsteps; ++i) CUDA_TRY(cudaGraphLaunch(c->rk_exec, c->stream));
    return BS_OK;
}

int bs_status(bs_ctx* c)
{
    if (!c) return fail(BS_ERR_ARG, "null context");
    CUDA_TRY(cudaSetDevice(c->device));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->side));
    int st = 0;
    if (c->w.status) {
        CUDA_TRY(cudaMemcpy(&st, c->w.status, sizeof(int), cudaMemcpyDeviceToHost));
        // cleared on the context's stream, before any later evaluation on it
        CUDA_TRY(cudaMemsetAsync(c->w.status, 0, sizeof(int), c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    if (st & ST_NONFINITE) return fail(BS_ERR_NONFINITE, "non-finite node position");
    if (st & ST_GEOMETRY) return fail(BS_ERR_GEOMETRY, "a segment is longer than min(L)/4");
    if (st & ST_TIMEOUT) return fail(BS_ERR_TIMEOUT, "a tensor copy did not complete within its wait limit");
    return BS_OK;
}

int bs_stage_times(bs_ctx* c, float* ms, int n, int* n_out)
{
    if (!c || !ms) return fail(BS_ERR_ARG, "null argument");
    if (!(c->p.flags & BS_TIMING)) return fail(BS_ERR_STATE, "context created without BS_TIMING");
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->side));
    // geometry, sr sort, short range, lr sort, spread, fft fwd, k-space,
    // fft inv, interpolation + sum, whole evaluation
    static const int beg[10] = { 0, 1, 2, 1, 4, 5, 6, 7, 9, 0 };
    static const int end[10] = { 1, 2, 3, 4, 5, 6, 7, 8, 10, 10 };
    const int ns = 10;
    for (int i = 0; i < ns && i < n; ++i) {
        float t = 0;
        CUDA_TRY(cudaEventElapsedTime(&t, c->ev_t[beg[i]], c->ev_t[end[i]]));
        ms[i] = t;
    }
    if (n_out) *n_out = ns;
    return BS_OK;
}

int bs_workspace_bytes(bs_ctx* c, long long* bytes)
{
    if (!c || !bytes) return fail(BS_ERR_ARG, "null argument");
    *bytes = c->bytes;
    return BS_OK;
}

void bs_destroy(bs_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);  // NULL: the legacy stream
    if (c->side) cudaStreamSynchronize(c->side);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    rk4_drop_graph(c);
    if (c->plans) {
        if (c->plan_fwd) cufftDestroy(c->plan_fwd);
        if (c->plan_inv) cufftDestroy(c->plan_inv);
    }
    free_list(c, c->alloc_n);
    free_list(c, c->alloc_g);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    for (int i = 0; i < bs_ctx::kStages; ++i)
        if (c->ev_t[i]) cudaEventDestroy(c->ev_t[i]);
    if (c->side) cudaStreamDestroy(c->side);
    delete c;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of independent configurations.  Member i is a full context with
// its own grid sizes.  Small members share one launch per stage (the staged
// group: each stage's CTAs look up their member in a table); the others are
// issued one by one on a pool of streams (largest first, round-robin).  Both
// run concurrently and are captured together into one CUDA graph, so the
// whole batch costs one graph launch.
// ---------------------------------------------------------------------------

// Members up to this many nodes join the staged group by default.  Measured
// on GB300 (mixed form, float32 kernels), staged against issued one by one:
// 32 members of ~300 nodes 0.35 against 0.66 ms, 128 of ~300 1.13 against
// 2.41 ms, 32 of ~1e3 0.94 against 1.08 ms, 128 of ~1e3 3.49 against 3.93 ms;
// but 64 members of ~4e3 nodes 5.6 against 5.0 ms and 64 of 1e4..3e4 18.4
// against 16.1 ms: a stage ends only when its slowest member does, where
// separate members overlap their stages and kernel types.
constexpr int64_t kStageMaxNodes = 2048;

struct bs_batch {
    int nconf = 0;
    // the staged group: the members' descriptors and block starts in one
    // device arena, bound to the node and velocity buffers it was built for
    std::vector<char> grouped;  // member i is in the staged group
    int ngrouped = 0;
    std::vector<int> mode;      // per member: 0 size rule, BS_BATCH_PER_MEMBER, BS_BATCH_STAGED
    void* arena = nullptr;
    size_t arena_bytes = 0;
    const double* a_nodes = nullptr;
    double* a_vel = nullptr;
    std::vector<BatchL> stages;
    std::vector<bs_ctx*> ctx;
    std::vector<int64_t> node_off;  // nconf + 1, member i owns nodes [node_off[i], node_off[i+1])
    std::vector<int> order;         // issue order, largest member first
    cudaStream_t stream = nullptr;  // caller's stream
    std::vector<cudaStream_t> pool;
    std::vector<cudaEvent_t> ev_done;
    cudaEvent_t ev_start = nullptr;
    cudaStream_t gmain = nullptr;  // the staged group's long range
    cudaStream_t side = nullptr;   // the staged group's short range
    cudaEvent_t ev_side = nullptr;
    cudaEvent_t ev_group = nullptr;
    int device = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const double* g_nodes = nullptr;
    double* g_vel = nullptr;
};

namespace {

void batch_drop_graph(bs_batch* b)
{
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    b->g_nodes = nullptr;
    b->g_vel = nullptr;
}

// Drops the staged launches' descriptors (the members changed).
void batch_drop_stages(bs_batch* b)
{
    if (b->arena) cudaFree(b->arena);
    b->arena = nullptr;
    b->arena_bytes = 0;
    b->a_nodes = nullptr;
    b->a_vel = nullptr;
    b->stages.clear();
}

// Host image of the batched launches' device arena: descriptor arrays and
// block starts, 256-byte aligned; BatchL pointers are offsets until upload.
struct Arena {
    std::vector<unsigned char> bytes;
    size_t put(const void* p, size_t n)
    {
        const size_t o = (bytes.size() + 255) & ~(size_t)255;
        bytes.resize(o + n);
        memcpy(bytes.data() + o, p, n);
        return o;
    }
};

// One stage: a descriptor per member and its CTA count.
template <typename D>
BatchL stage(Arena& A, const std::vector<D>& desc, const std::vector<int>& blocks, int threads, size_t smem)
{
    std::vector<int> bs(desc.size() + 1, 0);
    for (size_t m = 0; m < desc.size(); ++m) bs[m + 1] = bs[m] + blocks[m];
    BatchL L;
    L.desc = (const void*)A.put(desc.data(), sizeof(D) * desc.size());
    L.bstart = (const int*)A.put(bs.data(), sizeof(int) * bs.size());
    L.n = (int)desc.size();
    L.total = bs.back();
    L.threads = threads;
    L.smem = smem;
    return L;
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// Address of complex element k of a T-complex array.
template <typename T>
const void* cx_at(const void* p, size_t k)
{
    return (const unsigned char*)p + k * 2 * sizeof(T);
}

// Whether a member can take the batched stage launches: the plain velocity
// path (fused interpolation, cubic curves on the warp spline, no psi, cuFFT
// or deterministic mode, the warp-per-node short range).
bool batch_stageable(const bs_ctx* c)
{
    const bs_params& p = c->p;
    if ((p.flags & (BS_WANT_PSI | BS_DETERMINISTIC | BS_FFT_CUFFT | BS_SHORT_TILED)) || !c->d.fuse_interp ||
        p.spline_order != 4 || p.local_frac > 0.0)
        return false;
    const size_t rb = p.precision == BS_FP64 ? 8 : 4;
    return 9 * (size_t)c->w.nmax_fil * rb <= kSplineSmemMax && c->d.m <= 8;
}

// Chooses the staged group: the non-empty members that can take the stage
// launches and ask for it (BS_BATCH_STAGED) or, by default, have at most
// kStageMaxNodes nodes; all of them with the precision, kernel width and
// z-column CTA size of the first such member.
void batch_group(bs_batch* b)
{
    b->grouped.assign(b->nconf, 0);
    b->ngrouped = 0;
    const bs_ctx* c0 = nullptr;
    for (int i = 0; i < b->nconf; ++i) {
        const bs_ctx* c = b->ctx[i];
        if (c->N == 0 || b->mode[i] == BS_BATCH_PER_MEMBER || !batch_stageable(c)) continue;
        if (b->mode[i] == 0 && c->N > kStageMaxNodes) continue;
        if (c0 && (c->p.precision != c0->p.precision || c->p.nufft_w != c0->p.nufft_w ||
                   c->d.zthreads != c0->d.zthreads))
            continue;
        if (!c0) c0 = c;
        b->grouped[i] = 1;
        ++b->ngrouped;
    }
}

// Builds the descriptors of every batched stage for these node and velocity
// buffers and uploads them (synchronously; not inside a stream capture).
template <typename T>
int batch_build(bs_batch* b, const double* nodes, double* vel)
{
    Arena A;
    std::vector<BatchL> st;
    std::vector<int> blk;
    std::vector<bs_ctx*> mem;
    std::vector<int64_t> noff;
    for (int i = 0; i < b->nconf; ++i)
        if (b->grouped[i]) {
            mem.push_back(b->ctx[i]);
            noff.push_back(b->node_off[i]);
        }
    const size_t nm = mem.size();
    const int zt = mem[0]->d.zthreads;
    auto add = [&](auto& desc, int threads, size_t smem) {
        st.push_back(stage(A, desc, blk, threads, smem));
        blk.clear();
    };
    {   // 0 spline
        std::vector<SplineD<T>> D;
        size_t sm = 0;
        for (size_t m = 0; m < nm; ++m) {
            const bs_ctx* c = mem[m];
            const Work& w = c->w;
            D.push_back({ nodes + 3 * noff[m], w.off, w.shift, c->nfil, w.nmax_fil, (T*)w.hseg, (T*)w.dp, (T*)w.ds,
                          (T*)w.Mm, (T*)w.Tper });
            blk.push_back(c->nfil);
            sm = std::max(sm, spline_smem<T>(w.nmax_fil));
        }
        add(D, 32, sm);
    }
    {   // 1 nodes
        std::vector<NodesD<T>> D;
        for (size_t m = 0; m < nm; ++m) {
            const bs_ctx* c = mem[m];
            const Work& w = c->w;
            NodesD<T> e;
            fill_geom(c, e.P);
            e.P.want_psi = 0;
            e.nodes = nodes + 3 * noff[m];
            e.fil_of = w.fil_of;
            e.prev = w.prev;
            e.off = w.off;
            e.shift = w.shift;
            e.hseg = (const T*)w.hseg;
            e.dp = (const T*)w.dp;
            e.ds = (const T*)w.ds;
            e.Mm = (const T*)w.Mm;
            e.Tper = (const T*)w.Tper;
            e.Dd = nullptr;
            e.sr_rec = (SrRec<T>*)w.sr_rec;
            e.sr_key = w.sr_key;
            e.lr_rec = (LrRec<T>*)w.lr_rec;
            e.lr_key = w.lr_key;
            e.tgt = (SrTgt<T>*)w.tgt;
            e.vls = w.vls;
            e.pls = w.pls;
            e.status = w.status;
            D.push_back(e);
            blk.push_back(cdiv(c->N, 128));
        }
        add(D, 128, 0);
    }
    // counting sorts: zero the counts, count, scan, copy to the cursors, scatter
    auto zero_stage = [&](auto cnt_of, auto n_of) {
        std::vector<ZeroD> Z;
        for (size_t m = 0; m < nm; ++m) {
            Z.push_back({ cnt_of(mem[m]), n_of(mem[m]) + 1 });
            blk.push_back(std::min(cdiv(n_of(mem[m]) + 1, 256), 256));
        }
        add(Z, 256, 0);
    };
    auto scan_stage = [&](auto cnt_of, auto n_of, auto tmp_of) {
        std::vector<ScanD> S;
        std::vector<int> one;
        for (size_t m = 0; m < nm; ++m) {
            const int n = n_of(mem[m]);
            S.push_back({ cnt_of(mem[m]), n, tmp_of(mem[m]), scan_blocks(n) });
            blk.push_back(scan_blocks(n));
            one.push_back(1);
        }
        add(S, 1024, 0);
        blk = one;
        add(S, 1024, 0);
    };
    auto copy_stage = [&](auto cnt_of, auto n_of, auto cur_of) {
        std::vector<CopyD> Cd;
        for (size_t m = 0; m < nm; ++m) {
            Cd.push_back({ cnt_of(mem[m]), cur_of(mem[m]), n_of(mem[m]) });
            blk.push_back(std::min(cdiv(n_of(mem[m]), 256), 256));
        }
        add(Cd, 256, 0);
    };
    auto cell_cnt = [](bs_ctx* c) { return c->w.cell_cnt; };
    auto cell_n = [](bs_ctx* c) { return (int)c->d.ncells; };
    auto cell_tmp = [](bs_ctx* c) { return c->w.scan_tmp; };
    auto cell_cur = [](bs_ctx* c) { return c->w.cell_cur; };
    zero_stage(cell_cnt, cell_n);                                                          // 2 zero
    {   // 3 count
        std::vector<CountD> D;
        for (size_t m = 0; m < nm; ++m) {
            D.push_back({ mem[m]->w.sr_key, (int)mem[m]->NQ, mem[m]->w.cell_cnt });
            blk.push_back(cdiv(mem[m]->NQ, kThreads));
        }
        add(D, kThreads, 0);
    }
    scan_stage(cell_cnt, cell_n, cell_tmp);                                                // 4, 5 scan
    copy_stage(cell_cnt, cell_n, cell_cur);                                                // 6 copy
    {   // 7 scatter
        std::vector<ScatterD<SrRec<T>>> D;
        for (size_t m = 0; m < nm; ++m) {
            const Work& w = mem[m]->w;
            D.push_back({ w.sr_key, (const SrRec<T>*)w.sr_rec, (int)mem[m]->NQ, w.cell_cur, (SrRec<T>*)w.sr_sorted });
            blk.push_back(cdiv(mem[m]->NQ, kThreads));
        }
        add(D, kThreads, 0);
    }
    {   // 8 short range (warp per node)
        std::vector<ShortD<T>> D;
        for (size_t m = 0; m < nm; ++m) {
            const Work& w = mem[m]->w;
            ShortD<T> e;
            fill_short(mem[m], false, e.P);
            e.tgt = (const SrTgt<T>*)w.tgt;
            e.prev = w.prev;
            e.start = w.cell_cnt;
            e.src = (const SrRec<T>*)w.sr_sorted;
            e.vsr = w.vsr;
            e.psr = w.psr;
            D.push_back(e);
            blk.push_back(cdiv(32LL * mem[m]->N, 256));
        }
        add(D, 256, 0);
    }
    auto col_cnt = [](bs_ctx* c) { return c->w.col_cnt; };
    auto colb_n = [](bs_ctx* c) { return c->d.ncolb; };  // spread bins: blocks x z-buckets
    auto col_n = [](bs_ctx* c) { return c->d.ncols; };   // node bins: blocks
    auto col_tmp = [](bs_ctx* c) { return c->w.scan_tmp2; };
    auto col_cur = [](bs_ctx* c) { return c->w.col_cur; };
    zero_stage(col_cnt, colb_n);                                                           // 9 zero
    {   // 10 column count, 13 column scatter share the descriptor shape
        std::vector<ColD<T>> D;
        for (size_t m = 0; m < nm; ++m) {
            const Work& w = mem[m]->w;
            ColD<T> e;
            fill_colp(mem[m], e.P);
            e.rec = (const LrRec<T>*)w.lr_rec;
            e.n = (int)mem[m]->NQ;
            e.cnt = w.col_cnt;
            e.out = nullptr;
            e.pts = nullptr;
            D.push_back(e);
            blk.push_back(cdiv(mem[m]->NQ, kThreads));
        }
        add(D, kThreads, 0);
    }
    scan_stage(col_cnt, colb_n, col_tmp);                                                  // 11, 12 scan
    copy_stage(col_cnt, colb_n, col_cur);                                                  // 13 copy
    {   // 14 column scatter
        std::vector<ColD<T>> D;
        for (size_t m = 0; m < nm; ++m) {
            const Work& w = mem[m]->w;
            ColD<T> e;
            fill_colp(mem[m], e.P);
            e.rec = (const LrRec<T>*)w.lr_rec;
            e.n = (int)mem[m]->NQ;
            e.cnt = w.col_cur;
            e.out = w.col_rec;
            e.pts = w.col_pts;
            D.push_back(e);
            blk.push_back(cdiv(mem[m]->NQ, kThreads));
        }
        add(D, kThreads, 0);
    }
    {   // 15 spread + z transform
        std::vector<SpzD<T>> D;
        size_t sm = 0;
        for (size_t m = 0; m < nm; ++m) {
            const bs_ctx* c = mem[m];
            const Work& w = c->w;
            SpzD<T> e;
            fill_spzp<T>(c, false, e.P);
            e.cstart = w.col_cnt;
            e.recs = w.col_rec;
            e.pts = w.col_pts;
            e.tw2 = cx_at<T>(w.tw, c->d.ng[0] + c->d.ng[1]);
            e.F1 = w.spec;
            e.vacc = nullptr;
            D.push_back(e);
            blk.push_back(c->d.nbx * c->d.nby);
            sm = std::max(sm, spread_zfft_smem<T>(e.P));
        }
        add(D, zt, sm);
    }
    auto ffty = [&](int sign) {
        std::vector<FftYD<T>> D;
        size_t sm = 0;
        for (size_t m = 0; m < nm; ++m) {
            const bs_ctx* c = mem[m];
            const Work& w = c->w;
            FftYD<T> e;
            fill_fftyp<T>(c, e.P);
            e.F1 = w.spec;
            e.F2 = w.f2;
            e.tw1 = cx_at<T>(w.tw, c->d.ng[0]);
            e.sign = sign;
            D.push_back(e);
            const int MC = 1 << e.P.lmc, nk = c->d.K[2] + 1;
            blk.push_back(3 * c->d.ng[0] * ((nk + MC - 1) / MC));
            sm = std::max(sm, fft_y_smem<T>(e.P));
        }
        add(D, kThreads, sm);
    };
    ffty(-1);  // 16
    {   // 17 x transform + k-space pass + inverse x transform
        std::vector<FftXD<T>> D;
        size_t sm = 0;
        for (size_t m = 0; m < nm; ++m) {
            const bs_ctx* c = mem[m];
            const Work& w = c->w;
            FftXD<T> e;
            fill_fftxp<T>(c, e.P);
            e.F2 = w.f2;
            e.tw0 = w.tw;
            e.tab0 = (const T*)w.ktab;
            e.tab1 = e.tab0 + (c->d.K[0] + 1);
            e.tab2 = e.tab1 + (c->d.K[1] + 1);
            D.push_back(e);
            const int MC = 1 << e.P.lmc, nk = c->d.K[2] + 1;
            blk.push_back((2 * c->d.K[1] + 1) * ((nk + MC - 1) / MC));
            sm = std::max(sm, fft_x_smem<T>(e.P));
        }
        add(D, zt, sm);
    }
    ffty(+1);  // 18
    {   // 19 zero: the interpolation sums and the node-block counts
        std::vector<ZeroD> Z;
        for (size_t m = 0; m < nm; ++m) {
            const bs_ctx* c = mem[m];
            const int nv = (int)(3 * c->N * (long long)sizeof(T) / sizeof(int));
            Z.push_back({ (int*)c->w.vacc, nv });
            blk.push_back(std::min(cdiv(nv, 256), 256));
            Z.push_back({ c->w.ncol_cnt, c->d.ncols + 1 });
            blk.push_back(std::min(cdiv(c->d.ncols + 1, 256), 256));
        }
        add(Z, 256, 0);
    }
    std::vector<NodeWD<T>> NW;
    for (size_t m = 0; m < nm; ++m) {
        const bs_ctx* c = mem[m];
        const Work& w = c->w;
        NodeWD<T> e;
        fill_interp(c, false, e.P);
        e.tx = c->d.tx;
        e.ty = c->d.ty;
        e.nbx = c->d.nbx;
        e.nodes = nodes + 3 * noff[m];
        e.rec = w.nd_rec;
        e.key = w.nd_key;
        e.rank = w.nd_rank;
        e.cnt = w.ncol_cnt;
        e.sorted = w.nd_sorted;
        NW.push_back(e);
        blk.push_back(cdiv(c->N, kThreads));
    }
    add(NW, kThreads, 0);                                                                  // 20 node weights
    auto nb_cnt = [](bs_ctx* c) { return c->w.ncol_cnt; };
    auto nb_tmp = [](bs_ctx* c) { return c->w.scan_tmp; };
    scan_stage(nb_cnt, col_n, nb_tmp);                                                     // 21, 22 scan
    for (size_t m = 0; m < nm; ++m) blk.push_back(cdiv(mem[m]->N, kThreads));
    add(NW, kThreads, 0);                                                                  // 23 node scatter
    {   // 24 inverse z transform + interpolation
        std::vector<SpzD<T>> D;
        size_t sm = 0;
        for (size_t m = 0; m < nm; ++m) {
            const bs_ctx* c = mem[m];
            const Work& w = c->w;
            SpzD<T> e;
            fill_spzp<T>(c, false, e.P);
            e.cstart = w.ncol_cnt;
            e.recs = w.nd_sorted;
            e.pts = nullptr;
            e.tw2 = cx_at<T>(w.tw, c->d.ng[0] + c->d.ng[1]);
            e.F1 = w.spec;
            e.vacc = (T*)w.vacc;
            D.push_back(e);
            blk.push_back(c->d.nbx * c->d.nby);
            sm = std::max(sm, zfft_interp_smem<T>(e.P));
        }
        add(D, zt, sm);
    }
    {   // 25 final sum
        std::vector<SumD<T>> D;
        for (size_t m = 0; m < nm; ++m) {
            const bs_ctx* c = mem[m];
            D.push_back({ (int)(3 * c->N), (const T*)c->w.vacc, c->w.vls, c->w.vsr, vel + 3 * noff[m] });
            blk.push_back(std::min(cdiv(3 * c->N, 256), 4096));
        }
        add(D, 256, 0);
    }
    // upload, then turn the offsets into device pointers.  The group's
    // streams finish with the old tables first; the copy is ordered on the
    // group's stream and waited for (a plain copy from pageable memory may
    // return before its DMA lands, and the group's streams do not wait for
    // the legacy stream it runs on).
    CUDA_TRY(cudaStreamSynchronize(b->gmain));
    CUDA_TRY(cudaStreamSynchronize(b->side));
    if (b->arena) cudaFree(b->arena);
    b->arena = nullptr;
    CUDA_TRY(cudaMalloc(&b->arena, A.bytes.size()));
    b->arena_bytes = A.bytes.size();
    CUDA_TRY(cudaMemcpyAsync(b->arena, A.bytes.data(), A.bytes.size(), cudaMemcpyHostToDevice, b->gmain));
    CUDA_TRY(cudaStreamSynchronize(b->gmain));
    for (BatchL& L : st) {
        L.desc = (const unsigned char*)b->arena + (size_t)L.desc;
        L.bstart = (const int*)((const unsigned char*)b->arena + (size_t)L.bstart);
    }
    b->stages = st;
    b->a_nodes = nodes;
    b->a_vel = vel;
    return BS_OK;
}

// Issues the staged group's launches (one per stage, every grouped member in
// each) on s, the short range and the node binning on b->side.
template <typename T>
int batch_issue_staged(bs_batch* b, cudaStream_t s)
{
    const std::vector<BatchL>& L = b->stages;
    int w = 0;
    for (int i = 0; i < b->nconf; ++i)
        if (b->grouped[i]) {
            w = b->ctx[i]->p.nufft_w;
            break;
        }
    CE(launch_spline_b<T>(L[0], s));
    CE(launch_nodes_b<T>(L[1], s));
    // the short range and the node binning on a side stream, as in run()
    cudaStream_t ss = b->side;
    CE(cudaEventRecord(b->ev_side, s));
    CE(cudaStreamWaitEvent(ss, b->ev_side, 0));
    CE(launch_zero_b(L[2], ss));
    CE(launch_count_b(L[3], ss));
    CE(launch_scan_b(L[4], L[5], ss));
    CE(launch_copy_b(L[6], ss));
    CE(launch_scatter_b<SrRec<T>>(L[7], ss));
    CE(launch_short_b<T>(L[8], ss));
    CE(launch_zero_b(L[19], ss));
    CE(launch_node_w_b<T>(w, L[20], ss));
    CE(launch_scan_b(L[21], L[22], ss));
    CE(launch_node_scatter_b<T>(w, L[23], ss));
    CE(cudaEventRecord(b->ev_side, ss));
    CE(launch_zero_b(L[9], s));
    CE(launch_col_count_b<T>(L[10], s));
    CE(launch_scan_b(L[11], L[12], s));
    CE(launch_copy_b(L[13], s));
    CE(launch_col_scatter_b<T>(w, L[14], s));
    CE(launch_spread_zfft_b<T>(w, L[15], s));
    CE(launch_fft_y_b<T>(L[16], s));
    CE(launch_fft_x_kspace_b<T>(L[17], s));
    CE(launch_fft_y_b<T>(L[18], s));
    CE(cudaStreamWaitEvent(s, b->ev_side, 0));
    CE(launch_zfft_interp_b<T>(w, L[24], s));
    CE(launch_interp_sum_b<T>(L[25], s));
    return BS_OK;
}

// Precision of the staged group (false: empty or float32 kernels).
bool group_f64(const bs_batch* b)
{
    for (int i = 0; i < b->nconf; ++i)
        if (b->grouped[i]) return b->ctx[i]->p.precision == BS_FP64;
    return false;
}

// (Re)builds the staged group's tables for these buffers if needed.
int batch_ensure_stages(bs_batch* b, const double* nodes, double* vel)
{
    if (b->ngrouped == 0 || (b->a_nodes == nodes && b->a_vel == vel)) return BS_OK;
    return group_f64(b) ? batch_build<double>(b, nodes, vel) : batch_build<float>(b, nodes, vel);
}

// Issues the staged group on b->stream and every other member's evaluation
// on the pool, joined back to b->stream.
int batch_issue(bs_batch* b, const double* nodes, double* vel)
{
    CUDA_TRY(cudaEventRecord(b->ev_start, b->stream));
    for (cudaStream_t s : b->pool) CUDA_TRY(cudaStreamWaitEvent(s, b->ev_start, 0));
    for (int i : b->order) {
        bs_ctx* c = b->ctx[i];
        if (c->N == 0 || b->grouped[i]) continue;
        const size_t o = 3 * (size_t)b->node_off[i];
        const int rc = c->p.precision == BS_FP64 ? run<double>(c, nodes + o, vel + o, nullptr, nullptr, nullptr)
                                                 : run<float>(c, nodes + o, vel + o, nullptr, nullptr, nullptr);
        if (rc != BS_OK) return rc;
    }
    if (b->ngrouped > 0) {
        const int rc = batch_ensure_stages(b, nodes, vel);
        if (rc != BS_OK) return rc;
        CUDA_TRY(cudaStreamWaitEvent(b->gmain, b->ev_start, 0));
        const int rs = group_f64(b) ? batch_issue_staged<double>(b, b->gmain)
                                    : batch_issue_staged<float>(b, b->gmain);
        if (rs != BS_OK) return rs;
        CUDA_TRY(cudaEventRecord(b->ev_group, b->gmain));
        CUDA_TRY(cudaStreamWaitEvent(b->stream, b->ev_group, 0));
    }
    for (size_t k = 0; k < b->pool.size(); ++k) {
        CUDA_TRY(cudaEventRecord(b->ev_done[k], b->pool[k]));
        CUDA_TRY(cudaStreamWaitEvent(b->stream, b->ev_done[k], 0));
    }
    return BS_OK;
}

}  // namespace

extern "C" {

void bs_batch_destroy(bs_batch* b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    for (cudaStream_t s : b->pool) cudaStreamSynchronize(s);
    cudaStreamSynchronize(b->stream);
    if (b->gmain) cudaStreamSynchronize(b->gmain);
    if (b->side) cudaStreamSynchronize(b->side);
    batch_drop_graph(b);
    batch_drop_stages(b);
    for (bs_ctx* c : b->ctx) bs_destroy(c);
    for (cudaEvent_t e : b->ev_done) cudaEventDestroy(e);
    if (b->ev_start) cudaEventDestroy(b->ev_start);
    if (b->ev_side) cudaEventDestroy(b->ev_side);
    if (b->ev_group) cudaEventDestroy(b->ev_group);
    for (cudaStream_t s : b->pool) cudaStreamDestroy(s);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->gmain) cudaStreamDestroy(b->gmain);
    delete b;
}

int bs_batch_create(bs_batch** out, int nconf, const bs_params* params, void* stream)
{
    if (!out || !params || nconf <= 0) return fail(BS_ERR_ARG, "bad batch arguments");
    *out = nullptr;
    bs_batch* b = new bs_batch();
    b->nconf = nconf;
    b->stream = (cudaStream_t)stream;
    b->node_off.assign(nconf + 1, 0);
    cudaError_t e = cudaGetDevice(&b->device);
    const int ns = std::min(nconf, 8);
    int prio_lo = 0, prio_hi = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    // the staged group's short range at the highest priority, as in a
    // single context (17.2 against 17.7 ms for the 64-member batch staged
    // whole); the pool and the group's long range at the default
    for (int k = 0; k < ns && e == cudaSuccess; ++k) {
        cudaStream_t s = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->pool.push_back(s);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->ev_done.push_back(ev);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->side, cudaStreamNonBlocking, prio_hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->gmain, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_side, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_group, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        const int rc = fail(BS_ERR_CUDA, "CUDA set-up failed: %s", cudaGetErrorString(e));
        bs_batch_destroy(b);
        return rc;
    }
    for (int i = 0; i < nconf; ++i) {
        const int f = params[i].flags & (BS_BATCH_PER_MEMBER | BS_BATCH_STAGED);
        if (f == (BS_BATCH_PER_MEMBER | BS_BATCH_STAGED)) {
            bs_batch_destroy(b);
            return fail(BS_ERR_ARG, "batch member %d asks for both BS_BATCH_PER_MEMBER and BS_BATCH_STAGED", i);
        }
        b->mode.push_back(f);
    }
    b->grouped.assign(nconf, 0);
    for (int i = 0; i < nconf; ++i) {
        bs_params p = params[i];
        // stage events cannot be read back from a graph
        p.flags &= ~(BS_TIMING | BS_BATCH_PER_MEMBER | BS_BATCH_STAGED);
        bs_ctx* c = nullptr;
        const int rc = bs_create(&c, &p, nullptr);
        if (rc != BS_OK) {
            std::string msg = g_err;
            bs_batch_destroy(b);
            fail(rc, "batch member %d: %s", i, msg.c_str());
            return rc;
        }
        b->ctx.push_back(c);
    }
    *out = b;
    return BS_OK;
}

int bs_batch_set(bs_batch* b, int i, int nfil, const int64_t* offsets, const int32_t* closing)
{
    if (!b || i < 0 || i >= b->nconf) return fail(BS_ERR_ARG, "bad batch or member index");
    batch_drop_graph(b);
    batch_drop_stages(b);
    const int rc = bs_set_filaments(b->ctx[i], nfil, offsets, closing);
    if (rc != BS_OK) return rc;
    batch_group(b);
    for (int k = 0; k < b->nconf; ++k) b->node_off[k + 1] = b->node_off[k] + b->ctx[k]->N;
    b->order.resize(b->nconf);
    for (int k = 0; k < b->nconf; ++k) b->order[k] = k;
    std::stable_sort(b->order.begin(), b->order.end(),
                     [b](int x, int y) { return b->ctx[x]->N > b->ctx[y]->N; });
    size_t r = 0;  // the members issued one by one, round-robin over the pool
    for (int k : b->order)
        if (!b->grouped[k]) b->ctx[k]->stream = b->pool[r++ % b->pool.size()];
    return BS_OK;
}

int bs_batch_staged_members(bs_batch* b, int32_t* staged)
{
    if (!b || !staged) return fail(BS_ERR_ARG, "null argument");
    for (int k = 0; k < b->nconf; ++k) staged[k] = b->grouped[k] ? 1 : 0;
    return BS_OK;
}

int bs_batch_node_offsets(bs_batch* b, int64_t* offsets)
{
    if (!b || !offsets) return fail(BS_ERR_ARG, "null argument");
    for (int k = 0; k <= b->nconf; ++k) offsets[k] = b->node_off[k];
    return BS_OK;
}

int bs_batch_compute(bs_batch* b, const double* nodes, double* vel)
{
    if (!b) return fail(BS_ERR_ARG, "null batch");
    for (int i = 0; i < b->nconf; ++i)
        if (!b->ctx[i]->have_fil) return fail(BS_ERR_STATE, "batch member %d has no filaments", i);
    if (b->node_off[b->nconf] == 0) return BS_OK;
    if (!nodes || !vel) return fail(BS_ERR_ARG, "null nodes or vel");
    CUDA_TRY(cudaSetDevice(b->device));
    if (!b->stream) return batch_issue(b, nodes, vel);  // the legacy stream cannot be captured
    if (!b->gexec || b->g_nodes != nodes || b->g_vel != vel) {
        batch_drop_graph(b);
        // the staged launches' descriptors are uploaded before the capture
        const int rb = batch_ensure_stages(b, nodes, vel);
        if (rb != BS_OK) return rb;
        CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        const int rc = batch_issue(b, nodes, vel);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (rc != BS_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return fail(BS_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
        b->graph = g;
        CUDA_TRY(cudaGraphInstantiate(&b->gexec, b->graph, cudaGraphInstantiateFlagUseNodePriority));
        b->g_nodes = nodes;
        b->g_vel = vel;
    }
    CUDA_TRY(cudaGraphLaunch(b->gexec, b->stream));
    return BS_OK;
}

int bs_batch_status(bs_batch* b)
{
    if (!b) return fail(BS_ERR_ARG, "null batch");
    CUDA_TRY(cudaSetDevice(b->device));
    // every stream the batch issues on (the caller's may be the legacy one)
    CUDA_TRY(cudaStreamSynchronize(b->stream));
    for (cudaStream_t s : b->pool) CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaStreamSynchronize(b->gmain));
    CUDA_TRY(cudaStreamSynchronize(b->side));
    int first = BS_OK;
    for (int i = 0; i < b->nconf; ++i) {
        const int rc = bs_status(b->ctx[i]);
        if (rc != BS_OK && first == BS_OK) first = rc;
    }
    return first;
}

int bs_batch_member(bs_batch* b, int i, bs_ctx** member)
{
    if (!b || !member || i < 0 || i >= b->nconf) return fail(BS_ERR_ARG, "bad batch or member index");
    *member = b->ctx[i];
    return BS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Choice of the Ewald parameter by measurement (Sec. 5.3 picks alpha =
// C_beta N^(1/3) / L from CPU timings; the balance between the short- and
// long-range parts differs on this GPU, so it is measured here).
// ---------------------------------------------------------------------------
extern "C" int bs_autotune_alpha(const bs_params* base, int nfil, const int64_t* offsets, const int32_t* closing,
                                 const double* nodes, int ncand, const double* cbeta, int reps, bs_params* best,
                                 float* ms_out)
{
    if (!base || !cbeta || !best || !nodes || ncand <= 0 || reps <= 0 || nfil <= 0 || !offsets)
        return fail(BS_ERR_ARG, "bad autotune arguments");
    const double beta = base->alpha * base->rc;
    if (!(beta > 0)) return fail(BS_ERR_ARG, "base parameters need alpha * rc = beta > 0");
    const double Lmin = std::min(base->L[0], std::min(base->L[1], base->L[2]));
    const long long N = offsets[nfil];
    cudaStream_t s = nullptr;
    CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    double* vel = nullptr;
    if (ce == cudaSuccess) ce = cudaMalloc(&vel, sizeof(double) * 3 * (size_t)N);
    if (ce != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaStreamDestroy(s);
        return fail(BS_ERR_CUDA, "autotune set-up failed: %s", cudaGetErrorString(ce));
    }
    int rc = BS_OK, nbest = -1;
    float tbest = 0.0f;
    for (int i = 0; i < ncand && rc == BS_OK; ++i) {
        if (ms_out) ms_out[i] = -1.0f;
        // alpha from the candidate C_beta, M the smallest odd count with
        // k_max >= 2 beta alpha, then alpha re-derived from k_max
        double alpha = cbeta[i] * cbrt((double)N) / Lmin;
        alpha = std::max(alpha, 2.0 * beta / Lmin);  // rc <= L/2
        const int K = (int)ceil(beta * alpha * Lmin / kPi);
        bs_params p;
        if ((rc = bs_params_from_beta(beta, base->L, 2 * K + 1, 0, &p)) != BS_OK) break;
        bs_params q = *base;
        q.alpha = p.alpha;
        q.rc = p.rc;
        for (int c = 0; c < 3; ++c) q.M[c] = p.M[c];
        q.flags &= ~BS_TIMING;
        bs_ctx* c = nullptr;
        if ((rc = bs_create(&c, &q, s)) != BS_OK) {
            // a candidate the library cannot take (its spread grid too large,
            // r_c beyond L/2) is skipped, with -1 in ms_out
            if (rc == BS_ERR_ARG || rc == BS_ERR_RC_GT_HALF_L) {
                rc = BS_OK;
                continue;
            }
            break;
        }
        rc = bs_set_filaments(c, nfil, offsets, closing);
        float t = 0.0f;
        for (int r = 0; r < reps + 1 && rc == BS_OK; ++r) {  // the first call warms up
            if (r == 1) cudaEventRecord(e0, s);
            rc = bs_compute(c, nodes, vel, nullptr);
        }
        if (rc == BS_OK) {
            cudaEventRecord(e1, s);
            ce = cudaEventSynchronize(e1);
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
            if (ce != cudaSuccess) rc = fail(BS_ERR_CUDA, "autotune timing: %s", cudaGetErrorString(ce));
        }
        if (rc == BS_OK) rc = bs_status(c);
        bs_destroy(c);
        if (rc != BS_OK) break;
        t /= (float)reps;
        if (ms_out) ms_out[i] = t;
        if (nbest < 0 || t < tbest) {
            nbest = i;
            tbest = t;
            *best = q;
        }
    }
    cudaFree(vel);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (rc == BS_OK && nbest < 0) return fail(BS_ERR_ARG, "no autotune candidate is admissible");
    return rc;
}

extern "C" int bs_autotune_tiles(const bs_params* base, int nfil, const int64_t* offsets, const int32_t* closing,
                                 const double* nodes, int ncand, const int* cand, int reps, bs_params* best,
                                 float* ms_out)
{
    if (!base || !cand || !best || !nodes || ncand <= 0 || reps <= 0 || nfil <= 0 || !offsets)
        return fail(BS_ERR_ARG, "bad autotune arguments");
    const long long N = offsets[nfil];
    cudaStream_t s = nullptr;
    CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    double* vel = nullptr;
    if (ce == cudaSuccess) ce = cudaMalloc(&vel, sizeof(double) * 3 * (size_t)std::max<long long>(N, 1));
    if (ce != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaStreamDestroy(s);
        return fail(BS_ERR_CUDA, "autotune set-up failed: %s", cudaGetErrorString(ce));
    }
    int rc = BS_OK, nbest = -1;
    float tbest = 0.0f;
    for (int i = 0; i < ncand && rc == BS_OK; ++i) {
        if (ms_out) ms_out[i] = -1.0f;
        bs_params q = *base;
        q.block_x = cand[4 * i];
        q.block_y = cand[4 * i + 1];
        q.block_threads = cand[4 * i + 2];
        q.cell_div = cand[4 * i + 3];
        q.flags &= ~BS_TIMING;
        bs_ctx* c = nullptr;
        if ((rc = bs_create(&c, &q, s)) != BS_OK) {
            if (rc == BS_ERR_ARG) {  // a block the library cannot take: skipped
                rc = BS_OK;
                continue;
            }
            break;
        }
        rc = bs_set_filaments(c, nfil, offsets, closing);
        float t = 0.0f;
        for (int r = 0; r < reps + 1 && rc == BS_OK; ++r) {  // the first call warms up
            if (r == 1) cudaEventRecord(e0, s);
            rc = bs_compute(c, nodes, vel, nullptr);
        }
        if (rc == BS_OK) {
            cudaEventRecord(e1, s);
            ce = cudaEventSynchronize(e1);
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
            if (ce != cudaSuccess) rc = fail(BS_ERR_CUDA, "autotune timing: %s", cudaGetErrorString(ce));
        }
        if (rc == BS_OK) rc = bs_status(c);
        bs_destroy(c);
        if (rc != BS_OK) break;
        t /= (float)reps;
        if (ms_out) ms_out[i] = t;
        if (nbest < 0 || t < tbest) {
            nbest = i;
            tbest = t;
            *best = q;
        }
    }
    cudaFree(vel);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(s);
    if (rc == BS_OK && nbest < 0) return fail(BS_ERR_ARG, "no tile candidate is admissible");
    return rc;
}
