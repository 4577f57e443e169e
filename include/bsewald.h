/*
 * bsewald.h -- C ABI of the GB300 (sm_103a) library that evaluates the
 * periodic Biot-Savart velocity (and optionally the streamfunction) induced
 * by a set of closed or periodic vortex filaments at their own nodes, with
 * the Ewald splitting of J. I. Polanco, "Fast and accurate evaluation of
 * Biot-Savart integrals over spatial curves in periodic domains"
 * (arXiv:2406.07366):
 *
 *     v(s0) = v_local(s0) + v^(n)(s0) + v^(f)(s0) - v^(f)_self(s0)
 *                                        (Sec. 3, Eq. ewald_velocity_splitting)
 *
 * Conventions shared by every call:
 *   - Every function returns a status code (BS_OK = 0); on failure a
 *     thread-local message is available from bs_last_error().  No call
 *     aborts the process and none falls back to a CPU path.
 *   - Arrays of 3-vectors are row-major (x, y, z) per entry, float64.
 *   - "device" pointers are CUDA global-memory pointers on the context's
 *     device; "host" pointers are ordinary or pinned host memory.
 *   - The caller owns every input and output buffer.  The library owns its
 *     workspace, which it allocates only in bs_create / bs_set_filaments
 *     and frees in bs_destroy.  The compute calls allocate nothing.
 *   - All device work is issued on the stream given to bs_create (or set
 *     with bs_set_stream); the compute calls return before that work ends,
 *     except bs_compute_host and bs_status, which synchronise that stream.
 *   - Node positions are the unwrapped curve coordinates; the library wraps
 *     them into the box [0, L) only to bin them.
 */
#ifndef BSEWALD_H
#define BSEWALD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
enum {
    BS_OK = 0,
    BS_ERR_ARG = 1,            /* invalid argument or parameter            */
    BS_ERR_RC_GT_HALF_L = 2,   /* r_c > min(L)/2 (minimum-image rule, Sec. 5.2 footnote) */
    BS_ERR_NET_VORTICITY = 3,  /* sum of closing offsets n_l is not zero: the
                                  mean vorticity must vanish (Sec. 2.2) */
    BS_ERR_SPLINE = 4,         /* a filament has fewer nodes than the spline order */
    BS_ERR_NONFINITE = 5,      /* a non-finite node position was seen        */
    BS_ERR_OOM = 6,            /* device allocation failed                   */
    BS_ERR_CUDA = 7,           /* a CUDA runtime call failed                 */
    BS_ERR_CUFFT = 8,          /* a cuFFT call failed                        */
    BS_ERR_TIMEOUT = 9,        /* a bounded device wait gave up              */
    BS_ERR_STATE = 10,         /* call out of order (e.g. no filaments set)  */
    BS_ERR_GEOMETRY = 11       /* a segment is longer than min(L)/4, so its
                                  minimum image is not the curve itself     */
};

/* ---- precision forms ------------------------------------------------- */
enum {
    BS_FP64 = 0,   /* every stage in float64 (cuFFT D2Z/Z2D)                */
    BS_MIXED = 1   /* float32 spread/FFT/k-space/interp/short range; float64
                      node positions, cell-relative offsets and the final sum */
};

/* ---- flags ----------------------------------------------------------- */
enum {
    BS_WANT_PSI = 1,   /* also produce the streamfunction (Eq. ewald_streamfunction_splitting) */
    BS_TIMING = 2,     /* record per-stage CUDA-event times (bs_stage_times) */
    BS_FFT_CUFFT = 4,  /* long range through full cuFFT R2C/C2R transforms instead of
                          the library's pruned per-axis transforms (a cross-check path) */
    BS_DETERMINISTIC = 8,  /* bitwise-reproducible results on a given GPU and build: the binned
                              sources keep a fixed order and no floating-point sum depends on thread
                              timing (slower spread); not with BS_FFT_CUFFT (BS_ERR_ARG) */
    /* Short-range kernel choice (Sec. 3.2); by default the library picks by the
       mean count of nodes per r_c cube (8 or more: tiled).  The two give the
       same sum up to rounding order. */
    BS_SHORT_TILED = 16,    /* a CTA per r_c cube of nodes stages its neighbour sources in
                               shared memory (cells per cut-off up to 4) */
    BS_SHORT_PER_NODE = 32, /* a warp per node walks its neighbour rows in global memory */
    BS_BATCH_PER_MEMBER = 64, /* bs_batch_create only: issue this member's evaluation by
                                 itself on the stream pool, whatever its size */
    BS_BATCH_STAGED = 128     /* bs_batch_create only: this member joins the one-launch-per-
                                 stage group whatever its size (when it can take that path) */
};

/*
 * Problem and method parameters (Sec. 2 problem statement; Sec. 3 split;
 * Sec. 4 cut-offs; Appendix A NUFFT).
 *   L[3]          periods of the box (Sec. 2.1)
 *   kappa         circulation (Sec. 2.2)
 *   a, delta      core radius and core-profile constant Delta (Sec. 2.3)
 *   alpha         Ewald splitting parameter (Eq. ewald_green_functions)
 *   rc            short-range cut-off, rc <= min(L)/2
 *   M[3]          resolved Fourier modes per axis; the mode cube is
 *                 |m_d| <= floor((M_d - 1)/2), k_max,d = (2 pi / L_d) floor((M_d-1)/2)
 *                 (Sec. 3.3, the Nyquist mode of even M is not used)
 *   quad_Q        Gauss-Legendre points per segment, 1..8 (Eq. line_integral_quadrature)
 *   spline_order  4 (cubic) or 6 (quintic, the paper's production setting)
 *   nufft_sigma   oversampling factor sigma > 1 (Appendix A)
 *   nufft_w       spreading width in grid points, even, 2..16 (Appendix A)
 *   precision     BS_FP64 or BS_MIXED
 *   flags         BS_WANT_PSI | BS_TIMING | BS_FFT_CUFFT | BS_DETERMINISTIC |
 *                 BS_SHORT_TILED | BS_SHORT_PER_NODE
 *   cell_div      cells per cut-off length m (cells of edge >= rc/m); the
 *                 paper uses 3 (Sec. 5.3); 0 selects the library default
 *   local_frac    0: the local terms (Eqs. BS_local, streamfunction_local)
 *                 cover the two whole local segments.  In (0, 1): the local
 *                 segments are subdivided (Sec. 5.2): the Taylor expansions
 *                 cover the fraction local_frac of each next to the node and
 *                 the rest is integrated with the plain Biot-Savart kernel,
 *                 quad_Q-point Gauss-Legendre on the pieces [f, 2f], [2f, 4f],
 *                 ..., [2^m f, 1] of the segment (f = local_frac, measured from
 *                 the node).  The paper uses about 0.1.
 *   block_x, block_y   z-column block of the spread, the fused inverse-z
 *                 interpolation and the x pass: block_x x block_y grid
 *                 columns per CTA, each in {1, 2, 4}, block_y even unless
 *                 the interpolation may run unfused; 0, 0 selects the
 *                 library default (blocks sized for about 50-85 KB of shared
 *                 memory).  bs_autotune_tiles picks them by timing.
 *   block_threads threads per CTA of those kernels: 256, or 512 (float32
 *                 only); 0 selects the default
 */
typedef struct {
    double L[3];
    double kappa;
    double a;
    double delta;
    double alpha;
    double rc;
    int M[3];
    int quad_Q;
    int spline_order;
    double nufft_sigma;
    int nufft_w;
    int precision;
    int flags;
    int cell_div;
    double local_frac;
    int block_x;
    int block_y;
    int block_threads;
} bs_params;

typedef struct bs_ctx bs_ctx;

/*
 * Fill *out from the accuracy coefficient beta (Sec. 4, after Eq.
 * error_trunc_streamfunction: r_c = beta/alpha, k_max = 2 beta alpha).
 *   M > 0 : M modes per axis are kept and alpha = k_max / (2 beta) with
 *           k_max = (2 pi / min L) floor((M-1)/2).
 *   M == 0: alpha = C_beta N^(1/3) / min L (Eq. alpha_optimal_performance,
 *           C_beta from Table tab:performance, interpolated in beta), and
 *           M = 2 ceil(beta alpha min(L) / pi) + 1, then alpha re-derived.
 * nufft_w is the Table tab:performance width for beta (sigma = 1.5).
 * The other fields take the paper's defaults (kappa = 1, a = 1e-8,
 * delta = 1/4, Q = 3, cubic, BS_FP64).  Host-only; returns BS_ERR_ARG for
 * beta <= 0, non-positive L or N < 0 with M == 0.
 */
int bs_params_from_beta(double beta, const double L[3], int M, long long N, bs_params* out);

/*
 * Truncation error estimates of Sec. 4 (Eqs. error_trunc_velocity,
 * error_trunc_streamfunction) for a total vortex length total_length, with
 * beta = alpha * rc.  Host-only.  Either output may be NULL.
 */
int bs_error_estimate(const bs_params* p, double total_length, double* eps_v, double* eps_psi);

/*
 * Host-side helper (Appendix A, Eq. kaiser_bessel_bw): the spread grid size
 * n_g[3] the context will use and, if table != NULL, the per-axis
 * deconvolution factors F_d(m), m = 0..floor((M_d-1)/2), concatenated over
 * the three axes, where F(m) = (w/2) phi_hat(pi m w / n_g) / phi(0) is the
 * Fourier transform of the normalised spreading kernel divided by the grid
 * spacing.  table must hold sum_d (floor((M_d-1)/2) + 1) doubles.
 */
int bs_nufft_setup(const bs_params* p, int n_g[3], double* table);

/* Create a context on the current CUDA device; stream is a cudaStream_t
 * (NULL = legacy default stream).  Validates *p: BS_ERR_ARG,
 * BS_ERR_RC_GT_HALF_L. */
int bs_create(bs_ctx** out, const bs_params* p, void* stream);

/* Replace the stream used for subsequent calls. */
int bs_set_stream(bs_ctx* ctx, void* stream);

/*
 * Set the filament topology and allocate the workspace for it.
 *   nfil              number of filaments, >= 0
 *   offsets  (host)   nfil+1 int64, offsets[0] = 0, filament l owns nodes
 *                     offsets[l] .. offsets[l+1]-1 (Sec. 3.3: N_l may differ)
 *   closing  (host)   nfil x 3 int32, n_l with s(tau + T) = s(tau) + n_l L
 *                     (Sec. 2.1); NULL means every filament is closed.
 * Errors: BS_ERR_ARG (bad offsets), BS_ERR_SPLINE (N_l < spline order),
 * BS_ERR_NET_VORTICITY (sum_l n_l != 0), BS_ERR_OOM.
 */
int bs_set_filaments(bs_ctx* ctx, int nfil, const int64_t* offsets, const int32_t* closing);

/*
 * Velocity (and streamfunction) at every node.
 *   nodes (device) N x 3 node positions
 *   vel   (device) N x 3 output
 *   psi   (device) N x 3 output, or NULL; needs BS_WANT_PSI at bs_create
 * Allocates nothing; asynchronous on the context stream.  Device-side
 * problems (non-finite input, over-long segments) are recorded in a status
 * word that bs_status() reports.
 */
int bs_compute(bs_ctx* ctx, const double* nodes, double* vel, double* psi);

/* As bs_compute with HOST buffers: copies nodes in, computes, copies the
 * results out and synchronises the stream.  Use pinned memory for speed. */
int bs_compute_host(bs_ctx* ctx, const double* nodes, double* vel, double* psi);

/*
 * Kinetic energy per unit mass (Sec. 2.4, Eq. kinetic_energy_streamfunction,
 * E = kappa/(2V) oint psi . ds), with the velocity and streamfunction of
 * the same evaluation.  The long-range part is the float64 Fourier
 * reduction (1/2) sum_{k != 0} e^{-k^2/4 alpha^2} |omega_k|^2 / k^2 over the
 * resolved modes; the rest (psi_local + psi^(n) - psi^(f)_self at the nodes,
 * dotted with the tau-derivative of the curve) is interpolated by a periodic
 * spline of the curve's order (cubic or quintic) on the same knots and
 * integrated exactly along each filament.
 *   nodes  (device) N x 3
 *   vel    (device) N x 3 output, or NULL
 *   psi    (device) N x 3 output, or NULL
 *   energy (host)   scalar output
 * Needs BS_WANT_PSI; synchronises the stream.  Cubic curves: filaments up
 * to 5120 nodes.
 */
int bs_compute_energy(bs_ctx* ctx, const double* nodes, double* vel, double* psi, double* energy);

/*
 * The four parts of Eq. ewald_velocity_splitting separately, for parity
 * tests: parts (device) 4 x N x 3 = [v_local, v^(n), v^(f), v^(f)_self];
 * psi_parts (device) the same for the streamfunction, or NULL.
 */
int bs_compute_parts(bs_ctx* ctx, const double* nodes, double* parts, double* psi_parts);

/*
 * Quadrature points and charges of the curves through nodes (Eq.
 * vorticity_fourier_coefs: q = w_i dtau_j s'(tau)): nodes (device) N x 3;
 * qX, qq (device) N*Q x 3 float64 outputs, point (j, i) at row j*Q + i,
 * positions wrapped into [0, L).  Refits the splines; allocates nothing.
 */
int bs_get_quadrature(bs_ctx* ctx, const double* nodes, double* qX, double* qq);

/*
 * bs_energy_spectrum -- kinetic energy spectrum of the filaments' velocity
 * field on the context's Fourier modes (Eq. def_energy_spectrum):
 *   E(k_m) = 1/(2 dk) sum over |k| in [k_m - dk/2, k_m + dk/2) of |v_k|^2,
 *   k_m = m dk, dk = 2 pi / min L, m = 0..nbins-1,
 * with v_k = i k x omega_k / k^2 from the same spread and forward transforms
 * as bs_compute (the modes |m_d| <= K_d, k = 0 excluded).  smoothed = 0: the
 * full (unsmoothed) field's truncated spectrum; smoothed = 1: the long-range
 * field's, E(k) e^{-k^2 / 2 alpha^2} (Sec. 6, Fig. fig:energy_spectra).
 *   nodes (device) N x 3; Ek (host) nbins doubles; dk_out (host, or NULL)
 * Shells past the corner of the mode cube are zero.  Synchronises the
 * context stream.  Needs the default transform path (BS_ERR_STATE with
 * BS_FFT_CUFFT).  Errors: BS_ERR_ARG, BS_ERR_STATE, BS_ERR_CUDA.
 */
int bs_energy_spectrum(bs_ctx* ctx, const double* nodes, int smoothed, int nbins, double* Ek, double* dk_out);

/*
 * bs_coarse_velocity -- the long-range (Gaussian-filtered, coarse-grained)
 * velocity v^(f) on the context's spread grid (Sec. 3.3 and Sec. 6): the
 * same spread, transforms and k-space pass as bs_compute, with the spread's
 * deconvolution only (no interpolation), so that
 *   grid[c][x][y][z] = sum over the mode cube of v^(f)_k e^{i k . x_g},
 *   x_g = (x L_0 / n_0, y L_1 / n_1, z L_2 / n_2), c = 0, 1, 2.
 *   nodes (device) N x 3; grid (device) 3 n_0 n_1 n_2 float64, or NULL to
 *   query the size; n_g (host, or NULL) receives n_0, n_1, n_2.
 * Asynchronous on the context stream.  Needs the default transform path
 * (BS_ERR_STATE with BS_FFT_CUFFT).  Errors: BS_ERR_ARG, BS_ERR_STATE,
 * BS_ERR_CUDA.
 */
int bs_coarse_velocity(bs_ctx* ctx, const double* nodes, double* grid, int n_g[3]);

/*
 * Capture one bs_compute(ctx, nodes, vel, psi) into a CUDA graph bound to
 * these device buffers (both branches of the evaluation become graph
 * branches), replacing any previous graph; bs_graph_launch replays it on
 * the context stream.  Needs a non-default stream (bs_create /
 * bs_set_stream).  A later bs_set_filaments drops the graph.  The buffers
 * must stay valid while the graph is used; their contents are read at
 * replay time.  Errors: BS_ERR_ARG, BS_ERR_STATE (replay without capture),
 * BS_ERR_CUDA.
 */
int bs_graph_capture(bs_ctx* ctx, const double* nodes, double* vel, double* psi);
int bs_graph_launch(bs_ctx* ctx);

/*
 * Time stepping (Sec. 5.2): nodes advance by ds/dt = v(s) with the classical
 * fourth-order Runge-Kutta scheme; every stage refits the spline, because
 * every evaluation does.  nodes (device, N x 3 float64) are read and
 * overwritten in place.
 * bs_rk4_step: one step of size dt, issued directly on the context stream.
 * bs_rk4_capture: capture one step, bound to this node buffer, into a CUDA
 * graph (non-default stream needed; replaces a previous capture; dropped by
 * bs_set_filaments); bs_rk4_launch replays it nsteps times.
 * The first call allocates the RK4 workspace (15 N doubles).  dt is fixed at
 * capture; the paper's stable choice is the Kelvin-wave period at the
 * smallest node spacing.  Geometry faults surface through bs_status.
 * Errors: BS_ERR_ARG (dt <= 0 or not finite, null nodes, default stream for
 * capture), BS_ERR_STATE (launch without capture), BS_ERR_OOM, BS_ERR_CUDA.
 */
int bs_rk4_step(bs_ctx* ctx, double* nodes, double dt);
int bs_rk4_capture(bs_ctx* ctx, double* nodes, double dt);
int bs_rk4_launch(bs_ctx* ctx, int nsteps);

/*
 * Batches of independent configurations (the paper evaluates one
 * configuration at a time; a batch evaluates many of the Sec. 5 problems,
 * each with its own parameters and grid, in one call).
 *
 * bs_batch_create: nconf members, params[i] for member i (host array,
 * copied; BS_TIMING is ignored).  stream: cudaStream_t the batch runs on.
 * The staged group: members that take the plain velocity path (no
 * BS_WANT_PSI, BS_DETERMINISTIC, BS_FFT_CUFFT or BS_SHORT_TILED, cubic
 * curves, no subdivided local segments) and have at most 2048 nodes (or carry
 * BS_BATCH_STAGED; never with BS_BATCH_PER_MEMBER), with the precision,
 * kernel width and z-column CTA size of the first of them.  Each stage of
 * the group's evaluation is ONE launch for all its members: member m runs
 * its own blocks of the launch with its own parameters, taken from a device
 * table (about 30 launches whatever the member count).  Every other member's
 * evaluation is issued by itself on an internal pool of up to 8 streams,
 * concurrently with the group.  Passing both batch flags on one member is
 * BS_ERR_ARG.  With a non-default
 * stream bs_batch_compute captures the whole batch into one CUDA graph on
 * its first call (again whenever the node or velocity pointer changes, or
 * after bs_batch_set) and replays it; with the legacy default stream (NULL)
 * the work is issued directly.  The stage tables are built (cudaMalloc and a
 * synchronous copy) when the node or velocity pointer changes.
 * bs_batch_set: filaments of member i, as bs_set_filaments.
 * bs_batch_node_offsets: offsets[0..nconf] (host) of each member's nodes in
 * the concatenated node array.
 * bs_batch_staged_members: staged[0..nconf-1] (host) = 1 for the members of
 * the staged group, 0 for those issued by themselves (as of the last
 * bs_batch_set).
 * bs_batch_compute: nodes (device, N_total x 3 float64, members back to
 * back in index order) -> vel (device, same layout).  Asynchronous.
 * bs_batch_status: synchronise and return the first member status that is
 * not BS_OK (clears all).  bs_batch_member: the member's context, owned by
 * the batch (for bs_compute_parts, bs_compute_energy ...; do not destroy it,
 * and do not change its stream).
 * Errors: BS_ERR_ARG, BS_ERR_STATE (a member without filaments), the codes
 * of bs_create / bs_set_filaments, BS_ERR_CUDA.
 */
typedef struct bs_batch bs_batch;
int bs_batch_create(bs_batch** out, int nconf, const bs_params* params, void* stream);
int bs_batch_set(bs_batch* b, int i, int nfil, const int64_t* offsets, const int32_t* closing);
int bs_batch_node_offsets(bs_batch* b, int64_t* offsets);
int bs_batch_staged_members(bs_batch* b, int32_t* staged);
int bs_batch_compute(bs_batch* b, const double* nodes, double* vel);
int bs_batch_status(bs_batch* b);
int bs_batch_member(bs_batch* b, int i, bs_ctx** member);
void bs_batch_destroy(bs_batch* b);

/*
 * bs_autotune_alpha -- pick the Ewald parameter by timing (Sec. 5.3 sets
 * alpha = C_beta N^(1/3) / L with C_beta fitted to CPU timings; the balance
 * of the short- and long-range costs differs on a GPU).  The accuracy
 * coefficient beta = base->alpha * base->rc is kept.  For each candidate
 * cbeta[i]: alpha = cbeta[i] N^(1/3) / min L (at least 2 beta / min L, so
 * rc <= L/2), M the smallest odd count with k_max >= 2 beta alpha, alpha then
 * re-derived from k_max and rc = beta / alpha; every other field comes from
 * *base.  Each candidate context evaluates the filaments (offsets, closing
 * as bs_set_filaments; nodes on the device, N x 3) once to warm up and then
 * reps times on an internal stream, timed with CUDA events.
 *   best   (host) the fastest candidate's parameters
 *   ms_out (host, ncand, or NULL) mean milliseconds per evaluation, -1 for
 *          candidates the library cannot take (spread grid above 1024 points,
 *          r_c above L/2: skipped) or not reached after an error
 * Allocates and frees one context at a time (and an N x 3 scratch); run it
 * before other work on the device, not inside a stream capture.  Errors:
 * BS_ERR_ARG (also when no candidate is admissible), the codes of
 * bs_set_filaments / bs_compute, BS_ERR_CUDA.
 */
int bs_autotune_alpha(const bs_params* base, int nfil, const int64_t* offsets, const int32_t* closing,
                      const double* nodes, int ncand, const double* cbeta, int reps, bs_params* best, float* ms_out);

/*
 * bs_autotune_tiles -- pick the tile shapes and bin sizes of a context by
 * timing on this GPU (an implementation choice: the paper's CPU code has no
 * counterpart): for each candidate i, the z-column block
 * cand[4 i] x cand[4 i + 1] with cand[4 i + 2] threads per CTA (see
 * bs_params.block_x / block_y / block_threads; 0, 0, 0 is the library
 * default) and cand[4 i + 3] cells per cut-off of the short-range cell lists
 * (bs_params.cell_div; 0 the default).  Every other field comes from *base;
 * the method and its accuracy are unchanged (the results differ only by
 * rounding order).  Each candidate context evaluates the filaments (as
 * bs_autotune_alpha: offsets, closing, nodes on the device) once to warm up,
 * then reps times, timed with CUDA events; candidates the library cannot take
 * (too large for shared memory, odd block_y with the fused interpolation)
 * are skipped.
 *   best   (host) the fastest candidate's parameters
 *   ms_out (host, ncand, or NULL) mean milliseconds per evaluation, -1 for
 *          skipped candidates
 * Allocates and frees one context at a time (and an N x 3 scratch); not
 * inside a stream capture.  Errors: BS_ERR_ARG (also when no candidate is
 * admissible), the codes of bs_set_filaments / bs_compute, BS_ERR_CUDA.
 */
int bs_autotune_tiles(const bs_params* base, int nfil, const int64_t* offsets, const int32_t* closing,
                      const double* nodes, int ncand, const int* cand, int reps, bs_params* best, float* ms_out);

/* Synchronise the stream and return the device status word as a status
 * code (BS_OK, BS_ERR_NONFINITE, BS_ERR_GEOMETRY, BS_ERR_TIMEOUT when a
 * kernel's bounded wait for its tensor copies gave up); clears it. */
int bs_status(bs_ctx* ctx);

/*
 * Per-stage times of the last compute call in milliseconds (needs
 * BS_TIMING; the short-range branch stays concurrent with the long-range
 * one, each stage timed by CUDA events on its own stream).  ms[0..n-1]
 * receive, in order: geometry, short-range binning, short range, spread
 * binning, spread, forward FFT, k-space, inverse FFT, interpolation + sum
 * (from the join of both branches), whole evaluation.  Where the inverse z
 * transform is fused with the interpolation (the default pruned path), the
 * inverse-FFT entry covers the inverse y transform and the interpolation
 * entry the inverse z transform, the interpolation and the sum.
 * Synchronises the streams.  Returns the number of entries through *n_out.
 */
int bs_stage_times(bs_ctx* ctx, float* ms, int n, int* n_out);

/*
 * bs_short_range_static -- the short-range velocity sum (the v^(n) part of
 * bs_compute_parts, float64) on caller-given sources and targets, for
 * callers that cannot allocate device memory: an application that owns all
 * device memory through its own allocator or a fixed budget, or a
 * latency-critical loop that must avoid the implicit device synchronisation
 * of cudaMalloc / cudaFree.  The paper has no counterpart; this is a
 * library-side packaging of its short-range sum.
 *
 * It allocates nothing.  Its cell-list scratch is one fixed array of about
 * 9 MiB compiled into the library, present on every device that loads the
 * library until the process exits.  Limits: nsrc <= 131072 sources and at
 * most 65536 cells (cells of edge >= rc/m, m lowered from 3 to 1 to fit;
 * BS_ERR_ARG with a message beyond that).  Every call looks up the
 * scratch address on the current device (cudaGetSymbolAddress, which
 * allocates nothing), so a device reset between calls is harmless.  Every call
 * shares the one array and leaves its contents behind; the call clears
 * what must start at zero.  Calls whose work overlaps on the GPU (two
 * streams, two threads) race on the array: serialise them.
 *
 *   L[3]                 box periods (host)
 *   kappa, alpha, rc     circulation, Ewald parameter, cut-off (rc <= min L / 2)
 *   src_pos  (device)    nsrc x 3 source positions (any image)
 *   src_q    (device)    nsrc x 3 vector charges
 *   src_seg  (device)    nsrc segment ids
 *   tgt_pos  (device)    ntgt x 3 target positions
 *   tgt_omit (device)    ntgt x 2 segment ids each target omits (its C_0)
 *   vel      (device)    ntgt x 3 output, kappa/4pi included
 *   stream               cudaStream_t (NULL = legacy default stream)
 * Asynchronous on stream.  Errors: BS_ERR_ARG, BS_ERR_RC_GT_HALF_L, BS_ERR_CUDA.
 */
int bs_short_range_static(const double L[3], double kappa, double alpha, double rc, int nsrc, const double* src_pos,
                          const double* src_q, const int* src_seg, int ntgt, const double* tgt_pos,
                          const int* tgt_omit, double* vel, void* stream);

/*
 * bs_fma_peak -- measured fused multiply-add throughput of the current
 * device in flop/s (2 per FMA), precision BS_FP64 or BS_MIXED (float32):
 * the denominator of the roofline of the ALU-bound kernels (the short
 * range; the method has no dense contraction, Sec. 3.2).  Eight
 * independent FMA chains per thread, 8 CTAs of 256 threads per SM, best of
 * three timed launches after a warm-up (about 0.1 s each).  Synchronous on
 * the legacy default stream.  Errors: BS_ERR_ARG (null output),
 * BS_ERR_OOM, BS_ERR_CUDA.
 */
int bs_fma_peak(int precision, double* flops_per_s);

/*
 * bs_erfc_f32 -- the float32 complementary error function that the
 * short-range kernels use for g^(n) and f^(n) (Sec. 3.1, Eq.
 * ewald_green_functions): erfc(x) = exp(-x^2) erfcx(x), erfcx a fitted
 * polynomial in 1 / (1 + x/2) on [0, 8].  A diagnostic, so that its error
 * can be measured against CUDA's erfcf / erfc.
 *   x   (device) n float32 arguments in [0, 8]
 *   out (device) n float32 results
 * Asynchronous on stream (NULL = legacy default stream).  Errors:
 * BS_ERR_ARG, BS_ERR_CUDA.
 */
int bs_erfc_f32(int n, const float* x, float* out, void* stream);

/* Device bytes held by the context's workspace. */
int bs_workspace_bytes(bs_ctx* ctx, long long* bytes);

/* Free the context and its workspace (NULL is a no-op). */
void bs_destroy(bs_ctx* ctx);

/* Thread-local message of the last failing call ("" if none). */
const char* bs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BSEWALD_H */
