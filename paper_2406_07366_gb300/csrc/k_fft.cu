// Long-range pipeline on a pruned 3-D FFT (Sec. 3.3, Appendix A).
//
// Only the modes |m_d| <= K_d of the spread grid are needed (Sec. 3.3: the
// k-space pass zeroes every other mode), so the three axes are transformed
// one at a time and each pass writes only what the next one reads:
//
//   A  spread + z real FFT (fused): one CTA owns Tx x Ty full z-columns of
//      the grid in shared memory, spreads every point whose support reaches
//      them, transforms the 3 Tx Ty real z-lines and writes modes 0..K2.
//      F1[c][x][y][mz]
//   B  y FFT of F1, writes |m_y| <= K1.                F2[c][x][my][mz]
//   C  x FFT of F2, the k-space pass (deconvolution, Gaussian filter, curl,
//      1/k^2, truncation, k = 0), inverse x FFT, back into F2 (and F2psi).
//   D  inverse y FFT (zero-padded) into F1.
//   E  inverse z real FFT (zero-padded) fused with the interpolation: the
//      CTA of a column block transforms its 3 Tx Ty z-lines in shared memory
//      and every node whose support reaches the block adds its part of the
//      type-2 sum (k_zfft_interp); the real grid is not written.  For psi,
//      the deterministic mode and the coarse-grained field the inverse z
//      transform writes the real grid instead (k_fft_z_c2r).
//
// The 1-D transforms run in place on lines held in shared memory (lengths
// 2^a 3^b; radix 8, 4, 3, 2), unnormalised, forward sign e^{-2 pi i jk/n}:
// forward transforms by decimation in frequency (natural order in, frequency
// k out at position rev(k)), inverse transforms by decimation in time
// (frequency k in at rev(k), natural order out).  Consumers index rev(k)
// directly, so no reordering pass is needed, and one buffer per line set
// suffices.  Twiddles e^{-2 pi i j/n} come from a table computed on the host
// in float64.  Two real lines are transformed as one complex line.
#include <math.h>

#include <algorithm>
#include <mutex>

#include <cudaTypedefs.h>
#include <string.h>

#include "bs_internal.cuh"

namespace bsw {

// Spread records per staged chunk (two chunks in flight): 64 in float64
// keeps the float64 spread CTA's shared memory at its single-buffered size.
template <typename T>
constexpr int spz_rec_chunk()
{
    return sizeof(T) == 4 ? 128 : 64;
}
// Spread copies per warp chunk in the bucketed record loop (two chunks per
// warp in flight); with at most 512 threads in float32 and 256 in float64 the
// warps' buffers fit in the two block-wide chunks above.
constexpr int kSpzWarpChunk = 8;
// Threads of a z-column-block CTA (spread, fused interpolation): 256, or up
// to 512 for float32.
constexpr int kZThreadsMax = 512;
template <typename T>
constexpr int z_threads_max()
{
    return sizeof(T) == 4 ? kZThreadsMax : kThreads;
}
template <typename T>
int z_threads(const SpZP& P)
{
    return P.nthreads > 0 && P.nthreads <= z_threads_max<T>() ? P.nthreads : kThreads;
}

template <typename T> struct Cx;
template <> struct Cx<float> { using t = float2; };
template <> struct Cx<double> { using t = double2; };

template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C>
__device__ __forceinline__ C cmul(C a, C b) { C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r; }
// multiply by sign * i
template <typename C>
__device__ __forceinline__ C cmuli(C a, int sign) { C r; r.x = -sign * a.y; r.y = sign * a.x; return r; }

// Asynchronous global -> shared copy of one complex value (8 or 16 bytes,
// both addresses aligned to it); visible to the thread after
// cp_async_wait_all(), to the block after the barrier that follows.  A load
// phase issues all its copies before waiting, so every thread keeps many
// loads in flight instead of one.
template <typename C>
__device__ __forceinline__ void cp_async_cx(C* smem_dst, const C* gsrc)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    if constexpr (sizeof(C) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
    else
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// Groups of copies: commit the copies issued so far as one group; wait until
// at most N of this thread's groups are still in flight.
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---- tensor copies (TMA) with an mbarrier, one phase per CTA ----
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for phase `parity` of the barrier, at most about 2^31 clock cycles
// (about a second); false when it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > (1LL << 31)) return false;
    return true;
}
// Generic-proxy writes to shared memory made visible to the tensor copies.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// Tiled 3-D tensor copy global -> shared (box of the map at x, y, z), its
// bytes counted on bar.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z,
                                            unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_u32(dst)),
        "l"(tm), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
// Tiled 3-D tensor copy shared -> global; elements outside the tensor are
// not written.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* tm, int x, int y, int z, const void* src)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(tm),
                 "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* tm, int x, int y, int z, int w,
                                            unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(smem_u32(dst)),
        "l"(tm), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_4d(const CUtensorMap* tm, int x, int y, int z, int w, const void* src)
{
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];\n" ::"l"(tm),
                 "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void tma_store_commit_and_wait_read()
{
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
// First 128-byte aligned byte of the dynamic shared memory (tensor copies
// need it; the launches ask for 128 more bytes).
__device__ __forceinline__ unsigned char* smem_align128(unsigned char* p)
{
    return p + ((128u - (smem_u32(p) & 127u)) & 127u);
}

// e^{-2 pi i m / R} for the composite in-register sizes R in {6, 9, 12, 16,
// 24, 32}, m = 0..R-1, written once per device from float64 values
// (set_fft_constants).  Indices are compile-time constants after unrolling,
// so the factors come straight from the constant bank.
constexpr int kTwOff6 = 0, kTwOff9 = 6, kTwOff12 = 15, kTwOff16 = 27, kTwOff24 = 43, kTwOff32 = 67, kTwCount = 99;
__constant__ float2 c_twf[kTwCount];
__constant__ double2 c_twd[kTwCount];

template <int R> struct TwOff;
template <> struct TwOff<6> { static constexpr int v = kTwOff6; };
template <> struct TwOff<9> { static constexpr int v = kTwOff9; };
template <> struct TwOff<12> { static constexpr int v = kTwOff12; };
template <> struct TwOff<16> { static constexpr int v = kTwOff16; };
template <> struct TwOff<24> { static constexpr int v = kTwOff24; };
template <> struct TwOff<32> { static constexpr int v = kTwOff32; };

template <typename T> __device__ __forceinline__ typename Cx<T>::t ctw(int i);
template <> __device__ __forceinline__ float2 ctw<float>(int i) { return c_twf[i]; }
template <> __device__ __forceinline__ double2 ctw<double>(int i) { return c_twd[i]; }

// Factor R = A * B of a composite size: A the leading base radix.
template <int R> struct Split;
template <> struct Split<6> { static constexpr int A = 3, B = 2; };
template <> struct Split<9> { static constexpr int A = 3, B = 3; };
template <> struct Split<12> { static constexpr int A = 4, B = 3; };
template <> struct Split<16> { static constexpr int A = 4, B = 4; };
template <> struct Split<24> { static constexpr int A = 8, B = 3; };
template <> struct Split<32> { static constexpr int A = 8, B = 4; };

// In-register DFT of size R with exponent sign S (+1 or -1, a compile-time
// constant so that every sign folds into the constants):
// x[k] <- sum_n x[n] e^{S 2 pi i n k / R}, natural order in and out.
template <typename T, int R, int S>
__device__ __forceinline__ void dft(typename Cx<T>::t* x)
{
    constexpr int sign = S;
    using C = typename Cx<T>::t;
    if constexpr (R == 2) {
        const C a = x[0], b = x[1];
        x[0] = cadd(a, b);
        x[1] = csub(a, b);
    } else if constexpr (R == 3) {
        const T h = (T)0.86602540378443864676 * (T)sign;  // sin(2 pi / 3) with the sign
        const C s = cadd(x[1], x[2]);
        const C d = csub(x[1], x[2]);
        C t;
        t.x = x[0].x - (T)0.5 * s.x;
        t.y = x[0].y - (T)0.5 * s.y;
        C u;  // i h d
        u.x = -h * d.y;
        u.y = h * d.x;
        x[0] = cadd(x[0], s);
        x[1] = cadd(t, u);
        x[2] = csub(t, u);
    } else if constexpr (R == 4) {
        const C a = cadd(x[0], x[2]), b = csub(x[0], x[2]);
        const C c = cadd(x[1], x[3]), d = cmuli(csub(x[1], x[3]), sign);
        x[0] = cadd(a, c);
        x[2] = csub(a, c);
        x[1] = cadd(b, d);
        x[3] = csub(b, d);
    } else if constexpr (R == 8) {
        C e[4] = { x[0], x[2], x[4], x[6] };
        C o[4] = { x[1], x[3], x[5], x[7] };
        dft<T, 4, S>(e);
        dft<T, 4, S>(o);
        const T r2 = (T)0.70710678118654752440;
        // w8^m = e^{sign 2 pi i m / 8}
        C w1;
        w1.x = r2;
        w1.y = (T)sign * r2;
        C w3;
        w3.x = -r2;
        w3.y = (T)sign * r2;
        o[1] = cmul(o[1], w1);
        o[2] = cmuli(o[2], sign);
        o[3] = cmul(o[3], w3);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            x[m] = cadd(e[m], o[m]);
            x[m + 4] = csub(e[m], o[m]);
        }
    } else {
        // n = a B + b, k = k1 + A k2:
        // X[k1 + A k2] = sum_b w_B^{b k2} [ w_R^{b k1} sum_a x[a B + b] w_A^{a k1} ]
        constexpr int A = Split<R>::A, B = Split<R>::B;
        C y[R];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            C t[A];
#pragma unroll
            for (int a = 0; a < A; ++a) t[a] = x[a * B + b];
            dft<T, A, S>(t);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) {
                C v = t[k1];
                const int m = (b * k1) % R;
                if (m != 0) {
                    if (4 * m == R) {
                        v = cmuli(v, sign);
                    } else if (2 * m == R) {
                        v.x = -v.x;
                        v.y = -v.y;
                    } else if (4 * m == 3 * R) {
                        v = cmuli(v, -sign);
                    } else {
                        C w = ctw<T>(TwOff<R>::v + m);  // e^{-2 pi i m / R}
                        if constexpr (S > 0) w.y = -w.y;
                        v = cmul(v, w);
                    }
                }
                y[k1 * B + b] = v;
            }
        }
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) {
            C t[B];
#pragma unroll
            for (int b = 0; b < B; ++b) t[b] = y[k1 * B + b];
            dft<T, B, S>(t);
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2) x[k1 + A * k2] = t[k2];
        }
    }
}

// One in-place pass of radix R over nlines lines (stride ls) of length n:
// span L = st R, butterfly (b, j) on elements b L + j + q st.
//   dif: DFT_R, then multiply output m by w_L^{j m};
//   dit: multiply input q by w_L^{j q}, then DFT_R.
// Butterflies are numbered line-fastest, so consecutive threads touch
// different lines at the same offset (distinct banks, one twiddle address).
// x[q] *= w^q, q = 1..R-1, w = e^{S 2 pi i m / n} taken from the float64-
// computed table tw[m] = e^{-2 pi i m / n}.  Only w and w^4 are read; the
// other powers are products of at most three table values (w^2 = w w,
// w^3 = w^2 w, w^5 = w^4 w, w^6 = w^4 w^2, w^7 = w^4 w^3), which keeps the
// rounding within a few units in the last place.
template <typename T, int R, int S>
__device__ __forceinline__ void apply_twiddles(typename Cx<T>::t* x, const typename Cx<T>::t* __restrict__ tw, int m)
{
    using C = typename Cx<T>::t;
    C w[R];
    w[1] = tw[m];
    if constexpr (S > 0) w[1].y = -w[1].y;
    if constexpr (R > 2) w[2] = cmul(w[1], w[1]);
    if constexpr (R > 3) w[3] = cmul(w[2], w[1]);
    if constexpr (R > 4) {
        w[4] = tw[4 * m];
        if constexpr (S > 0) w[4].y = -w[4].y;
    }
    if constexpr (R > 5) w[5] = cmul(w[4], w[1]);
    if constexpr (R > 6) w[6] = cmul(w[4], w[2]);
    if constexpr (R > 7) w[7] = cmul(w[4], w[3]);
    static_assert(R <= 8, "twiddle powers are built for radices up to 8");
#pragma unroll
    for (int q = 1; q < R; ++q) x[q] = cmul(x[q], w[q]);
}

// Line layouts: line-major (TR false: element e of line l at l ls + e) or
// mode-major (TR true: at e nlines + l, the order a tiled bulk copy of rows
// of consecutive modes leaves in shared memory; consecutive lanes on
// consecutive lines read consecutive words).
template <typename T, int R, bool DIF, bool TR = false>
__device__ __forceinline__ void fft_pass(typename Cx<T>::t* __restrict__ buf, int nlines, const FastDiv& dl, int ls,
                                         int n, int st, const FastDiv& sd, int tws,
                                         const typename Cx<T>::t* __restrict__ tw)
{
    constexpr int S = DIF ? -1 : 1;  // forward transforms by DIF, inverse by DIT
    using C = typename Cx<T>::t;
    const int nb = n / R;
    // Shared memory serves 8-byte elements a half-warp (16 lanes) and 16-byte
    // ones a quarter-warp (8 lanes) at a time.  A line count between half of
    // that group and the group that does not divide it (12 of 16, 6 of 8) is
    // numbered as a full group with the extra lines idle: then each group
    // covers G lines at one offset, which an odd line stride spreads over all
    // banks.
    constexpr int G = sizeof(C) == 8 ? 16 : 8;
    const bool pad = nlines < G && (G % nlines) != 0 && 2 * nlines > G;
    const int tot = (pad ? G : nlines) * nb;
    const int L = st * R;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
        int i, line;
        if (pad) {
            i = idx / G;
            line = idx & (G - 1);
            if (line >= nlines) continue;
        } else {
            i = fdiv(idx, dl);
            line = idx - i * nlines;
        }
        const int b = fdiv(i, sd);
        const int j = i - b * st;
        const int es = TR ? nlines : 1;  // element stride
        C* p = TR ? buf + line + (b * L + j) * es : buf + line * ls + b * L + j;
        C x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = p[q * st * es];
        if (!DIF && j > 0) apply_twiddles<T, R, S>(x, tw, j * tws);
        dft<T, R, S>(x);
        if (DIF && j > 0) apply_twiddles<T, R, S>(x, tw, j * tws);
#pragma unroll
        for (int q = 0; q < R; ++q) p[q * st * es] = x[q];
    }
}

// The same pass with the plan and the line count fixed at compile time
// (every stride, twiddle step and index division becomes a constant).
template <typename T, int R, bool DIF, int N, int ST, int TWS, int NL, bool TR>
__device__ __forceinline__ void fft_pass_c(typename Cx<T>::t* __restrict__ buf, int ls,
                                           const typename Cx<T>::t* __restrict__ tw)
{
    constexpr int S = DIF ? -1 : 1;
    using C = typename Cx<T>::t;
    constexpr int G = sizeof(C) == 8 ? 16 : 8;
    constexpr bool pad = NL < G && (G % NL) != 0 && 2 * NL > G;
    constexpr int NLV = pad ? G : NL;
    constexpr int nb = N / R;
    constexpr int tot = NLV * nb;
    constexpr int L = ST * R;
#pragma unroll 1
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
        const int i = idx / NLV;
        const int line = idx % NLV;
        if (pad && line >= NL) continue;
        const int b = i / ST;
        const int j = i % ST;
        constexpr int ES = TR ? NL : 1;  // element stride
        C* p = TR ? buf + line + (b * L + j) * ES : buf + line * ls + b * L + j;
        C x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = p[q * ST * ES];
        if (!DIF && j > 0) apply_twiddles<T, R, S>(x, tw, j * TWS);
        dft<T, R, S>(x);
        if (DIF && j > 0) apply_twiddles<T, R, S>(x, tw, j * TWS);
#pragma unroll
        for (int q = 0; q < R; ++q) p[q * ST * ES] = x[q];
    }
}

// Transform of plan (Rs...) with N = product of the radices and NL lines:
// forward passes in plan order (stride N / R0 first), inverse in reverse.
template <typename T, bool TR, int NL, int N, int ST, int TWS, int R, int... Rest>
__device__ __forceinline__ void fft_c_fwd(typename Cx<T>::t* buf, int ls, const typename Cx<T>::t* __restrict__ tw)
{
    fft_pass_c<T, R, true, N, ST / R, TWS, NL, TR>(buf, ls, tw);
    __syncthreads();
    if constexpr (sizeof...(Rest) > 0) fft_c_fwd<T, TR, NL, N, ST / R, TWS * R, Rest...>(buf, ls, tw);
}

template <typename T, bool TR, int NL, int N, int ST, int TWS, int R, int... Rest>
__device__ __forceinline__ void fft_c_inv(typename Cx<T>::t* buf, int ls, const typename Cx<T>::t* __restrict__ tw)
{
    if constexpr (sizeof...(Rest) > 0) fft_c_inv<T, TR, NL, N, ST / R, TWS * R, Rest...>(buf, ls, tw);
    fft_pass_c<T, R, false, N, ST / R, TWS, NL, TR>(buf, ls, tw);
    __syncthreads();
}

template <typename T, bool DIF, bool TR, int NL, int... Rs>
__device__ __forceinline__ void fft_c(typename Cx<T>::t* buf, int ls, const typename Cx<T>::t* __restrict__ tw)
{
    constexpr int N = (Rs * ...);
    if constexpr (DIF)
        fft_c_fwd<T, TR, NL, N, N, 1, Rs...>(buf, ls, tw);
    else
        fft_c_inv<T, TR, NL, N, N, 1, Rs...>(buf, ls, tw);
}

template <int... Rs>
__device__ __forceinline__ bool plan_is(const FftPlan& pl)
{
    constexpr int r[] = { Rs... };
    if (pl.nr != (int)sizeof...(Rs)) return false;
#pragma unroll
    for (int s = 0; s < (int)sizeof...(Rs); ++s)
        if (pl.r[s] != r[s]) return false;
    return true;
}

// Plans with a compiled form (float): 384 = 8 x 8 x 6 at 12, 16 or 24 lines
// (the 1e5-node tangle), 768 = 8 x 6 x 4 x 4 at 6, 8, 12 or 16 lines (the 4e6-node
// tangle), 192 = 8 x 6 x 4 at 16 or 24 lines (the largest batch members).
template <typename T, bool DIF, bool TR = false>
__device__ __forceinline__ bool fft_const(typename Cx<T>::t* buf, int nlines, int ls, const FftPlan& pl,
                                          const typename Cx<T>::t* __restrict__ tw)
{
    if constexpr (sizeof(T) == 4) {
        if (plan_is<8, 8, 6>(pl)) {
            switch (nlines) {
            case 12: fft_c<T, DIF, TR, 12, 8, 8, 6>(buf, ls, tw); return true;
            case 16: fft_c<T, DIF, TR, 16, 8, 8, 6>(buf, ls, tw); return true;
            case 24: fft_c<T, DIF, TR, 24, 8, 8, 6>(buf, ls, tw); return true;
            default: break;
            }
        } else if (plan_is<8, 6, 4, 4>(pl)) {
            switch (nlines) {
            case 6: fft_c<T, DIF, TR, 6, 8, 6, 4, 4>(buf, ls, tw); return true;
            case 8: fft_c<T, DIF, TR, 8, 8, 6, 4, 4>(buf, ls, tw); return true;
            case 12: fft_c<T, DIF, TR, 12, 8, 6, 4, 4>(buf, ls, tw); return true;
            case 16: fft_c<T, DIF, TR, 16, 8, 6, 4, 4>(buf, ls, tw); return true;
            default: break;
            }
        } else if (plan_is<8, 6, 4>(pl)) {
            switch (nlines) {
            case 16: fft_c<T, DIF, TR, 16, 8, 6, 4>(buf, ls, tw); return true;
            case 24: fft_c<T, DIF, TR, 24, 8, 6, 4>(buf, ls, tw); return true;
            default: break;
            }
        }
    }
    return false;
}

template <typename T, bool DIF, int RM, bool TR = false>
__device__ __forceinline__ void fft_stage(typename Cx<T>::t* buf, int nlines, const FastDiv& dl, int ls,
                                          const FftPlan& pl, int s, const typename Cx<T>::t* __restrict__ tw)
{
    const int R = pl.r[s];
#define BSW_PASS(RR) fft_pass<T, RR, DIF, TR>(buf, nlines, dl, ls, pl.n, pl.st[s], pl.sd[s], pl.tws[s], tw)
    // only the radices up to RM are compiled into this kernel (register budget)
    switch (R) {
    case 32: if constexpr (RM >= 32) BSW_PASS(32); break;
    case 24: if constexpr (RM >= 24) BSW_PASS(24); break;
    case 16: if constexpr (RM >= 16) BSW_PASS(16); break;
    case 12: if constexpr (RM >= 12) BSW_PASS(12); break;
    case 9: if constexpr (RM >= 9) BSW_PASS(9); break;
    case 8: BSW_PASS(8); break;
    case 6: BSW_PASS(6); break;
    case 4: BSW_PASS(4); break;
    case 3: BSW_PASS(3); break;
    default: BSW_PASS(2); break;
    }
#undef BSW_PASS
    __syncthreads();
}

// Forward transform (decimation in frequency), natural order in, frequency
// k left at position rev(k).
template <typename T, int RM, bool TR = false>
__device__ __forceinline__ void fft_fwd_dif(typename Cx<T>::t* buf, int nlines, const FastDiv& dl, int ls, const FftPlan& pl,
                            const typename Cx<T>::t* __restrict__ tw)
{
    if (fft_const<T, true, TR>(buf, nlines, ls, pl, tw)) return;
    for (int s = 0; s < pl.nr; ++s) fft_stage<T, true, RM, TR>(buf, nlines, dl, ls, pl, s, tw);
}

// Inverse transform (decimation in time), frequency k taken at position
// rev(k), natural order out.
template <typename T, int RM, bool TR = false>
__device__ __forceinline__ void fft_inv_dit(typename Cx<T>::t* buf, int nlines, const FastDiv& dl, int ls, const FftPlan& pl,
                            const typename Cx<T>::t* __restrict__ tw)
{
    if (fft_const<T, false, TR>(buf, nlines, ls, pl, tw)) return;
    for (int s = pl.nr - 1; s >= 0; --s) fft_stage<T, false, RM, TR>(buf, nlines, dl, ls, pl, s, tw);
}


// Digit-reversed positions of 8 consecutive frequencies 8q + d (and of
// n - 8q - d) when the plan's first radix is 8 (stride st0 = n / 8): the first
// pass digit is d, so rev(8q + d) = rev(8q) + d st0, and, for d > 0,
// rev(n - 8q - d) = rev(8 (n/8 - q - 1)) + (8 - d) st0.  Three table reads
// instead of sixteen; other plans read the table per frequency.
struct Rev8 {
    int p0, pa, pb, st0;
    bool ok;
};

__device__ __forceinline__ Rev8 rev8_bases(const int* __restrict__ rev, const FftPlan& pl, int q)
{
    Rev8 r;
    r.ok = pl.r[0] == 8;
    r.st0 = pl.st[0];
    r.p0 = r.pa = r.pb = 0;
    if (r.ok) {
        const int n = pl.n;
        r.p0 = rev[8 * q];
        r.pa = rev[(n - 8 * q) % n];
        r.pb = 8 * q + 8 <= n ? rev[n - 8 * q - 8] : 0;
    }
    return r;
}

__device__ __forceinline__ int rev8_pos(const Rev8& r, const int* __restrict__ rev, int k, int d)
{
    return r.ok ? r.p0 + d * r.st0 : rev[k];
}

__device__ __forceinline__ int rev8_neg(const Rev8& r, const int* __restrict__ rev, int n, int k, int d)
{
    return r.ok ? (d == 0 ? r.pa : r.pb + (8 - d) * r.st0) : rev[k == 0 ? 0 : n - k];
}

template <typename T>
__device__ __forceinline__ T kb_val(T z, T zeta, T inorm)
{
    T s2 = (T)1 - z * z;
    s2 = s2 > (T)0 ? s2 : (T)0;
    const T s = sqrt(s2);
    const T num = (s > (T)1e-6) ? -expm1((T)-2 * zeta * s) / s : (T)2 * zeta;
    return exp(zeta * (s - (T)1)) * num * inorm;
}

// ---------------------------------------------------------------------------
// Binning of the spread records by z-column block, each point copied into
// every block its support reaches (with the offset of its support relative
// to that block), so that a block reads only points that touch it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void col_range(int ib, int H, int Tb, int& b0, int& b1)
{
    const int lo = ib - H + 1, hi = ib + H;
    b0 = lo >= 0 ? lo / Tb : -((-lo + Tb - 1) / Tb);
    b1 = hi / Tb;
}

// Rank of a point within its block b (b < 0: no point), one atomic per run of
// equal blocks in the warp; every lane of the warp calls it.
__device__ __forceinline__ int warp_rank(int b, int* __restrict__ cnt)
{
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    int r = 0;
    if (b >= 0 && lane == leader) r = atomicAdd(&cnt[b], __popc(peers));
    r = __shfl_sync(0xffffffffu, r, leader);
    return r + __popc(peers & ((1u << lane) - 1u));
}

// Blocks reached by a point: x blocks [x0, x0 + nx), y blocks [y0, y0 + ny)
// (unwrapped), nx ny copies.
__device__ __forceinline__ void col_span(const ColP& P, int base, int& x0, int& nx, int& y0, int& ny)
{
    int x1, y1;
    col_range(base & 1023, P.w / 2, P.tx, x0, x1);
    col_range((base >> 10) & 1023, P.w / 2, P.ty, y0, y1);
    nx = x1 - x0 + 1;
    ny = y1 - y0 + 1;
}

__device__ __forceinline__ int col_wrap(int b, int nb)
{
    return b < 0 ? b + nb : (b >= nb ? b - nb : b);
}

// Bin of a copy in block b: with P.nzb > 1 the copies of a block are further
// sorted by the z-bucket of their support start (P.w planes per bucket) for
// the bucketed spread; ib2 is the point's cell along z.
__device__ __forceinline__ int col_bin(const ColP& P, int b, int ib2)
{
    if (P.nzb == 1) return b;
    int z0 = ib2 - P.w / 2 + 1;
    z0 = z0 < 0 ? z0 + P.n2 : z0;
    return b * P.nzb + z0 / P.w;
}

// Copies per bin.  The lanes of a warp take their k-th copies together,
// one atomic per run of equal bins (neighbouring points along a filament
// mostly reach the same blocks).
template <typename T>
__device__ __forceinline__ void k_col_count_body(const ColP& P, const LrRec<T>* __restrict__ rec, int n,
                                                 int* __restrict__ cnt, int bid)
{
    const int i = bid * blockDim.x + threadIdx.x;
    int x0 = 0, nx = 0, y0 = 0, ny = 0, ib2 = 0;
    if (i < n) {
        const int base = rec[i].base;
        col_span(P, base, x0, nx, y0, ny);
        ib2 = (base >> 20) & 1023;
    }
    const int nk = __reduce_max_sync(0xffffffffu, nx * ny);
    for (int k = 0; k < nk; ++k) {
        int b = -1;
        if (k < nx * ny) {
            const int ky = k / nx;
            b = col_bin(P, col_wrap(x0 + (k - ky * nx), P.nbx) + P.nbx * col_wrap(y0 + ky, P.nby), ib2);
        }
        warp_rank(b, cnt);
    }
}

template <typename T>
__global__ void k_col_count(ColP P, const LrRec<T>* __restrict__ rec, int n, int* __restrict__ cnt)
{
    k_col_count_body<T>(P, rec, n, cnt, blockIdx.x);
}

// One thread per point: the 3 W kernel weights are evaluated once and written
// with the charge into pts[i]; every block its support reaches gets the pair
// (i, support start relative to the block: r0 + 128 | (r1 + 128) << 8, with
// the z support start's bucket and offset above), 8 bytes per copy instead
// of the copy's weights.
template <typename T, int W>
__device__ __forceinline__ void k_col_scatter_body(const ColP& P, const LrRec<T>* __restrict__ rec, int n,
                                                   int* __restrict__ cur, int2* __restrict__ out,
                                                   SpPt<T, W>* __restrict__ pts, int bid)
{
    const int i = bid * blockDim.x + threadIdx.x;
    constexpr int H = W / 2;
    LrRec<T> R;
    R.base = 0;
    int x0 = 0, nx = 0, y0 = 0, ny = 0;
    if (i < n) {
        R = rec[i];
        col_span(P, R.base, x0, nx, y0, ny);
    }
    const int nk = __reduce_max_sync(0xffffffffu, nx * ny);
    if (nk == 0) return;
    const int ib0 = R.base & 1023, ib1 = (R.base >> 10) & 1023;
    // z support start z0 = zs + d, zs a multiple of W: d in bits 16-19, zs in
    // bits 20-29 of the copy's entry (read by the bucketed spread)
    int zbits = 0;
    {
        int z0 = ((R.base >> 20) & 1023) - H + 1;
        z0 = z0 < 0 ? z0 + P.n2 : z0;
        zbits = ((z0 % W) << 16) | ((z0 - z0 % W) << 20);
    }
    if (i < n) {
        // weight of support point t along axis d: psi((f_d + H - 1 - t) / (W / 2))
        const T zeta = (T)P.zeta;
        const T inorm = (T)P.inorm;
        SpPt<T, W> D;
        D.base = R.base;
        D.q[0] = R.q[0];
        D.q[1] = R.q[1];
        D.q[2] = R.q[2];
#pragma unroll
        for (int t = 0; t < W; ++t) {
            D.wx[t] = kb_val((R.f[0] + (T)(H - 1 - t)) * ((T)2 / (T)W), zeta, inorm);
            D.wy[t] = kb_val((R.f[1] + (T)(H - 1 - t)) * ((T)2 / (T)W), zeta, inorm);
            D.wz[t] = kb_val((R.f[2] + (T)(H - 1 - t)) * ((T)2 / (T)W), zeta, inorm);
        }
        pts[i] = D;
    }
    for (int k = 0; k < nk; ++k) {
        const bool live = k < nx * ny;
        const int kyi = live ? k / nx : 0;
        const int bx = x0 + (k - kyi * nx), by = y0 + kyi;
        const int b = live ? col_bin(P, col_wrap(bx, P.nbx) + P.nbx * col_wrap(by, P.nby), (R.base >> 20) & 1023) : -1;
        const int p = warp_rank(b, cur);
        if (!live) continue;
        const int r1 = ib1 - H + 1 - by * P.ty;  // support start relative to the block (unwrapped block)
        const int r0 = ib0 - H + 1 - bx * P.tx;
        out[p] = make_int2(i, (r0 + 128) | ((r1 + 128) << 8) | zbits);
    }
}

template <typename T, int W>
__global__ void k_col_scatter(ColP P, const LrRec<T>* __restrict__ rec, int n, int* __restrict__ cur,
                              int2* __restrict__ out, SpPt<T, W>* __restrict__ pts)
{
    k_col_scatter_body<T, W>(P, rec, n, cur, out, pts, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Points sorted once by the z-column block of their grid cell ("home"
// block).  A CTA gathers the lists of the home blocks whose cells' supports
// reach its block: cell index ib with [ib - W/2 + 1, ib + W/2] meeting
// [b T, b T + T - 1], at most kHomeMax blocks, each once.
// ---------------------------------------------------------------------------
constexpr int kHomeMax = 64;

__device__ __forceinline__ int floor_div(int a, int b)
{
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

// Number of home ranges of block (bx, by); thread tid < nr fetches the start
// and length of range tid.
__device__ __forceinline__ int home_fetch(const SpZP& P, const int* __restrict__ cstart, int bx, int by, int H,
                                          int& rb0, int& rlen)
{
    const int Tx = P.tx, Ty = P.ty, tid = threadIdx.x;
    const int hx0 = floor_div(bx * Tx - H, Tx), hx1 = floor_div(bx * Tx + Tx + H - 2, Tx);
    const int hy0 = floor_div(by * Ty - H, Ty), hy1 = floor_div(by * Ty + Ty + H - 2, Ty);
    const int nhx = hx1 - hx0 + 1, nr = nhx * (hy1 - hy0 + 1);
    rb0 = 0;
    rlen = 0;
    if (tid < nr) {
        const int hy = hy0 + tid / nhx, hx = hx0 + tid % nhx;
        const int wx = hx < 0 ? hx + P.nbx : (hx >= P.nbx ? hx - P.nbx : hx);
        const int wy = hy < 0 ? hy + P.nby : (hy >= P.nby ? hy - P.nby : hy);
        const int b = wx + P.nbx * wy;
        rb0 = cstart[b];
        rlen = cstart[b + 1] - rb0;
    }
    return nr;
}

// After the fetched starts and lengths were stored (r_beg[r], r_pre[r + 1])
// and a barrier: warp 0 turns the lengths into the prefix r_pre[0..64].
__device__ __forceinline__ void home_prefix(int* r_pre)
{
    const int lane = threadIdx.x & 31;
    if ((threadIdx.x >> 5) != 0) return;
    int v0 = r_pre[lane + 1], v1 = r_pre[lane + 33];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u0 = __shfl_up_sync(0xffffffffu, v0, o), u1 = __shfl_up_sync(0xffffffffu, v1, o);
        if (lane >= o) {
            v0 += u0;
            v1 += u1;
        }
    }
    v1 += __shfl_sync(0xffffffffu, v0, 31);
    r_pre[lane + 1] = v0;
    r_pre[lane + 33] = v1;
    if (lane == 0) r_pre[0] = 0;
}

// Support start of a point relative to a block (cell index ib, block start
// b0, block width T, grid n), for the periodic image that meets the block.
__device__ __forceinline__ int home_rel(int ib, int H, int b0, int T, int n, int W)
{
    int r = ib - H + 1 - b0;
    return r > T - 1 ? r - n : (r + W - 1 < 0 ? r + n : r);
}

// Eight consecutive complex values v[8q .. 8q+7] of a row of nk (entries at
// or past nk are left unset): 16-byte loads for float32 rows of an even
// length (16-byte aligned), else one load per value.
template <typename C>
__device__ __forceinline__ void load8(const C* __restrict__ row, int nk, int q, C* v)
{
    if (sizeof(C) == 8 && (nk & 1) == 0 && 8 * q + 8 <= nk) {
        const float4* r4 = reinterpret_cast<const float4*>(row + 8 * q);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 u = r4[k];
            v[2 * k].x = u.x;
            v[2 * k].y = u.y;
            v[2 * k + 1].x = u.z;
            v[2 * k + 1].y = u.w;
        }
    } else {
#pragma unroll
        for (int d = 0; d < 8; ++d)
            if (8 * q + d < nk) v[d] = row[8 * q + d];
    }
}

// Zeroes n complex values of shared memory (16-byte stores for float32
// when n is even; the buffer is 16-byte aligned).
template <typename C>
__device__ __forceinline__ void zero_cx(C* buf, int n)
{
    if (sizeof(C) == 8 && (n & 1) == 0) {
        float4* b4 = reinterpret_cast<float4*>(buf);
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int i = threadIdx.x; i < n / 2; i += blockDim.x) b4[i] = z;
    } else {
        C zero;
        zero.x = 0;
        zero.y = 0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) buf[i] = zero;
    }
}

// Separates the two real transforms of every complex z-line of a spread
// block and writes modes 0..K2.  A thread takes 8 consecutive modes of one
// line: with the lanes on consecutive groups, the digit-reversed positions
// of one instruction fall in distinct banks.
template <typename T>
__device__ __forceinline__ void spz_unpack(const SpZP& P, const typename Cx<T>::t* cb, typename Cx<T>::t* F1,
                                           int bx, int by)
{
    using C = typename Cx<T>::t;
    const int Tx = P.tx, Ty = P.ty, n2 = P.ng[2], CS = P.cls;
    const int txy = Tx * Ty, nreal = 3 * txy, tid = threadIdx.x;
    const int nk = P.K[2] + 1;
    const int nq = (nk + 7) >> 3;
    for (int i = tid; i < nreal * nq; i += blockDim.x) {
        const int rl = i / nq, q = i - rl * nq;
        const int l = rl >> 1;
        const int c = fdiv(rl, P.d_txy), rem = rl - c * txy;
        const int lx = fdiv(rem, P.d_ty), ly = rem - lx * Ty;
        const int x = bx * Tx + lx, y = by * Ty + ly;
        C* dst = F1 + (((size_t)c * P.ng[0] + x) * P.ng[1] + y) * nk;
        const Rev8 rb = rev8_bases(P.rev, P.plan2, q);
        C o[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int mz = 8 * q + d;
            if (mz >= nk) break;
            const C zk = cb[l * CS + rev8_pos(rb, P.rev, mz, d)];
            const C zn = cb[l * CS + rev8_neg(rb, P.rev, n2, mz, d)];
            if ((rl & 1) == 0) {  // A_k = (Z_k + conj Z_{n-k}) / 2
                o[d].x = (T)0.5 * (zk.x + zn.x);
                o[d].y = (T)0.5 * (zk.y - zn.y);
            } else {              // B_k = (Z_k - conj Z_{n-k}) / (2i)
                o[d].x = (T)0.5 * (zk.y + zn.y);
                o[d].y = (T)0.5 * (zn.x - zk.x);
            }
        }
        if (sizeof(C) == 8 && (nk & 1) == 0 && 8 * q + 8 <= nk) {
            // two modes per 16-byte store (rows of an even mode count are 16-byte aligned)
            float4* d4 = reinterpret_cast<float4*>(dst + 8 * q);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float4 v;
                v.x = (float)o[2 * k].x;
                v.y = (float)o[2 * k].y;
                v.z = (float)o[2 * k + 1].x;
                v.w = (float)o[2 * k + 1].y;
                d4[k] = v;
            }
        } else {
#pragma unroll
            for (int d = 0; d < 8; ++d)
                if (8 * q + d < nk) dst[8 * q + d] = o[d];
        }
    }
}

// Bytes of a block's complex z-lines in shared memory, rounded up to 16 so
// that the record buffer after them takes 16-byte copies (an odd count of
// float32 lines at an odd stride would leave it 8-byte aligned).
template <typename T>
__host__ __device__ __forceinline__ size_t zlines_bytes(int ncl, int cls)
{
    return ((size_t)ncl * cls * 2 * sizeof(T) + 15) & ~(size_t)15;
}

// ---------------------------------------------------------------------------
// A: spread + z real FFT.
// The 3 Tx Ty real z-lines are accumulated directly as complex lines (real
// line 2l in .x, 2l+1 in .y of complex line l, stride cls), transformed in
// place, and separated while writing modes 0..K2.  The block's sources come
// as (index into the per-source records of charge and weights, support
// start relative to the block) pairs written by the binning; a chunk of
// records is gathered into shared memory with asynchronous copies,
// double-buffered (the next chunk's copies are in flight while the warps add
// the current one; each staging thread holds its next entry a chunk ahead),
// and dealt to the warps round-robin.  A lane owns one (local y column, z
// support point) slot and walks the block's x columns, so a warp's lanes
// always hold distinct cells; shared atomic adds resolve two warps meeting
// on a cell.
// ---------------------------------------------------------------------------
// Bucketed record loop.  The block's copies come sorted by the z-bucket of
// their support start (W planes per bucket, col_bin).  Warp wid takes an
// equal share of them in that order and gathers them, 8 at a time, into its
// own two buffers.  Lane (ly, t) holds in registers the sums of its cells
// (lx, ly, zs + t) and (lx, ly, zs + W + t), lx < TX, for the 3 components,
// zs the start of the warp's current bucket: a copy whose support starts at
// plane zs + d (0 <= d < W) reaches the first cell when t >= d (weight
// t - d), else the second (weight t - d + W), so every lane adds to one cell
// per copy.  When the warp's bucket changes the first cells are added to the
// block's lines (shared atomics: a neighbouring warp may hold the same
// cells) and the second ones take their place; a jump of more than one
// bucket adds both.  The lines see 3 TX atomic adds per lane and bucket
// instead of per lane and copy.  Needs an even Ty, Ty W <= 32 and n2 >= 2 W
// (the 2 W cells of a lane's window are distinct planes).
template <typename T, int W, int TX>
__device__ __forceinline__ void spread_bucketed(const SpZP& P, int s0, int s1, const int2* __restrict__ cidx,
                                                const SpPt<T, W>* __restrict__ pts, SpPt<T, W>* sbuf, T* accf)
{
    constexpr int RCW = kSpzWarpChunk;
    constexpr int kWords = (int)(sizeof(SpPt<T, W>) / 16);
    constexpr int kIt = (RCW * kWords + 31) / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int n2 = P.ng[2], Ty = P.ty, CS = P.cls;
    const int sx = Ty * CS, sc = TX * Ty * CS;  // float offsets of lx + 1 and of component c + 1
    const long long n = s1 - s0;
    const int e0 = s0 + (int)((wid * n) / nw), e1 = s0 + (int)(((wid + 1) * n) / nw);
    if (e0 >= e1) return;
    SpPt<T, W>* wb = sbuf + wid * 2 * RCW;
    const int ly = lane / W, t = lane - ly * W;
    const bool slot = lane < Ty * W;
    const int ab0 = ((ly >> 1) * CS) * 2 + (ly & 1);  // float offset of (lx 0, ly, z 0, component 0)
    T lo[TX][3], hi[TX][3];
#pragma unroll
    for (int a = 0; a < TX; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            lo[a][c] = 0;
            hi[a][c] = 0;
        }
    auto flush = [&](const T (&v)[TX][3], int z) {
        z = z >= n2 ? z - n2 : z;
        if (slot) {
            const int ab = ab0 + 2 * z;
#pragma unroll
            for (int a = 0; a < TX; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c) atomicAdd(&accf[ab + a * sx + c * sc], v[a][c]);
        }
    };
    // gathers the copies [c0, min(c0 + RCW, e1)) into buffer b; lane k < RCW
    // keeps copy k's relative support start
    auto stage = [&](int b, int c0) {
        const int2 e = (lane < RCW && c0 + lane < e1) ? __ldg(cidx + c0 + lane) : make_int2(-1, 0);
#pragma unroll
        for (int k = 0; k < kIt; ++k) {
            const int wd = lane + 32 * k;
            const int r = wd / kWords;
            const int src = __shfl_sync(0xffffffffu, e.x, r < RCW ? r : 0);
            if (wd < RCW * kWords && src >= 0) {
                const int4* g = reinterpret_cast<const int4*>(pts + src) + (wd - r * kWords);
                int4* d = reinterpret_cast<int4*>(wb + b * RCW + r) + (wd - r * kWords);
                const unsigned sa = (unsigned)__cvta_generic_to_shared(d);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
            }
        }
        cp_async_commit();
        return e.y;
    };
    int zs = -1;  // start of the warp's current bucket (none yet)
    int relc = stage(0, e0);
    for (int c0 = e0, it = 0; c0 < e1; c0 += RCW, ++it) {
        int reln = 0;
        if (c0 + RCW < e1) {
            reln = stage((it + 1) & 1, c0 + RCW);
            cp_async_wait_group<1>();
        } else {
            cp_async_wait_group<0>();
        }
        __syncwarp();
        const SpPt<T, W>* rb = wb + (it & 1) * RCW;
        const int nch = min(RCW, e1 - c0);
        for (int k = 0; k < nch; ++k) {
            const int rr = __shfl_sync(0xffffffffu, relc, k);
            const SpPt<T, W>& R = rb[k];
            const int zsb = rr >> 20;
            if (zsb != zs) {  // the same in the whole warp
                if (zs >= 0) {
                    flush(lo, zs + t);
                    if (zsb != zs + W) flush(hi, zs + W + t);
#pragma unroll
                    for (int a = 0; a < TX; ++a)
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            lo[a][c] = zsb == zs + W ? hi[a][c] : (T)0;
                            hi[a][c] = 0;
                        }
                }
                zs = zsb;
            }
            const int d = (rr >> 16) & 15;
            const int r0 = (rr & 255) - 128, jy = ly - (((rr >> 8) & 255) - 128);
            if (slot && (unsigned)jy < (unsigned)W) {
                const bool first = t >= d;
                const int tz = (W & (W - 1)) == 0 ? ((t - d) & (W - 1)) : (first ? t - d : t - d + W);
                const T wyz = R.wy[jy] * R.wz[tz];
                const T wl = first ? wyz : (T)0, wh = first ? (T)0 : wyz;
                T q0, q1, q2;
                if constexpr (sizeof(T) == 4) {
                    const float4 bq = *reinterpret_cast<const float4*>(&R);  // base, q[0..2]
                    q0 = bq.y;
                    q1 = bq.z;
                    q2 = bq.w;
                } else {
                    q0 = R.q[0];
                    q1 = R.q[1];
                    q2 = R.q[2];
                }
#pragma unroll
                for (int a = 0; a < TX; ++a) {
                    const int jx = a - r0;  // the same in the whole warp
                    if ((unsigned)jx < (unsigned)W) {
                        const T wx = R.wx[jx];
                        const T vl = wx * wl, vh = wx * wh;
                        lo[a][0] += vl * q0;
                        lo[a][1] += vl * q1;
                        lo[a][2] += vl * q2;
                        hi[a][0] += vh * q0;
                        hi[a][1] += vh * q1;
                        hi[a][2] += vh * q2;
                    }
                }
            }
        }
        __syncwarp();  // every lane is done with this buffer before it is refilled
        relc = reln;
    }
    flush(lo, zs + t);
    flush(hi, zs + W + t);
}

template <typename T, int W, int RM>
__device__ __forceinline__ void k_spread_zfft_body(const SpZP& P, const int* __restrict__ cstart,
                                                   const int2* __restrict__ cidx,
                                                   const SpPt<T, W>* __restrict__ pts,
                                                   const typename Cx<T>::t* __restrict__ tw2,
                                                   typename Cx<T>::t* __restrict__ F1, int bid)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Tx = P.tx, Ty = P.ty, n2 = P.ng[2];
    const int txy = Tx * Ty;
    const int nreal = 3 * txy;
    const int ncl = nreal / 2;
    const int CS = P.cls;
    C* cb = reinterpret_cast<C*>(smem_raw);
    T* accf = reinterpret_cast<T*>(cb);  // real line rl, position z at float ((rl>>1) CS + z) 2 + (rl&1)
    SpPt<T, W>* sbuf = reinterpret_cast<SpPt<T, W>*>(smem_raw + zlines_bytes<T>(ncl, CS));  // 2 chunks
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int by = fdiv(bid, P.d_nbx);
    const int bx = bid - by * P.nbx;
    zero_cx(cb, ncl * CS);

    constexpr int H = W / 2;
    constexpr int RC = spz_rec_chunk<T>();
    const int s0 = cstart[bid * P.nzb], s1 = cstart[(bid + 1) * P.nzb];
    const int nslot = Ty * W;
    if (P.nzb > 1) {
        __syncthreads();  // the lines are zeroed
        switch (Tx) {
        case 1: spread_bucketed<T, W, 1>(P, s0, s1, cidx, pts, sbuf, accf); break;
        case 2: spread_bucketed<T, W, 2>(P, s0, s1, cidx, pts, sbuf, accf); break;
        default: spread_bucketed<T, W, 4>(P, s0, s1, cidx, pts, sbuf, accf); break;
        }
        __syncthreads();
        fft_fwd_dif<T, RM>(cb, ncl, P.d_ncl, CS, P.plan2, tw2);
        spz_unpack<T>(P, cb, F1, bx, by);
        return;
    }
    // deterministic mode: warp wid owns z in [zlo, zhi) and adds every record
    // of the block in order (plain adds: one writer per cell, ordered sums)
    const int zlo = P.det ? (int)(((long long)wid * n2) / nw) : 0;
    const int zhi = P.det ? (int)(((long long)(wid + 1) * n2) / nw) : n2;
    // thread tid < RC gathers the record of its copy into slot tid of buffer
    // b (one group of this thread's copies; empty for the others) and writes
    // the copy's relative support start beside it; the copy's entry is
    // loaded a chunk ahead
    __shared__ int s_rel[2][RC];
    auto stage = [&](int b, int2 e) {
        if (e.x >= 0) {
            constexpr int kWords = (int)(sizeof(SpPt<T, W>) / 16);
            const int4* src = reinterpret_cast<const int4*>(pts + e.x);
            int4* dst = reinterpret_cast<int4*>(sbuf + b * RC + tid);
#pragma unroll
            for (int k = 0; k < kWords; ++k) {
                const unsigned sa = (unsigned)__cvta_generic_to_shared(dst + k);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src + k) : "memory");
            }
            s_rel[b][tid] = e.y;
        }
        cp_async_commit();
    };
    auto next_entry = [&](int c0r) {
        return (tid < RC && c0r + tid < s1) ? __ldg(cidx + c0r + tid) : make_int2(-1, 0);
    };
    int2 nxt = next_entry(s0);
    if (s0 < s1) stage(0, nxt);
    nxt = next_entry(s0 + RC);
    for (int c0r = s0, it = 0; c0r < s1; c0r += RC, ++it) {
        const int nch = min(RC, s1 - c0r);
        const SpPt<T, W>* srec = sbuf + (it & 1) * RC;
        const int* srel = s_rel[it & 1];
        __syncthreads();  // every warp is done with the buffer the next chunk goes to
        if (c0r + RC < s1) {
            stage((it + 1) & 1, nxt);
            nxt = next_entry(c0r + 2 * RC);
            cp_async_wait_group<1>();  // this chunk's copies have landed
        } else {
            cp_async_wait_group<0>();
        }
        __syncthreads();
        if (!P.det && nslot <= 32 && (Ty & 1) == 0) {
            // Fast path: every lane owns the same (y column, z offset) slot in
            // every record, so its slot indices and the parity of its real line
            // are fixed; the shared address of (lx, component c) is
            // abase + lx Ty CS + c txy CS (Ty and txy are even).
            const int ly = lane / W, t = lane - ly * W;
            const bool slot = lane < nslot;
            const int sx = Ty * CS, sc = txy * CS;
            for (int kk = wid; kk < nch; kk += nw) {
                const SpPt<T, W>& R = srec[kk];
                const int rr = srel[kk];
                const int r1 = ((rr >> 8) & 255) - 128;
                if (!slot || ly < r1 || ly > r1 + W - 1) continue;
                const int ib2 = (R.base >> 20) & 1023;
                const int r0 = (rr & 255) - 128;
                int z = ib2 - H + 1 + t;
                z = z < 0 ? z + n2 : (z >= n2 ? z - n2 : z);
                const int abase = ((ly >> 1) * CS + z) * 2 + (ly & 1);
                const T wyz = R.wy[ly - r1] * R.wz[t];
                const T q0 = R.q[0], q1 = R.q[1], q2 = R.q[2];
                const int lx0 = max(r0, 0), lx1 = min(r0 + W - 1, Tx - 1);  // the same in the whole warp
                for (int lx = lx0; lx <= lx1; ++lx) {
                    const T wv = R.wx[lx - r0] * wyz;
                    const int ad = abase + lx * sx;
                    atomicAdd(&accf[ad], wv * q0);
                    atomicAdd(&accf[ad + sc], wv * q1);
                    atomicAdd(&accf[ad + 2 * sc], wv * q2);
                }
            }
            continue;
        }
        for (int kk = P.det ? 0 : wid; kk < nch; kk += P.det ? 1 : nw) {
            const SpPt<T, W>& R = srec[kk];
            const int rr = srel[kk];
            const int ib2 = (R.base >> 20) & 1023;
            const int r0 = (rr & 255) - 128, r1 = ((rr >> 8) & 255) - 128;
            const int a0 = max(r0, 0), e0 = min(r0 + W - 1, Tx - 1);
            const int a1 = max(r1, 0), e1 = min(r1 + W - 1, Ty - 1);
            const T q0 = R.q[0], q1 = R.q[1], q2 = R.q[2];
            for (int sl = lane; sl < nslot; sl += 32) {
                const int ly = sl / W, t = sl - ly * W;
                if (ly < a1 || ly > e1) continue;
                int z = ib2 - H + 1 + t;
                z = z < 0 ? z + n2 : (z >= n2 ? z - n2 : z);
                const T wyz = R.wy[ly - r1] * R.wz[t];
                if (P.det) {
                    if (z < zlo || z >= zhi) continue;
                    for (int lx = a0; lx <= e0; ++lx) {
                        const T wv = R.wx[lx - r0] * wyz;
                        const int rl = lx * Ty + ly;
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const int rlc = rl + c * txy;
                            const T qc = c == 0 ? q0 : (c == 1 ? q1 : q2);
                            accf[((rlc >> 1) * CS + z) * 2 + (rlc & 1)] += wv * qc;
                        }
                    }
                    continue;
                }
                for (int lx = a0; lx <= e0; ++lx) {
                    const T wv = R.wx[lx - r0] * wyz;
                    const int rl = lx * Ty + ly;  // real line of component 0
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const int rlc = rl + c * txy;
                        const T qc = c == 0 ? q0 : (c == 1 ? q1 : q2);
                        atomicAdd(&accf[((rlc >> 1) * CS + z) * 2 + (rlc & 1)], wv * qc);
                    }
                }
            }
            if (P.det) __syncwarp();  // this record's adds precede the next record's
        }
    }
    __syncthreads();
    fft_fwd_dif<T, RM>(cb, ncl, P.d_ncl, CS, P.plan2, tw2);
    spz_unpack<T>(P, cb, F1, bx, by);
}

template <typename T, int W, int RM>
__global__ void __launch_bounds__(z_threads_max<T>(), 2) k_spread_zfft(SpZP P, const int* __restrict__ cstart,
                                                          const int2* __restrict__ cidx,
                                                          const SpPt<T, W>* __restrict__ pts,
                                                          const typename Cx<T>::t* __restrict__ tw2,
                                                          typename Cx<T>::t* __restrict__ F1)
{
    k_spread_zfft_body<T, W, RM>(P, cstart, cidx, pts, tw2, F1, blockIdx.x);
}

// ---------------------------------------------------------------------------
// B / D: transforms along y.  One CTA per (c, x, chunk of 2^lmc z-modes).
// forward: F1[c][x][y][mz] -> F2[c][x][my'][mz], my' = my + K1, |my| <= K1
// inverse: F2 -> F1 (zero-padded to n1)
// ---------------------------------------------------------------------------
template <typename T, int RM>
__device__ __forceinline__ void k_fft_y_tma(const FftYP& P, typename Cx<T>::t* __restrict__ F1,
                                            typename Cx<T>::t* __restrict__ F2,
                                            const typename Cx<T>::t* __restrict__ tw1, int sign, int bid,
                                            const CUtensorMap* tm, int* status);

template <typename T, int RM>
__device__ __forceinline__ void k_fft_y_body(const FftYP& P, typename Cx<T>::t* __restrict__ F1,
                                             typename Cx<T>::t* __restrict__ F2,
                                             const typename Cx<T>::t* __restrict__ tw1, int sign, int bid,
                                             const CUtensorMap* tm = nullptr, int* status = nullptr)
{
    if (tm) {
        k_fft_y_tma<T, RM>(P, F1, F2, tw1, sign, bid, tm, status);
        return;
    }
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = P.ng[1], K1 = P.K[1], nk = P.K[2] + 1;
    const int lmc = P.lmc, MC = 1 << lmc;
    const int LS = P.ls;
    C* a = reinterpret_cast<C*>(smem_raw);
    const int nch = (nk + MC - 1) >> lmc;
    const int cx = fdiv(bid, P.d_nch);  // c * n0 + x
    const int ch = bid - cx * nch;
    const int mz0 = ch << lmc;
    const int mcount = min(MC, nk - mz0);
    const int ny2 = 2 * K1 + 1;
    C zero;
    zero.x = 0;
    zero.y = 0;
    // MC divides the block: every thread keeps one mode l and walks the lines'
    // positions with a fixed step, so the global addresses advance by a
    // pointer increment instead of a 64-bit index product per element.
    const int l = threadIdx.x & (MC - 1);
    const int r0 = threadIdx.x >> lmc, rstep = blockDim.x >> lmc;
    const bool live = l < mcount;
    C* const al = a + l * LS;
    if (sign < 0) {
        const C* src = F1 + ((size_t)cx * n1 + r0) * nk + mz0 + l;
        const size_t sstep = (size_t)rstep * nk;
        for (int y = r0; y < n1; y += rstep, src += sstep) {
            if (live)
                cp_async_cx(&al[y], src);
            else
                al[y] = zero;
        }
        cp_async_wait_all();
        __syncthreads();
        fft_fwd_dif<T, RM>(a, MC, P.d_lines, LS, P.plan1, tw1);
        if (live) {
            C* dst = F2 + ((size_t)cx * ny2 + r0) * nk + mz0 + l;
            for (int myp = r0; myp < ny2; myp += rstep, dst += sstep) {
                const int my = myp - K1;
                *dst = al[P.rev[my < 0 ? my + n1 : my]];
            }
        }
    } else {
        const C* src = F2 + ((size_t)cx * ny2) * nk + mz0 + l;
        for (int y = r0; y < n1; y += rstep) {  // y: frequency index
            const int my = y <= n1 / 2 ? y : y - n1;
            C* d = &al[P.rev[y]];
            if (live && my >= -K1 && my <= K1)
                cp_async_cx(d, src + (size_t)(my + K1) * nk);
            else
                *d = zero;
        }
        cp_async_wait_all();
        __syncthreads();
        fft_inv_dit<T, RM>(a, MC, P.d_lines, LS, P.plan1, tw1);
        if (live) {
            C* dst = F1 + ((size_t)cx * n1 + r0) * nk + mz0 + l;
            const size_t dstep = (size_t)rstep * nk;
            for (int y = r0; y < n1; y += rstep, dst += dstep) *dst = al[y];
        }
    }
}

// The y pass with the F1 rows moved by tensor copies (tnb > 0).  The CTA's
// line set (the MC modes mz0.. of the n1 rows of one (c, x)) sits mode-major
// in shared memory, row y at y MC: exactly the layout of tnb boxes of tby
// rows of 2 MC reals.  Forward: one thread issues the boxes (rows past n1
// and modes past K2 arrive as zeros) and the block waits on an mbarrier,
// then transforms and writes the |my| <= K1 rows of F2 (thread per mode,
// digit-reversed rows).  Inverse: the F2 rows are gathered with per-element
// asynchronous copies into their digit-reversed rows (the zero padding
// written directly), transformed, and one thread stores the natural-order
// rows with tensor copies (rows past n1, modes past K2 are not written).
template <typename T, int RM>
__device__ __forceinline__ void k_fft_y_tma(const FftYP& P, typename Cx<T>::t* __restrict__ F1,
                                            typename Cx<T>::t* __restrict__ F2,
                                            const typename Cx<T>::t* __restrict__ tw1, int sign, int bid,
                                            const CUtensorMap* tm, int* status)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long s_bar;
    C* a = reinterpret_cast<C*>(smem_align128(smem_raw));
    const int n1 = P.ng[1], K1 = P.K[1], nk = P.K[2] + 1;
    const int lmc = P.lmc, MC = 1 << lmc;
    const int nch = (nk + MC - 1) >> lmc;
    const int cx = fdiv(bid, P.d_nch);  // c * n0 + x
    const int ch = bid - cx * nch;
    const int mz0 = ch << lmc;
    const int mcount = min(MC, nk - mz0);
    const int ny2 = 2 * K1 + 1;
    const int l = threadIdx.x & (MC - 1);
    const int r0 = threadIdx.x >> lmc, rstep = blockDim.x >> lmc;
    const bool live = l < mcount;
    const int boxc = P.tby * MC;  // complex values per box
    if (sign < 0) {
        if (threadIdx.x == 0) mbar_init(&s_bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_expect_tx(&s_bar, (unsigned)(P.tnb * boxc * sizeof(C)));
            for (int b = 0; b < P.tnb; ++b) tma_load_3d(a + (size_t)b * boxc, tm, 2 * mz0, b * P.tby, cx, &s_bar);
        }
        if (!mbar_wait_bounded(&s_bar, 0)) {
            if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
            return;
        }
        fft_fwd_dif<T, RM, true>(a, MC, P.d_lines, 0, P.plan1, tw1);
        if (live) {
            C* dst = F2 + ((size_t)cx * ny2 + r0) * nk + mz0 + l;
            const size_t dstep = (size_t)rstep * nk;
            for (int myp = r0; myp < ny2; myp += rstep, dst += dstep) {
                const int my = myp - K1;
                *dst = a[P.rev[my < 0 ? my + n1 : my] * MC + l];
            }
        }
    } else {
        C zero;
        zero.x = 0;
        zero.y = 0;
        const C* src = F2 + ((size_t)cx * ny2) * nk + mz0 + l;
        for (int y = r0; y < n1; y += rstep) {  // y: frequency index
            const int my = y <= n1 / 2 ? y : y - n1;
            C* d = &a[P.rev[y] * MC + l];
            if (live && my >= -K1 && my <= K1)
                cp_async_cx(d, src + (size_t)(my + K1) * nk);
            else
                *d = zero;
        }
        cp_async_wait_all();
        __syncthreads();
        fft_inv_dit<T, RM, true>(a, MC, P.d_lines, 0, P.plan1, tw1);
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int b = 0; b < P.tnb; ++b) tma_store_3d(tm, 2 * mz0, b * P.tby, cx, a + (size_t)b * boxc);
            tma_store_commit_and_wait_read();
        }
    }
}

template <typename T, int RM>
__global__ void __launch_bounds__(kThreads, 2) k_fft_y(FftYP P, typename Cx<T>::t* __restrict__ F1,
                                                    typename Cx<T>::t* __restrict__ F2,
                                                    const typename Cx<T>::t* __restrict__ tw1, int sign,
                                                    const __grid_constant__ CUtensorMap tm, int* status)
{
    k_fft_y_body<T, RM>(P, F1, F2, tw1, sign, blockIdx.x, P.tnb > 0 ? &tm : nullptr, status);
}

// ---------------------------------------------------------------------------
// C: x forward FFT + k-space pass + x inverse FFT, in place on F2.
// One CTA per (my', chunk of 2^lmc z-modes); the 3 components together (the
// curl couples them).  tabs: e^{-k_d^2/4alpha^2} / F_d(m)^2 per axis.
// ---------------------------------------------------------------------------
template <typename T, int RM>
__device__ __forceinline__ void k_fft_x_kspace_body(const FftXP& P, typename Cx<T>::t* __restrict__ F2,
                                                    typename Cx<T>::t* __restrict__ F2psi,
                                                    const typename Cx<T>::t* __restrict__ tw0,
                                                    const T* __restrict__ tab0, const T* __restrict__ tab1,
                                                    const T* __restrict__ tab2, int bid)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n0 = P.ng[0], K0 = P.K[0], K1 = P.K[1], nk = P.K[2] + 1;
    const int lmc = P.lmc, MC = 1 << lmc;
    const int ny2 = 2 * K1 + 1;
    const int LS = P.ls;
    const int want_psi = F2psi != nullptr;
    C* a = reinterpret_cast<C*>(smem_raw);  // lines [comp][mz], psi lines follow
    const int nch = (nk + MC - 1) >> lmc;
    const int myp = fdiv(bid, P.d_nch);
    const int ch = bid - myp * nch;
    const int mz0 = ch << lmc;
    const int mcount = min(MC, nk - mz0);
    C zero;
    zero.x = 0;
    zero.y = 0;
    // the MC modes of one (c, x) are adjacent in F2: lanes on them first, so a
    // warp reads whole 32-byte sectors.  MC divides the block, so a thread
    // keeps its mode l and steps x by a fixed amount (pointer increments).
    const int l = threadIdx.x & (MC - 1);
    const int x0 = threadIdx.x >> lmc, xstep = blockDim.x >> lmc;
    const bool live = l < mcount;
    const size_t gstep = (size_t)xstep * ny2 * nk;
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        C* const al = a + ((c << lmc) + l) * LS;
        const C* src = F2 + (((size_t)c * n0 + x0) * ny2 + myp) * nk + mz0 + l;
        for (int x = x0; x < n0; x += xstep, src += gstep) {
            if (live)
                cp_async_cx(&al[x], src);
            else
                al[x] = zero;
        }
    }
    cp_async_wait_all();
    __syncthreads();
    fft_fwd_dif<T, RM>(a, 3 * MC, P.d_lines, LS, P.plan0, tw0);
    // k-space pass: frequency (mx, my, mz) sits at position rev(xi) of line (c, l)
    const int my = myp - K1;
    const int amy = my < 0 ? -my : my;
    if (P.spectrum) {
        // energy spectrum (Eq. def_energy_spectrum): shell sums in shared memory
        double* bins = reinterpret_cast<double*>(a + (size_t)3 * MC * LS);
        for (int i = threadIdx.x; i < P.nbins; i += blockDim.x) bins[i] = 0.0;
        __syncthreads();
        const double kk0 = P.kk[0], kk1 = P.kk[1], kk2 = P.kk[2];
        const double sg = P.smoothed ? -P.inv4a2 : P.inv4a2;
        for (int i = threadIdx.x; i < (n0 << lmc); i += blockDim.x) {
            const int lk = i & (MC - 1), xi = i >> lmc;
            const int mx = xi <= n0 / 2 ? xi : xi - n0;
            const int amx = mx < 0 ? -mx : mx;
            const int mz = mz0 + lk;
            if (lk >= mcount || amx > K0 || (mx == 0 && my == 0 && mz == 0)) continue;
            const int pos = P.rev[xi];
            const C F0 = a[(0 * MC + lk) * LS + pos], F1 = a[(1 * MC + lk) * LS + pos],
                    F2v = a[(2 * MC + lk) * LS + pos];
            const double k0 = kk0 * mx, k1 = kk1 * my, k2 = kk2 * mz;
            const double ksq = k0 * k0 + k1 * k1 + k2 * k2;
            // |k x F|^2 = |k x Re F|^2 + |k x Im F|^2
            const double ar0 = k1 * F2v.x - k2 * F1.x, ar1 = k2 * F0.x - k0 * F2v.x, ar2 = k0 * F1.x - k1 * F0.x;
            const double ai0 = k1 * F2v.y - k2 * F1.y, ai1 = k2 * F0.y - k0 * F2v.y, ai2 = k0 * F1.y - k1 * F0.y;
            const double c2 = ar0 * ar0 + ar1 * ar1 + ar2 * ar2 + ai0 * ai0 + ai1 * ai1 + ai2 * ai2;
            const double tp = (double)tab0[amx] * (double)tab1[amy] * (double)tab2[mz];
            const double v = (mz > 0 ? 2.0 : 1.0) * c2 * tp * exp(sg * ksq) / (ksq * ksq);
            const int m = (int)(sqrt(ksq) / P.dk + 0.5);
            if (m < P.nbins) atomicAdd(&bins[m], v);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < P.nbins; i += blockDim.x)
            if (bins[i] != 0.0) atomicAdd(&P.spectrum[i], bins[i]);
        return;
    }
    double esum = 0.0;  // energy of this thread's modes (float64 reduction)
    // a thread takes 8 consecutive x frequencies of one line, the lanes on
    // consecutive groups (distinct banks at the digit-reversed positions)
    const int nq = n0 >> 3;
    const T kk0 = (T)P.kk[0], kk1 = (T)P.kk[1], kk2 = (T)P.kk[2];  // 2 pi / L_d
    const T scale = (T)P.scale;
    for (int i = threadIdx.x; i < nq * MC; i += blockDim.x) {
        const int lk = i / nq, q = i - lk * nq;
        const int mz = mz0 + lk;
        const Rev8 rb = rev8_bases(P.rev, P.plan0, q);
#pragma unroll 2
        for (int d = 0; d < 8; ++d) {
            const int xi = 8 * q + d;
            const int mx = xi <= n0 / 2 ? xi : xi - n0;
            const int amx = mx < 0 ? -mx : mx;
            const int pos = rev8_pos(rb, P.rev, xi, d);
            C* r0 = a + ((0 * MC + lk) * LS + pos);
            C* r1 = a + ((1 * MC + lk) * LS + pos);
            C* r2 = a + ((2 * MC + lk) * LS + pos);
            if (lk >= mcount || amx > K0 || (mx == 0 && my == 0 && mz == 0)) {
                *r0 = zero;
                *r1 = zero;
                *r2 = zero;
                if (want_psi) {
                    a[(3 * MC + lk) * LS + pos] = zero;
                    a[(4 * MC + lk) * LS + pos] = zero;
                    a[(5 * MC + lk) * LS + pos] = zero;
                }
                continue;
            }
            C w0 = *r0, w1 = *r1, w2 = *r2;
            const T k0 = kk0 * (T)mx, k1 = kk1 * (T)my, k2 = kk2 * (T)mz;
            const T ksq = k0 * k0 + k1 * k1 + k2 * k2;
            const T mult = scale * tab0[amx] * tab1[amy] * tab2[mz] / ksq;
            if (P.energy) {
                // (1/2) e^{-k^2/4a^2} |omega|^2 / k^2 = (kappa/V) mult |F|^2 / 2; the
                // half spectrum holds the pair (k, -k) once when mz > 0
                const double f2 = (double)w0.x * w0.x + (double)w0.y * w0.y + (double)w1.x * w1.x +
                                  (double)w1.y * w1.y + (double)w2.x * w2.x + (double)w2.y * w2.y;
                esum += (mz > 0 ? 1.0 : 0.5) * P.scale * (double)mult * f2;
            }
            w0.x *= mult; w0.y *= mult;
            w1.x *= mult; w1.y *= mult;
            w2.x *= mult; w2.y *= mult;
            // i k x w
            const T cr0 = k1 * w2.x - k2 * w1.x, ci0 = k1 * w2.y - k2 * w1.y;
            const T cr1 = k2 * w0.x - k0 * w2.x, ci1 = k2 * w0.y - k0 * w2.y;
            const T cr2 = k0 * w1.x - k1 * w0.x, ci2 = k0 * w1.y - k1 * w0.y;
            C o;
            o.x = -ci0; o.y = cr0; *r0 = o;
            o.x = -ci1; o.y = cr1; *r1 = o;
            o.x = -ci2; o.y = cr2; *r2 = o;
            if (want_psi) {
                a[(3 * MC + lk) * LS + pos] = w0;
                a[(4 * MC + lk) * LS + pos] = w1;
                a[(5 * MC + lk) * LS + pos] = w2;
            }
        }
    }
    if (P.energy) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) esum += __shfl_xor_sync(0xffffffffu, esum, o);
        if (P.epart) {
            // deterministic: warp sums in warp order, one partial per CTA
            double* wsum = reinterpret_cast<double*>(a + (size_t)(want_psi ? 6 : 3) * MC * LS);
            __syncthreads();
            if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = esum;
            __syncthreads();
            if (threadIdx.x == 0) {
                double t = 0.0;
                for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += wsum[k];
                P.epart[bid] = t;
            }
        } else if ((threadIdx.x & 31) == 0 && esum != 0.0) {
            atomicAdd(P.energy, esum);
        }
    }
    __syncthreads();
    fft_inv_dit<T, RM>(a, (want_psi ? 6 : 3) * MC, want_psi ? P.d_lines_psi : P.d_lines, LS, P.plan0, tw0);
    if (live) {
#pragma unroll 1
        for (int c = 0; c < 3; ++c) {
            const C* al = a + ((c << lmc) + l) * LS;
            const C* ap = a + (((3 + c) << lmc) + l) * LS;
            const size_t g0 = (((size_t)c * n0 + x0) * ny2 + myp) * nk + mz0 + l;
            C* dst = F2 + g0;
            C* dpsi = want_psi ? F2psi + g0 : nullptr;
            for (int x = x0; x < n0; x += xstep, dst += gstep) {
                *dst = al[x];
                if (want_psi) {
                    *dpsi = ap[x];
                    dpsi += gstep;
                }
            }
        }
    }
}

// The x pass of the velocity (no psi, spectrum or deterministic energy) with
// F2 moved by tensor copies (tnbx > 0).  The boxes land as x rows of the
// 3 MC lines' modes (line c MC + l, mode-major: x row at x 3 MC), the forward
// transform runs on that layout, the k-space pass walks positions (a thread
// per (position, mode), the frequency from the inverse digit-reversal
// table, so that consecutive lanes read consecutive words), the inverse
// transform returns natural order and one thread stores the rows back.
// Modes past K2 arrive as zeros and are not written back.
template <typename T, int RM>
__device__ __forceinline__ void k_fft_x_tma(const FftXP& P, typename Cx<T>::t* __restrict__ F2,
                                            const typename Cx<T>::t* __restrict__ tw0, const T* __restrict__ tab0,
                                            const T* __restrict__ tab1, const T* __restrict__ tab2, int bid,
                                            const CUtensorMap* tm, int* status)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long s_bar;
    C* a = reinterpret_cast<C*>(smem_align128(smem_raw));
    const int n0 = P.ng[0], K0 = P.K[0], K1 = P.K[1], nk = P.K[2] + 1;
    const int lmc = P.lmc, MC = 1 << lmc, NL = 3 * MC;
    const int nch = (nk + MC - 1) >> lmc;
    const int myp = fdiv(bid, P.d_nch);
    const int ch = bid - myp * nch;
    const int mz0 = ch << lmc;
    const int mcount = min(MC, nk - mz0);
    const int boxc = P.tbx * NL;  // complex values per box
    if (threadIdx.x == 0) mbar_init(&s_bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(&s_bar, (unsigned)(P.tnbx * boxc * sizeof(C)));
        for (int b = 0; b < P.tnbx; ++b)
            tma_load_4d(a + (size_t)b * boxc, tm, 2 * mz0, 0, b * P.tbx, myp, &s_bar);
    }
    if (!mbar_wait_bounded(&s_bar, 0)) {
        if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
        return;
    }
    fft_fwd_dif<T, RM, true>(a, NL, P.d_lines, 0, P.plan0, tw0);
    // k-space pass: frequency (mx, my, mz) of line (c, lk) sits at position
    // p with irev[p] = xi
    const int my = myp - K1;
    const int amy = my < 0 ? -my : my;
    double esum = 0.0;
    const T kk0 = (T)P.kk[0], kk1 = (T)P.kk[1], kk2 = (T)P.kk[2];
    const T scale = (T)P.scale;
    C zero;
    zero.x = 0;
    zero.y = 0;
    for (int i = threadIdx.x; i < (n0 << lmc); i += blockDim.x) {
        const int lk = i & (MC - 1), p = i >> lmc;
        const int xi = P.irev[p];
        const int mx = xi <= n0 / 2 ? xi : xi - n0;
        const int amx = mx < 0 ? -mx : mx;
        const int mz = mz0 + lk;
        C* r = a + (size_t)p * NL + lk;  // component c at r[c MC]
        if (lk >= mcount || amx > K0 || (mx == 0 && my == 0 && mz == 0)) {
            r[0] = zero;
            r[MC] = zero;
            r[2 * MC] = zero;
            continue;
        }
        C w0 = r[0], w1 = r[MC], w2 = r[2 * MC];
        const T k0 = kk0 * (T)mx, k1 = kk1 * (T)my, k2 = kk2 * (T)mz;
        const T ksq = k0 * k0 + k1 * k1 + k2 * k2;
        const T mult = scale * tab0[amx] * tab1[amy] * tab2[mz] / ksq;
        if (P.energy) {
            const double f2 = (double)w0.x * w0.x + (double)w0.y * w0.y + (double)w1.x * w1.x +
                              (double)w1.y * w1.y + (double)w2.x * w2.x + (double)w2.y * w2.y;
            esum += (mz > 0 ? 1.0 : 0.5) * P.scale * (double)mult * f2;
        }
        w0.x *= mult; w0.y *= mult;
        w1.x *= mult; w1.y *= mult;
        w2.x *= mult; w2.y *= mult;
        // i k x w
        const T cr0 = k1 * w2.x - k2 * w1.x, ci0 = k1 * w2.y - k2 * w1.y;
        const T cr1 = k2 * w0.x - k0 * w2.x, ci1 = k2 * w0.y - k0 * w2.y;
        const T cr2 = k0 * w1.x - k1 * w0.x, ci2 = k0 * w1.y - k1 * w0.y;
        C o;
        o.x = -ci0; o.y = cr0; r[0] = o;
        o.x = -ci1; o.y = cr1; r[MC] = o;
        o.x = -ci2; o.y = cr2; r[2 * MC] = o;
    }
    if (P.energy) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) esum += __shfl_xor_sync(0xffffffffu, esum, o);
        if ((threadIdx.x & 31) == 0 && esum != 0.0) atomicAdd(P.energy, esum);
    }
    __syncthreads();
    fft_inv_dit<T, RM, true>(a, NL, P.d_lines, 0, P.plan0, tw0);
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int b = 0; b < P.tnbx; ++b) tma_store_4d(tm, 2 * mz0, 0, b * P.tbx, myp, a + (size_t)b * boxc);
        tma_store_commit_and_wait_read();
    }
}

template <typename T, int RM>
__global__ void __launch_bounds__(z_threads_max<T>(), 2) k_fft_x_kspace(FftXP P, typename Cx<T>::t* __restrict__ F2,
                                                           typename Cx<T>::t* __restrict__ F2psi,
                                                           const typename Cx<T>::t* __restrict__ tw0,
                                                           const T* __restrict__ tab0, const T* __restrict__ tab1,
                                                           const T* __restrict__ tab2,
                                                           const __grid_constant__ CUtensorMap tm, int* status)
{
    if (P.tnbx > 0)
        k_fft_x_tma<T, RM>(P, F2, tw0, tab0, tab1, tab2, blockIdx.x, &tm, status);
    else
        k_fft_x_kspace_body<T, RM>(P, F2, F2psi, tw0, tab0, tab1, tab2, blockIdx.x);
}

// ---------------------------------------------------------------------------
// E: inverse z real FFT.  One CTA per (c, x, chunk of YC y-lines); two real
// lines per complex transform.
// ---------------------------------------------------------------------------
template <typename T, int RM, typename TO>
__global__ void __launch_bounds__(kThreads, 2) k_fft_z_c2r(FftZP P, const typename Cx<T>::t* __restrict__ F1,
                                                        const typename Cx<T>::t* __restrict__ tw2,
                                                        TO* __restrict__ grid)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n1 = P.ng[1], n2 = P.ng[2], nk = P.K[2] + 1, YC = P.yc;
    const int ncl = YC / 2;
    const int CS = P.cls;
    C* a = reinterpret_cast<C*>(smem_raw);
    const int nch = n1 / YC;
    const int cx = fdiv(blockIdx.x, P.d_nch);  // c * n0 + x
    const int ch = blockIdx.x - cx * nch;
    const int y0 = ch * YC;
    C zero;
    zero.x = 0;
    zero.y = 0;
    for (int i = threadIdx.x; i < ncl * CS; i += blockDim.x) a[i] = zero;
    __syncthreads();
    // Z_k = A_k + i B_k, Z_{n-k} = conj(A_k) + i conj(B_k), k = 0..K2, at rev
    // positions; a thread takes 8 consecutive k of one line pair (distinct
    // banks per instruction, 16 loads in flight)
    const int nq = (nk + 7) >> 3;
    for (int i = threadIdx.x; i < ncl * nq; i += blockDim.x) {
        const int l = i / nq, q = i - l * nq;
        const C* rowA = F1 + ((size_t)cx * n1 + y0 + 2 * l) * nk;
        const C* rowB = rowA + nk;
        C A[8], Bv[8];
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int k = 8 * q + d;
            if (k < nk) {
                A[d] = rowA[k];
                Bv[d] = rowB[k];
            }
        }
        const Rev8 rb = rev8_bases(P.rev, P.plan2, q);
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int k = 8 * q + d;
            if (k >= nk) break;
            C z;
            if (k == 0) {
                z.x = A[d].x;
                z.y = Bv[d].x;
                a[l * CS] = z;
            } else {
                z.x = A[d].x - Bv[d].y;
                z.y = A[d].y + Bv[d].x;
                a[l * CS + rev8_pos(rb, P.rev, k, d)] = z;
                z.x = A[d].x + Bv[d].y;
                z.y = -A[d].y + Bv[d].x;
                a[l * CS + rev8_neg(rb, P.rev, n2, k, d)] = z;
            }
        }
    }
    __syncthreads();
    fft_inv_dit<T, RM>(a, ncl, P.d_ncl, CS, P.plan2, tw2);
    const size_t gsz = (size_t)P.ng[0] * n1 * n2;
    const int c = fdiv(cx, P.d_n0), x = cx - c * P.ng[0];
    TO* gout = grid + c * gsz + ((size_t)x * n1 + y0) * n2;
    // the CTA's YC rows of n2 reals are contiguous in the grid; a thread reads
    // two adjacent complex values of line l and writes the pair to each of the
    // real rows 2l and 2l + 1 (n2 is even)
    using T2 = typename Cx<TO>::t;
    const int h2 = n2 >> 1;
    for (int i = threadIdx.x; i < ncl * h2; i += blockDim.x) {
        const int l = i / h2, zz = i - l * h2;
        const C v0 = a[l * CS + 2 * zz], v1 = a[l * CS + 2 * zz + 1];
        T2 ra, rbv;
        ra.x = v0.x;
        ra.y = v1.x;
        rbv.x = v0.y;
        rbv.y = v1.y;
        *reinterpret_cast<T2*>(gout + (size_t)(2 * l) * n2 + 2 * zz) = ra;
        *reinterpret_cast<T2*>(gout + (size_t)(2 * l + 1) * n2 + 2 * zz) = rbv;
    }
}

// ---------------------------------------------------------------------------
// E': inverse z real FFT fused with the interpolation of the velocity at the
// nodes (the type-2 step of Eq. long_range_velocity_interp).  One CTA per
// Tx x Ty block of z-columns with all three components, as in the spread:
// the modes 0..K2 of the 3 Tx Ty real lines are read two lines per complex
// line (real line 2l in .x, 2l+1 in .y; with Ty even the pair is two
// adjacent y rows of one (c, x)), transformed in place, and the nodes whose
// support reaches the block then take their weighted sums straight from
// shared memory, so the real grid is never written.  The nodes are sorted
// once by the block of their grid cell; a CTA gathers the few neighbouring
// blocks' lists (in flight while its lines are transformed).  A node's W^3
// sum is split over the blocks its support reaches; a thread sums the part
// inside its block and adds it into the node's accumulator.
// ---------------------------------------------------------------------------
template <typename T, int W, int RM>
__device__ __forceinline__ void k_zfft_interp_body(const SpZP& P, const int* __restrict__ cstart,
                                                   const NdW<T, W>* __restrict__ nds,
                                                   const typename Cx<T>::t* __restrict__ F1,
                                                   const typename Cx<T>::t* __restrict__ tw2, T* __restrict__ vacc,
                                                   int bid)
{
    using C = typename Cx<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int r_beg[kHomeMax], r_pre[kHomeMax + 1];  // home ranges and their prefix
    const int Tx = P.tx, Ty = P.ty, n0 = P.ng[0], n1 = P.ng[1], n2 = P.ng[2], nk = P.K[2] + 1;
    const int txy = Tx * Ty;
    const int ncl = 3 * txy / 2;
    const int CS = P.cls;
    C* cb = reinterpret_cast<C*>(smem_raw);
    const T* accf = reinterpret_cast<const T*>(cb);
    const int tid = threadIdx.x;
    const int by = fdiv(bid, P.d_nbx);
    const int bx = bid - by * P.nbx;
    constexpr int H = W / 2;
    // the home ranges are fetched while the buffer is cleared
    int rb0, rlen;
    const int nr = home_fetch(P, cstart, bx, by, H, rb0, rlen);
    zero_cx(cb, ncl * CS);
    if (tid < kHomeMax) {
        r_beg[tid] = rb0;
        r_pre[tid + 1] = rlen;
    }
    __syncthreads();
    home_prefix(r_pre);
    // Z_k = A_k + i B_k, Z_{n-k} = conj(A_k) + i conj(B_k) at the digit-reversed
    // positions, 8 consecutive k of one line pair per thread
    const int nq = (nk + 7) >> 3;
    for (int i = tid; i < ncl * nq; i += blockDim.x) {
        const int l = i / nq, q = i - l * nq;
        const int rl = 2 * l;
        const int c = fdiv(rl, P.d_txy), rem = rl - c * txy;
        const int lx = fdiv(rem, P.d_ty), ly = rem - lx * Ty;
        const C* rowA = F1 + (((size_t)c * n0 + bx * Tx + lx) * n1 + by * Ty + ly) * nk;
        const C* rowB = rowA + nk;
        C A[8], Bv[8];
        load8(rowA, nk, q, A);
        load8(rowB, nk, q, Bv);
        const Rev8 rb = rev8_bases(P.rev, P.plan2, q);
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int k = 8 * q + d;
            if (k >= nk) break;
            C z;
            if (k == 0) {
                z.x = A[d].x;
                z.y = Bv[d].x;
                cb[l * CS] = z;
            } else {
                z.x = A[d].x - Bv[d].y;
                z.y = A[d].y + Bv[d].x;
                cb[l * CS + rev8_pos(rb, P.rev, k, d)] = z;
                z.x = A[d].x + Bv[d].y;
                z.y = -A[d].y + Bv[d].x;
                cb[l * CS + rev8_neg(rb, P.rev, n2, k, d)] = z;
            }
        }
    }
    __syncthreads();
    const int ncand = r_pre[nr];
    fft_inv_dit<T, RM>(cb, ncl, P.d_ncl, CS, P.plan2, tw2);
    // periodic halo: positions n2 .. n2 + W - 2 of every line repeat 0 .. W - 2
    // (the line stride leaves room), so a node's W positions from its support
    // start taken modulo n2 are contiguous
    for (int i = tid; i < ncl * (W - 1); i += blockDim.x) {
        const int l = i / (W - 1), t = i - l * (W - 1);
        cb[l * CS + n2 + t] = cb[l * CS + t];
    }
    __syncthreads();
    // real line rl = c txy + lx Ty + ly at position z is the float
    // ((rl >> 1) CS + z) 2 + (rl & 1) = rbase(lx, ly) + 2 z + c txy CS
    const int sc = txy * CS;
    // a thread per candidate node of the gathered home ranges, its record read
    // from global memory (consecutive threads on consecutive records of a
    // range, mostly L2 hits); no block-wide waits, so every warp works
    int r = 0;  // range of candidate k (k only grows for a thread)
    {
        for (int k = tid; k < ncand; k += blockDim.x) {
            while (r + 1 < nr && r_pre[r + 1] <= k) ++r;
            const NdW<T, W>& R = nds[r_beg[r] + (k - r_pre[r])];
            const int base = R.base;
            // support start relative to the block, taking the periodic image
            // that meets it (the grid is wider than W + T)
            const int r0 = home_rel(base & 1023, H, bx * Tx, Tx, n0, W);
            const int r1 = home_rel((base >> 10) & 1023, H, by * Ty, Ty, n1, W);
            if (r0 > Tx - 1 || r0 + W - 1 < 0 || r1 > Ty - 1 || r1 + W - 1 < 0) continue;
            const int z0 = ((base >> 20) & 1023) - H + 1;
            const int zb2 = 2 * (z0 < 0 ? z0 + n2 : z0);  // float offset of the first position
            T wz[W];
#pragma unroll
            for (int t = 0; t < W; ++t) wz[t] = R.wz[t];
            const int lx0 = max(r0, 0), lx1 = min(r0 + W - 1, Tx - 1);
            const int ly0 = max(r1, 0), ly1 = min(r1 + W - 1, Ty - 1);
            T a0 = 0, a1 = 0, a2 = 0;
            // the rows ly = 2 lp and 2 lp + 1 of a column pair are the two
            // halves of one complex line: one 2-word read per position gives
            // both (the half outside the support weighted by 0)
            using T2 = typename Cx<T>::t;
            for (int lp = ly0 >> 1; lp <= ly1 >> 1; ++lp) {
                const int le = 2 * lp, lo = le + 1;
                const T wye = le >= ly0 ? R.wy[le - r1] : (T)0;
                const T wyo = lo <= ly1 ? R.wy[lo - r1] : (T)0;
                for (int lx = lx0; lx <= lx1; ++lx) {
                    const T* row = accf + lp * 2 * CS + lx * Ty * CS + zb2;
                    T e0 = 0, e1 = 0, e2 = 0, o0 = 0, o1 = 0, o2 = 0;
#pragma unroll
                    for (int t = 0; t < W; ++t) {
                        const T2 v0 = *reinterpret_cast<const T2*>(row + 2 * t);
                        const T2 v1 = *reinterpret_cast<const T2*>(row + sc + 2 * t);
                        const T2 v2 = *reinterpret_cast<const T2*>(row + 2 * sc + 2 * t);
                        e0 += wz[t] * v0.x;
                        o0 += wz[t] * v0.y;
                        e1 += wz[t] * v1.x;
                        o1 += wz[t] * v1.y;
                        e2 += wz[t] * v2.x;
                        o2 += wz[t] * v2.y;
                    }
                    const T wx = R.wx[lx - r0];
                    a0 += wx * (wye * e0 + wyo * o0);
                    a1 += wx * (wye * e1 + wyo * o1);
                    a2 += wx * (wye * e2 + wyo * o2);
                }
            }
            const size_t j = (size_t)R.j;
            atomicAdd(&vacc[3 * j + 0], a0);
            atomicAdd(&vacc[3 * j + 1], a1);
            atomicAdd(&vacc[3 * j + 2], a2);
        }
    }
}

template <typename T, int W, int RM>
__global__ void __launch_bounds__(z_threads_max<T>(), sizeof(T) == 4 ? 2 : 3) k_zfft_interp(SpZP P, const int* __restrict__ cstart,
                                                          const NdW<T, W>* __restrict__ nds,
                                                          const typename Cx<T>::t* __restrict__ F1,
                                                          const typename Cx<T>::t* __restrict__ tw2,
                                                          T* __restrict__ vacc)
{
    k_zfft_interp_body<T, W, RM>(P, cstart, nds, F1, tw2, vacc, blockIdx.x);
}

// One thread per node: grid cell and fraction (the interpolation's binning),
// the 3 W kernel weights, and the node's rank within the block of its cell
// (one atomic per run of equal blocks in a warp).
template <typename T, int W>
__device__ __forceinline__ void k_node_w_body(const InterpP& P, int tx, int ty, int nbx,
                                              const double* __restrict__ nodes, NdW<T, W>* __restrict__ out,
                                              int* __restrict__ key, int* __restrict__ rank, int* __restrict__ cnt,
                                              int bid)
{
    const int j = bid * blockDim.x + threadIdx.x;
    const bool live = j < P.N;
    constexpr int H = W / 2;
    int b = -1;
    if (live) {
        NdW<T, W> R;
        int ib[3];
        T fr[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double x = nodes[3 * j + d];
            if (!isfinite(x)) x = 0.0;
            double xw = x - P.L[d] * floor(x * P.iL[d]);
            if (xw >= P.L[d]) xw -= P.L[d];
            if (xw < 0.0) xw = 0.0;
            const double g = xw * P.ihg[d];
            int k = (int)floor(g);
            k = k < 0 ? 0 : (k >= P.ng[d] ? P.ng[d] - 1 : k);
            double f = g - (double)k;
            f = f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
            ib[d] = k;
            fr[d] = (T)f;
        }
        const T zeta = (T)P.zeta;
        const T inorm = (T)P.inorm;
#pragma unroll
        for (int t = 0; t < W; ++t) {
            R.wx[t] = kb_val((fr[0] + (T)(H - 1 - t)) * ((T)2 / (T)W), zeta, inorm);
            R.wy[t] = kb_val((fr[1] + (T)(H - 1 - t)) * ((T)2 / (T)W), zeta, inorm);
            R.wz[t] = kb_val((fr[2] + (T)(H - 1 - t)) * ((T)2 / (T)W), zeta, inorm);
        }
        R.base = ib[0] | (ib[1] << 10) | (ib[2] << 20);
        R.j = j;
        out[j] = R;
        b = ib[0] / tx + nbx * (ib[1] / ty);
        key[j] = b;
    }
    const int r = warp_rank(b, cnt);
    if (live) rank[j] = r;
}

template <typename T, int W>
__global__ void k_node_w(InterpP P, int tx, int ty, int nbx, const double* __restrict__ nodes,
                         NdW<T, W>* __restrict__ out, int* __restrict__ key, int* __restrict__ rank,
                         int* __restrict__ cnt)
{
    k_node_w_body<T, W>(P, tx, ty, nbx, nodes, out, key, rank, cnt, blockIdx.x);
}

template <typename T, int W>
__device__ __forceinline__ void k_node_scatter_body(int N, const NdW<T, W>* __restrict__ in,
                                                    const int* __restrict__ key, const int* __restrict__ rank,
                                                    const int* __restrict__ start, NdW<T, W>* __restrict__ out,
                                                    int bid)
{
    const int j = bid * blockDim.x + threadIdx.x;
    if (j < N) out[start[key[j]] + rank[j]] = in[j];
}

template <typename T, int W>
__global__ void k_node_scatter(int N, const NdW<T, W>* __restrict__ in, const int* __restrict__ key,
                               const int* __restrict__ rank, const int* __restrict__ start,
                               NdW<T, W>* __restrict__ out)
{
    k_node_scatter_body<T, W>(N, in, key, rank, start, out, blockIdx.x);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <typename T>
size_t col_pt_bytes(int w)
{
    switch (w) {
    case 2: return sizeof(SpPt<T, 2>);
    case 4: return sizeof(SpPt<T, 4>);
    case 6: return sizeof(SpPt<T, 6>);
    case 8: return sizeof(SpPt<T, 8>);
    case 10: return sizeof(SpPt<T, 10>);
    case 12: return sizeof(SpPt<T, 12>);
    case 14: return sizeof(SpPt<T, 14>);
    case 16: return sizeof(SpPt<T, 16>);
    default: return 0;
    }
}

template <typename T, int W>
static cudaError_t col_scatter_w(const ColP& P, const Work& w, int NQ, cudaStream_t s, bool det)
{
    // deterministic: the copies' entries go to the second buffer, then every
    // column block is put in increasing source order
    static_assert(sizeof(SpPt<T, W>) % 16 == 0, "records are gathered as 16-byte words");
    k_col_scatter<T, W><<<(NQ + kThreads - 1) / kThreads, kThreads, 0, s>>>(
        P, (const LrRec<T>*)w.lr_rec, NQ, w.col_cur, det ? w.col_rec2 : w.col_rec, (SpPt<T, W>*)w.col_pts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !det) return e;
    return launch_segsort_int2(w.col_cnt, P.ncols * P.nzb, w.col_rec2, w.col_rec, s);
}

template <typename T>
static cudaError_t launch_col_scatter_w(const ColP& P, const Work& w, int NQ, cudaStream_t s, bool det)
{
    switch (P.w) {
    case 2: return col_scatter_w<T, 2>(P, w, NQ, s, det);
    case 4: return col_scatter_w<T, 4>(P, w, NQ, s, det);
    case 6: return col_scatter_w<T, 6>(P, w, NQ, s, det);
    case 8: return col_scatter_w<T, 8>(P, w, NQ, s, det);
    case 10: return col_scatter_w<T, 10>(P, w, NQ, s, det);
    case 12: return col_scatter_w<T, 12>(P, w, NQ, s, det);
    case 14: return col_scatter_w<T, 14>(P, w, NQ, s, det);
    case 16: return col_scatter_w<T, 16>(P, w, NQ, s, det);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_col_sort(const ColP& P, const Work& w, int NQ, cudaStream_t s, bool det)
{
    const int nbins = P.ncols * P.nzb;
    cudaError_t e = cudaMemsetAsync(w.col_cnt, 0, sizeof(int) * (size_t)(nbins + 1), s);
    if (e != cudaSuccess) return e;
    if (NQ > 0) k_col_count<T><<<(NQ + kThreads - 1) / kThreads, kThreads, 0, s>>>(P, (const LrRec<T>*)w.lr_rec, NQ,
                                                                                  w.col_cnt);
    e = scan_exclusive(w.col_cnt, nbins, w.scan_tmp2, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(w.col_cur, w.col_cnt, sizeof(int) * (size_t)nbins, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    if (NQ > 0)
        e = launch_col_scatter_w<T>(P, w, NQ, s, det);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename T, int W>
static cudaError_t node_bin_w(const ColP& P, const InterpP& I, const double* nodes, const Work& w, cudaStream_t s)
{
    const int N = I.N;
    const int g = (N + kThreads - 1) / kThreads;
    k_node_w<T, W><<<g, kThreads, 0, s>>>(I, P.tx, P.ty, P.nbx, nodes, (NdW<T, W>*)w.nd_rec, w.nd_key, w.nd_rank,
                                           w.ncol_cnt);
    cudaError_t e = scan_exclusive(w.ncol_cnt, P.ncols, w.scan_tmp, s);
    if (e != cudaSuccess) return e;
    k_node_scatter<T, W><<<g, kThreads, 0, s>>>(N, (const NdW<T, W>*)w.nd_rec, w.nd_key, w.nd_rank, w.ncol_cnt,
                                                 (NdW<T, W>*)w.nd_sorted);
    return cudaGetLastError();
}

// Sorts the nodes with their weights by the z-column block of their grid
// cell for the fused inverse-z interpolation, and clears the accumulator it
// adds into.
template <typename T>
cudaError_t launch_node_bin(const ColP& P, const InterpP& I, const double* nodes, const Work& w, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(w.vacc, 0, sizeof(T) * 3 * (size_t)I.N, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w.ncol_cnt, 0, sizeof(int) * (size_t)(P.ncols + 1), s);
    if (e != cudaSuccess || I.N == 0) return e;
    switch (P.w) {
    case 2: return node_bin_w<T, 2>(P, I, nodes, w, s);
    case 4: return node_bin_w<T, 4>(P, I, nodes, w, s);
    case 6: return node_bin_w<T, 6>(P, I, nodes, w, s);
    case 8: return node_bin_w<T, 8>(P, I, nodes, w, s);
    case 10: return node_bin_w<T, 10>(P, I, nodes, w, s);
    case 12: return node_bin_w<T, 12>(P, I, nodes, w, s);
    case 14: return node_bin_w<T, 14>(P, I, nodes, w, s);
    case 16: return node_bin_w<T, 16>(P, I, nodes, w, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
size_t nd_rec_bytes(int w)
{
    switch (w) {
    case 2: return sizeof(NdW<T, 2>);
    case 4: return sizeof(NdW<T, 4>);
    case 6: return sizeof(NdW<T, 6>);
    case 8: return sizeof(NdW<T, 8>);
    case 10: return sizeof(NdW<T, 10>);
    case 12: return sizeof(NdW<T, 12>);
    case 14: return sizeof(NdW<T, 14>);
    case 16: return sizeof(NdW<T, 16>);
    default: return 0;
    }
}

template <typename T>
size_t spread_zfft_smem(const SpZP& P)
{
    using C = typename Cx<T>::t;
    const int ncl = 3 * P.tx * P.ty / 2;
    return zlines_bytes<T>(ncl, P.cls) + 2 * spz_rec_chunk<T>() * col_pt_bytes<T>(P.w);  // two record chunks
}

// Register-budget class of a plan: the largest radix it uses, rounded up to
// a compiled set.  Only radices up to 8 (with the composite 6) are compiled:
// measured on the 384-point lines of the 1e5-node tangle, two passes of
// radix 24 x 16 at 128 registers (two CTAs per SM) ran 30 % slower than three
// passes of 8 x 8 x 6 at 64 registers (five CTAs per SM, shared-memory bound).
static int plan_rm(const FftPlan& pl)
{
    int m = 2;
    for (int s = 0; s < pl.nr; ++s) m = pl.r[s] > m ? pl.r[s] : m;
    return m <= 8 ? 8 : (m <= 16 ? 16 : (m <= 24 ? 24 : 32));
}

// Calls f.run<RM>() with the plan's register class.
template <typename T, typename F>
static cudaError_t by_rm(const FftPlan& pl, F&& f)
{
    return plan_rm(pl) == 8 ? f.template run<8>() : cudaErrorInvalidValue;
}

template <typename T, int W>
struct SpzLaunch {
    const SpZP& P;
    const Work& w;
    cudaStream_t s;
    template <int RM>
    cudaError_t run()
    {
        using C = typename Cx<T>::t;
        const size_t sm = spread_zfft_smem<T>(P);
        cudaError_t e =
            cudaFuncSetAttribute(k_spread_zfft<T, W, RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_spread_zfft<T, W, RM><<<P.nbx * P.nby, z_threads<T>(P), sm, s>>>(
            P, w.col_cnt, w.col_rec, (const SpPt<T, W>*)w.col_pts, (const C*)w.tw + P.ng[0] + P.ng[1],
            (C*)w.spec);
        return cudaGetLastError();
    }
};

template <typename T, int W>
static cudaError_t spz_w(const SpZP& P, const Work& w, cudaStream_t s)
{
    return by_rm<T>(P.plan2, SpzLaunch<T, W>{ P, w, s });
}

template <typename T>
cudaError_t launch_spread_zfft(const SpZP& P, const Work& w, cudaStream_t s)
{
    switch (P.w) {
    case 2: return spz_w<T, 2>(P, w, s);
    case 4: return spz_w<T, 4>(P, w, s);
    case 6: return spz_w<T, 6>(P, w, s);
    case 8: return spz_w<T, 8>(P, w, s);
    case 10: return spz_w<T, 10>(P, w, s);
    case 12: return spz_w<T, 12>(P, w, s);
    case 14: return spz_w<T, 14>(P, w, s);
    case 16: return spz_w<T, 16>(P, w, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T, int W>
struct ZiLaunch {
    const SpZP& P;
    const Work& w;
    cudaStream_t s;
    template <int RM>
    cudaError_t run()
    {
        using C = typename Cx<T>::t;
        const size_t sm = zlines_bytes<T>(3 * P.tx * P.ty / 2, P.cls);
        cudaError_t e =
            cudaFuncSetAttribute(k_zfft_interp<T, W, RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_zfft_interp<T, W, RM><<<P.nbx * P.nby, z_threads<T>(P), sm, s>>>(
            P, w.ncol_cnt, (const NdW<T, W>*)w.nd_sorted, (const C*)w.spec, (const C*)w.tw + P.ng[0] + P.ng[1],
            (T*)w.vacc);
        return cudaGetLastError();
    }
};

template <typename T, int W>
static cudaError_t zi_w(const SpZP& P, const Work& w, cudaStream_t s)
{
    if (!zfft_interp_fits(P.tx, P.ty, W, P.ng[0], P.ng[1], P.nbx, P.nby)) return cudaErrorInvalidValue;
    return by_rm<T>(P.plan2, ZiLaunch<T, W>{ P, w, s });
}

template <typename T>
cudaError_t launch_zfft_interp(const SpZP& P, const Work& w, cudaStream_t s)
{
    switch (P.w) {
    case 2: return zi_w<T, 2>(P, w, s);
    case 4: return zi_w<T, 4>(P, w, s);
    case 6: return zi_w<T, 6>(P, w, s);
    case 8: return zi_w<T, 8>(P, w, s);
    case 10: return zi_w<T, 10>(P, w, s);
    case 12: return zi_w<T, 12>(P, w, s);
    case 14: return zi_w<T, 14>(P, w, s);
    case 16: return zi_w<T, 16>(P, w, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
struct FftYLaunch {
    const FftYP& P;
    const Work& w;
    void* f2;
    int sign;
    cudaStream_t s;
    const CUtensorMap* tm;
    template <int RM>
    cudaError_t run()
    {
        using C = typename Cx<T>::t;
        const int MC = 1 << P.lmc;
        FftYP Q = P;
        CUtensorMap map;
        if (tm && Q.tnb > 0) {
            map = *tm;
        } else {
            Q.tnb = 0;
            memset(&map, 0, sizeof map);
        }
        size_t sm = (size_t)MC * P.ls * sizeof(C);
        if (Q.tnb > 0) sm = (size_t)MC * std::max(P.ls, Q.tnb * Q.tby) * sizeof(C) + 128;
        cudaError_t e = cudaFuncSetAttribute(k_fft_y<T, RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        const int nk = P.K[2] + 1;
        const int nch = (nk + MC - 1) / MC;
        k_fft_y<T, RM><<<3 * P.ng[0] * nch, kThreads, sm, s>>>(Q, (C*)w.spec, (C*)f2, (const C*)w.tw + P.ng[0],
                                                                sign, map, w.status);
        return cudaGetLastError();
    }
};

template <typename T>
cudaError_t launch_fft_y(const FftYP& P, const Work& w, void* f2, int sign, cudaStream_t s, const CUtensorMap* tm_f1)
{
    return by_rm<T>(P.plan1, FftYLaunch<T>{ P, w, f2, sign, s, tm_f1 });
}

// cuTensorMapEncodeTiled through the runtime (no link against the driver
// library); null when the driver does not offer it.
static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
        cudaGetLastError();
    });
    return fn;
}

template <typename T>
bool make_tmap_y(void* F1, const FftYP& P, CUtensorMap* tm)
{
    const int MC = 1 << P.lmc, nk = P.K[2] + 1;
    // rows 16-byte multiples, box start (2 mz0 reals, mz0 a multiple of MC)
    // on a 16-byte boundary, box rows on 128-byte boundaries in shared memory
    if (MC < 2 || (sizeof(T) == 4 && nk % 2 != 0) || P.tnb <= 0 || P.tby <= 0 || P.tby > 256 ||
        (P.tby * MC * 2 * sizeof(T)) % 128 != 0 || P.tnb * P.tby < P.ng[1])
        return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return false;
    const cuuint64_t dim[3] = { (cuuint64_t)2 * nk, (cuuint64_t)P.ng[1], (cuuint64_t)3 * P.ng[0] };
    const cuuint64_t stride[2] = { (cuuint64_t)2 * nk * sizeof(T), (cuuint64_t)2 * nk * sizeof(T) * P.ng[1] };
    const cuuint32_t box[3] = { (cuuint32_t)(2 * MC), (cuuint32_t)P.tby, 1 };
    const cuuint32_t estr[3] = { 1, 1, 1 };
    const CUresult r = enc(tm, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                           F1, dim, stride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}
template bool make_tmap_y<float>(void*, const FftYP&, CUtensorMap*);
template bool make_tmap_y<double>(void*, const FftYP&, CUtensorMap*);

template <typename T>
bool make_tmap_x(void* F2, const FftXP& P, CUtensorMap* tm)
{
    const int MC = 1 << P.lmc, nk = P.K[2] + 1, n0 = P.ng[0], ny2 = 2 * P.K[1] + 1;
    // rows 16-byte multiples, box start (2 mz0 reals) on a 16-byte boundary,
    // boxes on 128-byte boundaries in shared memory
    if (MC < 2 || (sizeof(T) == 4 && nk % 2 != 0) || P.tnbx <= 0 || P.tbx <= 0 || P.tbx > 256 ||
        ((size_t)P.tbx * 3 * MC * 2 * sizeof(T)) % 128 != 0 || P.tnbx * P.tbx < n0 || !P.irev)
        return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return false;
    const cuuint64_t row = (cuuint64_t)2 * nk * sizeof(T);
    const cuuint64_t dim[4] = { (cuuint64_t)2 * nk, 3, (cuuint64_t)n0, (cuuint64_t)ny2 };
    const cuuint64_t stride[3] = { row * ny2 * n0, row * ny2, row };  // component, x, y mode
    const cuuint32_t box[4] = { (cuuint32_t)(2 * MC), 3, (cuuint32_t)P.tbx, 1 };
    const cuuint32_t estr[4] = { 1, 1, 1, 1 };
    const CUresult r = enc(tm, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
                           F2, dim, stride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}
template bool make_tmap_x<float>(void*, const FftXP&, CUtensorMap*);
template bool make_tmap_x<double>(void*, const FftXP&, CUtensorMap*);

template <typename T>
struct FftXLaunch {
    const FftXP& P;
    const Work& w;
    bool want_psi;
    cudaStream_t s;
    const CUtensorMap* tm;
    template <int RM>
    cudaError_t run()
    {
        using C = typename Cx<T>::t;
        const int MC = 1 << P.lmc;
        const int nl = (want_psi ? 6 : 3) * MC;
        FftXP Q = P;
        CUtensorMap map;
        if (tm && Q.tnbx > 0 && !want_psi && !P.spectrum && !P.epart) {
            map = *tm;
        } else {
            Q.tnbx = 0;
            memset(&map, 0, sizeof map);
        }
        size_t sm = (size_t)nl * P.ls * sizeof(C);
        if (Q.tnbx > 0) sm = (size_t)3 * MC * Q.tnbx * Q.tbx * sizeof(C) + 128;
        if (P.spectrum) sm = std::max(sm, (size_t)3 * MC * P.ls * sizeof(C) + sizeof(double) * (size_t)P.nbins);
        if (P.epart) sm += sizeof(double) * (kZThreadsMax / 32);
        cudaError_t e =
            cudaFuncSetAttribute(k_fft_x_kspace<T, RM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        const int nk = P.K[2] + 1;
        const int nch = (nk + MC - 1) / MC;
        const int ntab = P.K[0] + P.K[1] + P.K[2] + 3;
        const T* tab0 = (const T*)w.ktab + (P.single_decon ? ntab : 0);
        const T* tab1 = tab0 + (P.K[0] + 1);
        const T* tab2 = tab1 + (P.K[1] + 1);
        const int nt = P.nthreads > 0 && P.nthreads <= z_threads_max<T>() ? P.nthreads : kThreads;
        k_fft_x_kspace<T, RM><<<(2 * P.K[1] + 1) * nch, nt, sm, s>>>(
            Q, (C*)w.f2, want_psi ? (C*)w.f2psi : nullptr, (const C*)w.tw, tab0, tab1, tab2, map, w.status);
        return cudaGetLastError();
    }
};

template <typename T>
cudaError_t launch_fft_x_kspace(const FftXP& P, const Work& w, bool want_psi, cudaStream_t s)
{
    return by_rm<T>(P.plan0, FftXLaunch<T>{ P, w, want_psi, s, nullptr });
}

template <typename T>
cudaError_t launch_fft_x_kspace(const FftXP& P, const Work& w, bool want_psi, cudaStream_t s,
                                const CUtensorMap* tm_f2)
{
    return by_rm<T>(P.plan0, FftXLaunch<T>{ P, w, want_psi, s, tm_f2 });
}

template <typename T, typename TO>
struct FftZLaunch {
    const FftZP& P;
    const Work& w;
    TO* out;
    cudaStream_t s;
    template <int RM>
    cudaError_t run()
    {
        using C = typename Cx<T>::t;
        const size_t sm = (size_t)(P.yc / 2) * P.cls * sizeof(C);
        cudaError_t e =
            cudaFuncSetAttribute(k_fft_z_c2r<T, RM, TO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_fft_z_c2r<T, RM, TO><<<3 * P.ng[0] * (P.ng[1] / P.yc), kThreads, sm, s>>>(
            P, (const C*)w.spec, (const C*)w.tw + P.ng[0] + P.ng[1], out);
        return cudaGetLastError();
    }
};

template <typename T>
cudaError_t launch_fft_z_c2r(const FftZP& P, const Work& w, cudaStream_t s, double* out64)
{
    if (out64) return by_rm<T>(P.plan2, FftZLaunch<T, double>{ P, w, out64, s });
    if (!w.grid) return cudaErrorInvalidValue;
    return by_rm<T>(P.plan2, FftZLaunch<T, T>{ P, w, (T*)w.grid, s });
}

// ---------------------------------------------------------------------------
// Batched forms: one launch per stage for every member of a batch (member m
// runs its blocks [bstart[m], bstart[m+1]) of the launch).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_col_count_b(const ColD<T>* __restrict__ d, const int* __restrict__ bs, int n)
{
    int bid, nb;
    const ColD<T>& a = d[batch_member(bs, n, bid, nb)];
    k_col_count_body<T>(a.P, a.rec, a.n, a.cnt, bid);
}

template <typename T, int W>
__global__ void k_col_scatter_b(const ColD<T>* __restrict__ d, const int* __restrict__ bs, int n)
{
    int bid, nb;
    const ColD<T>& a = d[batch_member(bs, n, bid, nb)];
    k_col_scatter_body<T, W>(a.P, a.rec, a.n, a.cnt, (int2*)a.out, (SpPt<T, W>*)a.pts, bid);
}

template <typename T, int W, int RM>
__global__ void __launch_bounds__(z_threads_max<T>(), 2) k_spread_zfft_b(const SpzD<T>* __restrict__ d,
                                                                       const int* __restrict__ bs, int n)
{
    using C = typename Cx<T>::t;
    int bid, nb;
    const SpzD<T>& a = d[batch_member(bs, n, bid, nb)];
    __shared__ SpZP sP;
    batch_param_copy(sP, a.P);
    k_spread_zfft_body<T, W, RM>(sP, a.cstart, (const int2*)a.recs, (const SpPt<T, W>*)a.pts, (const C*)a.tw2,
                                 (C*)a.F1, bid);
}

template <typename T, int RM>
__global__ void __launch_bounds__(kThreads, 2) k_fft_y_b(const FftYD<T>* __restrict__ d, const int* __restrict__ bs,
                                                      int n)
{
    using C = typename Cx<T>::t;
    int bid, nb;
    const FftYD<T>& a = d[batch_member(bs, n, bid, nb)];
    __shared__ FftYP sP;
    batch_param_copy(sP, a.P);
    k_fft_y_body<T, RM>(sP, (C*)a.F1, (C*)a.F2, (const C*)a.tw1, a.sign, bid);
}

template <typename T, int RM>
__global__ void __launch_bounds__(z_threads_max<T>(), 2) k_fft_x_kspace_b(const FftXD<T>* __restrict__ d,
                                                                        const int* __restrict__ bs, int n)
{
    using C = typename Cx<T>::t;
    int bid, nb;
    const FftXD<T>& a = d[batch_member(bs, n, bid, nb)];
    __shared__ FftXP sP;
    batch_param_copy(sP, a.P);
    k_fft_x_kspace_body<T, RM>(sP, (C*)a.F2, nullptr, (const C*)a.tw0, a.tab0, a.tab1, a.tab2, bid);
}

template <typename T, int W>
__global__ void k_node_w_b(const NodeWD<T>* __restrict__ d, const int* __restrict__ bs, int n)
{
    int bid, nb;
    const NodeWD<T>& a = d[batch_member(bs, n, bid, nb)];
    k_node_w_body<T, W>(a.P, a.tx, a.ty, a.nbx, a.nodes, (NdW<T, W>*)a.rec, a.key, a.rank, a.cnt, bid);
}

template <typename T, int W>
__global__ void k_node_scatter_b(const NodeWD<T>* __restrict__ d, const int* __restrict__ bs, int n)
{
    int bid, nb;
    const NodeWD<T>& a = d[batch_member(bs, n, bid, nb)];
    k_node_scatter_body<T, W>(a.P.N, (const NdW<T, W>*)a.rec, a.key, a.rank, a.cnt, (NdW<T, W>*)a.sorted, bid);
}

template <typename T, int W, int RM>
__global__ void __launch_bounds__(z_threads_max<T>(), sizeof(T) == 4 ? 2 : 3) k_zfft_interp_b(
    const SpzD<T>* __restrict__ d, const int* __restrict__ bs, int n)
{
    using C = typename Cx<T>::t;
    int bid, nb;
    const SpzD<T>& a = d[batch_member(bs, n, bid, nb)];
    __shared__ SpZP sP;
    batch_param_copy(sP, a.P);
    k_zfft_interp_body<T, W, RM>(sP, a.cstart, (const NdW<T, W>*)a.recs, (const C*)a.F1, (const C*)a.tw2, a.vacc,
                                 bid);
}

#define BSW_BY_W(EXPR)                       \
    switch (w) {                             \
    case 2: { constexpr int W = 2; EXPR; break; }   \
    case 4: { constexpr int W = 4; EXPR; break; }   \
    case 6: { constexpr int W = 6; EXPR; break; }   \
    case 8: { constexpr int W = 8; EXPR; break; }   \
    case 10: { constexpr int W = 10; EXPR; break; } \
    case 12: { constexpr int W = 12; EXPR; break; } \
    case 14: { constexpr int W = 14; EXPR; break; } \
    case 16: { constexpr int W = 16; EXPR; break; } \
    default: return cudaErrorInvalidValue;   \
    }

template <typename T>
cudaError_t launch_col_count_b(const BatchL& L, cudaStream_t s)
{
    if (L.total > 0) k_col_count_b<T><<<L.total, kThreads, 0, s>>>((const ColD<T>*)L.desc, L.bstart, L.n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_col_scatter_b(int w, const BatchL& L, cudaStream_t s)
{
    if (L.total <= 0) return cudaSuccess;
    BSW_BY_W((k_col_scatter_b<T, W><<<L.total, kThreads, 0, s>>>((const ColD<T>*)L.desc, L.bstart, L.n)));
    return cudaGetLastError();
}

template <typename T, int W>
static cudaError_t spz_b(const BatchL& L, cudaStream_t s)
{
    cudaError_t e =
        cudaFuncSetAttribute(k_spread_zfft_b<T, W, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (e != cudaSuccess) return e;
    k_spread_zfft_b<T, W, 8><<<L.total, L.threads, L.smem, s>>>((const SpzD<T>*)L.desc, L.bstart, L.n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spread_zfft_b(int w, const BatchL& L, cudaStream_t s)
{
    if (L.total <= 0) return cudaSuccess;
    BSW_BY_W(return (spz_b<T, W>(L, s)));
    return cudaSuccess;
}

template <typename T>
size_t fft_y_smem(const FftYP& P)
{
    return (size_t)(1 << P.lmc) * P.ls * sizeof(typename Cx<T>::t);
}

template <typename T>
cudaError_t launch_fft_y_b(const BatchL& L, cudaStream_t s)
{
    if (L.total <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_fft_y_b<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (e != cudaSuccess) return e;
    k_fft_y_b<T, 8><<<L.total, kThreads, L.smem, s>>>((const FftYD<T>*)L.desc, L.bstart, L.n);
    return cudaGetLastError();
}

template <typename T>
size_t fft_x_smem(const FftXP& P)
{
    return (size_t)3 * (1 << P.lmc) * P.ls * sizeof(typename Cx<T>::t);
}

template <typename T>
cudaError_t launch_fft_x_kspace_b(const BatchL& L, cudaStream_t s)
{
    if (L.total <= 0) return cudaSuccess;
    cudaError_t e =
        cudaFuncSetAttribute(k_fft_x_kspace_b<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (e != cudaSuccess) return e;
    k_fft_x_kspace_b<T, 8><<<L.total, L.threads, L.smem, s>>>((const FftXD<T>*)L.desc, L.bstart, L.n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_node_w_b(int w, const BatchL& L, cudaStream_t s)
{
    if (L.total <= 0) return cudaSuccess;
    BSW_BY_W((k_node_w_b<T, W><<<L.total, kThreads, 0, s>>>((const NodeWD<T>*)L.desc, L.bstart, L.n)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_node_scatter_b(int w, const BatchL& L, cudaStream_t s)
{
    if (L.total <= 0) return cudaSuccess;
    BSW_BY_W((k_node_scatter_b<T, W><<<L.total, kThreads, 0, s>>>((const NodeWD<T>*)L.desc, L.bstart, L.n)));
    return cudaGetLastError();
}

template <typename T>
size_t zfft_interp_smem(const SpZP& P)
{
    return zlines_bytes<T>(3 * P.tx * P.ty / 2, P.cls);
}

template <typename T, int W>
static cudaError_t zi_b(const BatchL& L, cudaStream_t s)
{
    cudaError_t e =
        cudaFuncSetAttribute(k_zfft_interp_b<T, W, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (e != cudaSuccess) return e;
    k_zfft_interp_b<T, W, 8><<<L.total, L.threads, L.smem, s>>>((const SpzD<T>*)L.desc, L.bstart, L.n);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_zfft_interp_b(int w, const BatchL& L, cudaStream_t s)
{
    if (L.total <= 0) return cudaSuccess;
    BSW_BY_W(return (zi_b<T, W>(L, s)));
    return cudaSuccess;
}
#undef BSW_BY_W

#define BSW_INST_B(T)                                                                  \
    template cudaError_t launch_col_count_b<T>(const BatchL&, cudaStream_t);           \
    template cudaError_t launch_col_scatter_b<T>(int, const BatchL&, cudaStream_t);    \
    template cudaError_t launch_spread_zfft_b<T>(int, const BatchL&, cudaStream_t);    \
    template cudaError_t launch_fft_y_b<T>(const BatchL&, cudaStream_t);               \
    template cudaError_t launch_fft_x_kspace_b<T>(const BatchL&, cudaStream_t);        \
    template cudaError_t launch_node_w_b<T>(int, const BatchL&, cudaStream_t);         \
    template cudaError_t launch_node_scatter_b<T>(int, const BatchL&, cudaStream_t);   \
    template cudaError_t launch_zfft_interp_b<T>(int, const BatchL&, cudaStream_t);    \
    template size_t fft_y_smem<T>(const FftYP&);                                       \
    template size_t fft_x_smem<T>(const FftXP&);                                       \
    template size_t zfft_interp_smem<T>(const SpZP&);
BSW_INST_B(float)
BSW_INST_B(double)
#undef BSW_INST_B

template cudaError_t launch_col_sort<float>(const ColP&, const Work&, int, cudaStream_t, bool);
template cudaError_t launch_col_sort<double>(const ColP&, const Work&, int, cudaStream_t, bool);
template cudaError_t launch_spread_zfft<float>(const SpZP&, const Work&, cudaStream_t);
template cudaError_t launch_spread_zfft<double>(const SpZP&, const Work&, cudaStream_t);
template cudaError_t launch_zfft_interp<float>(const SpZP&, const Work&, cudaStream_t);
template cudaError_t launch_zfft_interp<double>(const SpZP&, const Work&, cudaStream_t);
template cudaError_t launch_node_bin<float>(const ColP&, const InterpP&, const double*, const Work&, cudaStream_t);
template cudaError_t launch_node_bin<double>(const ColP&, const InterpP&, const double*, const Work&, cudaStream_t);
template size_t nd_rec_bytes<float>(int);
template size_t nd_rec_bytes<double>(int);
template cudaError_t launch_fft_x_kspace<float>(const FftXP&, const Work&, bool, cudaStream_t, const CUtensorMap*);
template cudaError_t launch_fft_x_kspace<double>(const FftXP&, const Work&, bool, cudaStream_t, const CUtensorMap*);
template cudaError_t launch_fft_y<float>(const FftYP&, const Work&, void*, int, cudaStream_t, const CUtensorMap*);
template cudaError_t launch_fft_y<double>(const FftYP&, const Work&, void*, int, cudaStream_t, const CUtensorMap*);
template cudaError_t launch_fft_x_kspace<float>(const FftXP&, const Work&, bool, cudaStream_t);
template cudaError_t launch_fft_x_kspace<double>(const FftXP&, const Work&, bool, cudaStream_t);
template cudaError_t launch_fft_z_c2r<float>(const FftZP&, const Work&, cudaStream_t, double*);
template cudaError_t launch_fft_z_c2r<double>(const FftZP&, const Work&, cudaStream_t, double*);
// Writes the composite-radix twiddles into the current device's constant
// bank (once per device).
cudaError_t set_fft_constants()
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    float2 hf[kTwCount];
    double2 hd[kTwCount];
    const int sizes[6] = { 6, 9, 12, 16, 24, 32 };
    const int offs[6] = { kTwOff6, kTwOff9, kTwOff12, kTwOff16, kTwOff24, kTwOff32 };
    for (int k = 0; k < 6; ++k)
        for (int m = 0; m < sizes[k]; ++m) {
            const double ph = -2.0 * 3.14159265358979323846 * m / sizes[k];
            hd[offs[k] + m] = make_double2(cos(ph), sin(ph));
            hf[offs[k] + m] = make_float2((float)cos(ph), (float)sin(ph));
        }
    e = cudaMemcpyToSymbol(c_twf, hf, sizeof hf);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_twd, hd, sizeof hd);
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

template size_t col_pt_bytes<float>(int);
template size_t col_pt_bytes<double>(int);
template size_t spread_zfft_smem<float>(const SpZP&);
template size_t spread_zfft_smem<double>(const SpZP&);

}  // namespace bsw
