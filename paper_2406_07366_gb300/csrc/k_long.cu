// Long-range part (Sec. 3.3, Appendix A): type-1 NUFFT of the vector charges
// (spread -> FFT -> deconvolve), the Fourier-space Gaussian filter, curl and
// Poisson solve (Eqs. velocity_longrange_physical and the psi analogue), and
// the type-2 NUFFT back to the nodes (FFT^-1 -> interpolate), whose
// epilogue adds the other three parts of Eq. ewald_velocity_splitting.
//
// Kernel (Eq. kaiser_bessel_bw): backwards Kaiser-Bessel on [-1, 1], mapped
// to w grid points, normalised to phi(0) = 1:
//   psi(z) = sinh(zeta s) / (s sinh zeta), s = sqrt(1 - z^2),
// evaluated as exp(zeta (s-1)) (1 - e^{-2 zeta s}) / (s (1 - e^{-2 zeta})).
//
// Spread design.  The grid is very sparse in points (~0.004-0.02 per cell),
// so the spread is bound by writing the three grids.  Each CTA owns one
// tile of the grid in shared memory, gathers every point of the 27
// neighbouring tile bins whose support reaches the tile, accumulates with
// shared-memory atomics (one warp per point, lanes over the support cells),
// and writes the whole tile once: no zeroing pass, no global atomics.
#include <math.h>

#include "bs_internal.cuh"

namespace bsw {

template <typename T>
__device__ __forceinline__ T kb_eval(T z, T zeta, T inorm)
{
    T s2 = (T)1 - z * z;
    s2 = s2 > (T)0 ? s2 : (T)0;
    const T s = sqrt(s2);
    const T num = (s > (T)1e-6) ? -expm1((T)-2 * zeta * s) / s : (T)2 * zeta;
    return exp(zeta * (s - (T)1)) * num * inorm;
}

template <typename T, int W>
__global__ void __launch_bounds__(kThreads) k_spread(SpreadP P, const int* __restrict__ tstart,
                                                     const LrRec<T>* __restrict__ pts, T* __restrict__ grid)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T0 = P.tile[0], T1 = P.tile[1], T2 = P.tile[2];
    const int T2P = T2 + 1;  // padded row: lanes on different rows hit different banks
    const int tsz = T0 * T1 * T2P;
    T* acc = reinterpret_cast<T*>(smem_raw);
    T* ktab = acc + 3 * tsz;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    int* bstart = reinterpret_cast<int*>(ktab + nw * 3 * W);  // 27 bin starts
    int* bpre = bstart + 27;                                  // 28 prefix counts
    int* bwrap = bpre + 28;                                   // 27 x 3 image shifts (in grid points)
    const int b = blockIdx.x;
    const int nt0 = P.ntile[0], nt1 = P.ntile[1], nt2 = P.ntile[2];
    const int t0 = b % nt0, t1 = (b / nt0) % nt1, t2 = b / (nt0 * nt1);
    const int O0 = t0 * T0, O1 = t1 * T1, O2 = t2 * T2;
    for (int i = tid; i < 3 * tsz; i += blockDim.x) acc[i] = (T)0;
    // the 27 neighbouring tile bins (periodic), with the image shift of each
    int cnt = 0;
    if (tid < 27) {
        const int d0 = tid % 3 - 1, d1 = (tid / 3) % 3 - 1, d2 = tid / 9 - 1;
        int u0 = t0 + d0, u1 = t1 + d1, u2 = t2 + d2, s0 = 0, s1 = 0, s2 = 0;
        if (u0 < 0) { u0 += nt0; s0 = -P.ng[0]; } else if (u0 >= nt0) { u0 -= nt0; s0 = P.ng[0]; }
        if (u1 < 0) { u1 += nt1; s1 = -P.ng[1]; } else if (u1 >= nt1) { u1 -= nt1; s1 = P.ng[1]; }
        if (u2 < 0) { u2 += nt2; s2 = -P.ng[2]; } else if (u2 >= nt2) { u2 -= nt2; s2 = P.ng[2]; }
        const int nb = u0 + nt0 * (u1 + nt1 * u2);
        const int a = tstart[nb];
        cnt = tstart[nb + 1] - a;
        bstart[tid] = a;
        bwrap[3 * tid + 0] = s0;
        bwrap[3 * tid + 1] = s1;
        bwrap[3 * tid + 2] = s2;
    }
    if (wid == 0) {  // exclusive prefix of the 27 counts
        int v = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane < 27) bpre[lane + 1] = v;
        if (lane == 0) bpre[0] = 0;
    }
    __syncthreads();

    const T zeta = (T)P.zeta;
    const T inorm = (T)P.inorm;
    T* kw = ktab + wid * 3 * W;
    constexpr int H = W / 2;
    const int total = bpre[27];
    const int my_pre = (lane < 28) ? bpre[lane] : 0x7fffffff;
    for (int k = wid; k < total; k += nw) {
        // bin of entry k: the number of prefixes <= k, minus one
        const unsigned m = __ballot_sync(0xffffffffu, lane < 28 && my_pre <= k);
        const int bin = __popc(m) - 1;
        const LrRec<T> R = pts[bstart[bin] + (k - bpre[bin])];
        const int ib0 = R.base & 1023, ib1 = (R.base >> 10) & 1023, ib2 = (R.base >> 20) & 1023;
        const int r0 = ib0 + bwrap[3 * bin + 0] - O0 - H + 1;
        const int r1 = ib1 + bwrap[3 * bin + 1] - O1 - H + 1;
        const int r2 = ib2 + bwrap[3 * bin + 2] - O2 - H + 1;
        const int a0 = max(r0, 0), e0 = min(r0 + W - 1, T0 - 1);
        const int a1 = max(r1, 0), e1 = min(r1 + W - 1, T1 - 1);
        const int a2 = max(r2, 0), e2 = min(r2 + W - 1, T2 - 1);
        if (a0 > e0 || a1 > e1 || a2 > e2) continue;  // warp-uniform
        const T f0 = R.f[0], f1 = R.f[1], f2 = R.f[2];
        const T q0 = R.q[0], q1 = R.q[1], q2 = R.q[2];
        __syncwarp();
        for (int i = lane; i < 3 * W; i += 32) {
            const int d = i / W, t = i - d * W;
            const T f = d == 0 ? f0 : (d == 1 ? f1 : f2);
            kw[i] = kb_eval((f + (T)(H - 1 - t)) * ((T)2 / (T)W), zeta, inorm);
        }
        __syncwarp();
        // lanes over (row, z): rows = (x, y) pairs of the support box
        const int n0 = e0 - a0 + 1, n1 = e1 - a1 + 1, n2 = e2 - a2 + 1;
        const int rows_per = 32 / n2;
        const int rsub = lane / n2, c2 = lane - rsub * n2;
        if (rsub < rows_per) {
            const int x2 = a2 + c2;
            const T wz = kw[2 * W + x2 - r2];
            const int nrows = n0 * n1;
            for (int r = rsub; r < nrows; r += rows_per) {
                const int c0 = r / n1, c1 = r - c0 * n1;
                const int x0 = a0 + c0, x1 = a1 + c1;
                const T wv = kw[x0 - r0] * kw[W + x1 - r1] * wz;
                const int cell = (x0 * T1 + x1) * T2P + x2;
                atomicAdd(&acc[cell], wv * q0);
                atomicAdd(&acc[tsz + cell], wv * q1);
                atomicAdd(&acc[2 * tsz + cell], wv * q2);
            }
        }
    }
    __syncthreads();
    const size_t gsz = (size_t)P.ng[0] * P.ng[1] * P.ng[2];
    const int tcount = T0 * T1 * T2;
    for (int i = tid; i < tcount; i += blockDim.x) {
        const int x2 = i % T2, x1 = (i / T2) % T1, x0 = i / (T1 * T2);
        const int si = (x0 * T1 + x1) * T2P + x2;
        const size_t gi = ((size_t)(O0 + x0) * P.ng[1] + (O1 + x1)) * P.ng[2] + (O2 + x2);
        grid[gi] = acc[si];
        grid[gsz + gi] = acc[tsz + si];
        grid[2 * gsz + gi] = acc[2 * tsz + si];
    }
}

template <typename T> struct Cplx;
template <> struct Cplx<float> { using t = float2; };
template <> struct Cplx<double> { using t = double2; };

// k-space pass over the half spectrum (R2C layout, last axis 0..ng2/2):
//   omega_k = (kappa/V) F_k / prod_d F_d(m_d)      (type-1 deconvolution)
//   vhat_k  = i k x omega_k e^{-k^2/4alpha^2} / k^2 / prod_d F_d(m_d)
//   psihat  = omega_k e^{-k^2/4alpha^2} / k^2 / prod_d F_d(m_d)
// for |m_d| <= K_d, m != 0; every other mode is written as zero.  tab_d[m]
// holds e^{-k_d^2/4alpha^2} / F_d(m)^2.
template <typename T>
__global__ void k_kspace(KspaceP P, typename Cplx<T>::t* __restrict__ spec, typename Cplx<T>::t* __restrict__ spsi,
                         const T* __restrict__ tab0, const T* __restrict__ tab1, const T* __restrict__ tab2)
{
    using C = typename Cplx<T>::t;
    const long long n1h = (long long)P.ng[1] * P.nh;
    const long long tot = (long long)P.ng[0] * n1h;
    double esum = 0.0;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i2 = (int)(idx % P.nh);
        const int i1 = (int)((idx / P.nh) % P.ng[1]);
        const int i0 = (int)(idx / n1h);
        const int m0 = i0 <= P.ng[0] / 2 ? i0 : i0 - P.ng[0];
        const int m1 = i1 <= P.ng[1] / 2 ? i1 : i1 - P.ng[1];
        const int m2 = i2;
        const int a0 = m0 < 0 ? -m0 : m0, a1 = m1 < 0 ? -m1 : m1;
        C z;
        z.x = 0;
        z.y = 0;
        if (a0 > P.K[0] || a1 > P.K[1] || m2 > P.K[2] || (m0 == 0 && m1 == 0 && m2 == 0)) {
            spec[idx] = z;
            spec[tot + idx] = z;
            spec[2 * tot + idx] = z;
            if (spsi) {
                spsi[idx] = z;
                spsi[tot + idx] = z;
                spsi[2 * tot + idx] = z;
            }
            continue;
        }
        const T k0 = (T)(P.kk[0] * m0), k1 = (T)(P.kk[1] * m1), k2 = (T)(P.kk[2] * m2);
        const T ksq = k0 * k0 + k1 * k1 + k2 * k2;
        const T mult = (T)P.scale * tab0[a0] * tab1[a1] * tab2[m2] / ksq;
        const C f0 = spec[idx], f1 = spec[tot + idx], f2 = spec[2 * tot + idx];
        if (P.energy) {
            const double a2 = (double)f0.x * f0.x + (double)f0.y * f0.y + (double)f1.x * f1.x +
                              (double)f1.y * f1.y + (double)f2.x * f2.x + (double)f2.y * f2.y;
            esum += (m2 > 0 ? 1.0 : 0.5) * P.scale * (double)mult * a2;
        }
        const T w0r = f0.x * mult, w0i = f0.y * mult;
        const T w1r = f1.x * mult, w1i = f1.y * mult;
        const T w2r = f2.x * mult, w2i = f2.y * mult;
        // k x w (k real), then multiply by i: (a + ib) i = -b + ia
        const T cr0 = k1 * w2r - k2 * w1r, ci0 = k1 * w2i - k2 * w1i;
        const T cr1 = k2 * w0r - k0 * w2r, ci1 = k2 * w0i - k0 * w2i;
        const T cr2 = k0 * w1r - k1 * w0r, ci2 = k0 * w1i - k1 * w0i;
        C o;
        o.x = -ci0; o.y = cr0; spec[idx] = o;
        o.x = -ci1; o.y = cr1; spec[tot + idx] = o;
        o.x = -ci2; o.y = cr2; spec[2 * tot + idx] = o;
        if (spsi) {
            o.x = w0r; o.y = w0i; spsi[idx] = o;
            o.x = w1r; o.y = w1i; spsi[tot + idx] = o;
            o.x = w2r; o.y = w2i; spsi[2 * tot + idx] = o;
        }
    }
    if (P.energy) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) esum += __shfl_xor_sync(0xffffffffu, esum, o);
        if ((threadIdx.x & 31) == 0 && esum != 0.0) atomicAdd(P.energy, esum);
    }
}

// Type-2 interpolation at the nodes, plus the epilogue sum
//   out = add_d (float64: local - self) + add_t (short range, float64) + interp.
// part (optional) receives the interpolated long-range part alone.  The
// weights of the last two axes live in registers (static indices); those of
// the first axis are computed in the outer loop.
template <typename T, int W>
__global__ void __launch_bounds__(128) k_interp(InterpP P, const double* __restrict__ nodes, const T* __restrict__ grid,
                                                const double* __restrict__ add_d, const double* __restrict__ add_t,
                                                double* __restrict__ out, double* __restrict__ part)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.N) return;
    constexpr int H = W / 2;
    const T zeta = (T)P.zeta;
    const T inorm = (T)P.inorm;
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
    T ky[W], kz[W];
    int iy[W], iz[W];
#pragma unroll
    for (int t = 0; t < W; ++t) {
        ky[t] = kb_eval((fr[1] + (T)(H - 1 - t)) * ((T)2 / (T)W), zeta, inorm);
        kz[t] = kb_eval((fr[2] + (T)(H - 1 - t)) * ((T)2 / (T)W), zeta, inorm);
        int gy = ib[1] - H + 1 + t, gz = ib[2] - H + 1 + t;
        iy[t] = gy < 0 ? gy + P.ng[1] : (gy >= P.ng[1] ? gy - P.ng[1] : gy);
        iz[t] = gz < 0 ? gz + P.ng[2] : (gz >= P.ng[2] ? gz - P.ng[2] : gz);
    }
    const size_t gsz = (size_t)P.ng[0] * P.ng[1] * P.ng[2];
    T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll 1
    for (int p = 0; p < W; ++p) {
        const T kx = kb_eval((fr[0] + (T)(H - 1 - p)) * ((T)2 / (T)W), zeta, inorm);
        int gx = ib[0] - H + 1 + p;
        gx = gx < 0 ? gx + P.ng[0] : (gx >= P.ng[0] ? gx - P.ng[0] : gx);
        const size_t plane = (size_t)gx * P.ng[1];
#pragma unroll
        for (int q = 0; q < W; ++q) {
            const T wpq = kx * ky[q];
            const size_t row = (plane + iy[q]) * P.ng[2];
#pragma unroll
            for (int r = 0; r < W; ++r) {
                const size_t gi = row + iz[r];
                const T wv = wpq * kz[r];
                a0 += wv * grid[gi];
                a1 += wv * grid[gsz + gi];
                a2 += wv * grid[2 * gsz + gi];
            }
        }
    }
    if (part) {
        part[3 * j + 0] = (double)a0;
        part[3 * j + 1] = (double)a1;
        part[3 * j + 2] = (double)a2;
    }
    if (out) {
        double o0 = (double)a0, o1 = (double)a1, o2 = (double)a2;
        if (add_t) {
            o0 += (double)add_t[3 * j + 0];
            o1 += (double)add_t[3 * j + 1];
            o2 += (double)add_t[3 * j + 2];
        }
        if (add_d) {
            o0 += add_d[3 * j + 0];
            o1 += add_d[3 * j + 1];
            o2 += add_d[3 * j + 2];
        }
        out[3 * j + 0] = o0;
        out[3 * j + 1] = o1;
        out[3 * j + 2] = o2;
    }
}

template <typename T>
__global__ void k_to_double(const T* __restrict__ in, double* __restrict__ out, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = (double)in[i];
}

template <typename T>
static size_t spread_smem(const SpreadP& P)
{
    return sizeof(T) * (3 * (size_t)P.tile[0] * P.tile[1] * (P.tile[2] + 1) + (kThreads / 32) * 3 * (size_t)P.w) +
           sizeof(int) * (27 + 28 + 81);
}

template <typename T, int W>
static cudaError_t spread_w(const SpreadP& P, const Work& w, int ntiles, cudaStream_t s)
{
    const size_t sm = spread_smem<T>(P);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_spread<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_spread<T, W><<<ntiles, kThreads, sm, s>>>(P, w.tile_cnt, (const LrRec<T>*)w.lr_sorted, (T*)w.grid);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_spread(const SpreadP& P, const Work& w, int ntiles, cudaStream_t s)
{
    switch (P.w) {
    case 2: return spread_w<T, 2>(P, w, ntiles, s);
    case 4: return spread_w<T, 4>(P, w, ntiles, s);
    case 6: return spread_w<T, 6>(P, w, ntiles, s);
    case 8: return spread_w<T, 8>(P, w, ntiles, s);
    case 10: return spread_w<T, 10>(P, w, ntiles, s);
    case 12: return spread_w<T, 12>(P, w, ntiles, s);
    case 14: return spread_w<T, 14>(P, w, ntiles, s);
    case 16: return spread_w<T, 16>(P, w, ntiles, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
cudaError_t launch_kspace(const KspaceP& P, const Work& w, cudaStream_t s)
{
    using C = typename Cplx<T>::t;
    const long long tot = (long long)P.ng[0] * P.ng[1] * P.nh;
    const int tb = 256;
    long long g = (tot + tb - 1) / tb;
    if (g > 152LL * 64) g = 152LL * 64;
    const T* tab = (const T*)w.ktab;
    const T* tab0 = tab;
    const T* tab1 = tab0 + (P.K[0] + 1);
    const T* tab2 = tab1 + (P.K[1] + 1);
    k_kspace<T><<<(int)g, tb, 0, s>>>(P, (C*)w.spec, P.want_psi ? (C*)w.spec_psi : nullptr, tab0, tab1, tab2);
    return cudaGetLastError();
}

template <typename T, int W>
static cudaError_t interp_w(const InterpP& P, const double* nodes, const void* grid, const double* add_d, const double* add_t,
                            double* out, double* part, cudaStream_t s)
{
    const int tb = 128;
    k_interp<T, W><<<(P.N + tb - 1) / tb, tb, 0, s>>>(P, nodes, (const T*)grid, add_d, add_t, out, part);
    return cudaGetLastError();
}

// what: 0 velocity (adds vls + vsr), 1 streamfunction (adds pls + psr),
// 2 the long-range part alone (written to part_long).
template <typename T>
cudaError_t launch_interp(const InterpP& P, const double* nodes, const Work& w, const void* grid, int what,
                          double* out, double* part_long, cudaStream_t s)
{
    if (P.N <= 0) return cudaSuccess;
    const double* add_d = nullptr;
    const double* add_t = nullptr;
    if (what == 0) { add_d = w.vls; add_t = w.vsr; }
    if (what == 1) { add_d = w.pls; add_t = w.psr; }
    if (what == 2) out = nullptr;
    switch (P.w) {
    case 2: return interp_w<T, 2>(P, nodes, grid, add_d, add_t, out, part_long, s);
    case 4: return interp_w<T, 4>(P, nodes, grid, add_d, add_t, out, part_long, s);
    case 6: return interp_w<T, 6>(P, nodes, grid, add_d, add_t, out, part_long, s);
    case 8: return interp_w<T, 8>(P, nodes, grid, add_d, add_t, out, part_long, s);
    case 10: return interp_w<T, 10>(P, nodes, grid, add_d, add_t, out, part_long, s);
    case 12: return interp_w<T, 12>(P, nodes, grid, add_d, add_t, out, part_long, s);
    case 14: return interp_w<T, 14>(P, nodes, grid, add_d, add_t, out, part_long, s);
    case 16: return interp_w<T, 16>(P, nodes, grid, add_d, add_t, out, part_long, s);
    default: return cudaErrorInvalidValue;
    }
}

// The velocity (or the long-range part alone) from the accumulated
// long-range sums of the fused inverse-z interpolation, with the same sum
// order as the interpolation kernel's epilogue.
template <typename T>
__device__ __forceinline__ void k_interp_sum_body(int n3, const T* __restrict__ acc,
                                                  const double* __restrict__ add_d, const double* __restrict__ add_t,
                                                  double* __restrict__ out, double* __restrict__ part,
                                                  int bid, int nb)
{
    for (int i = bid * blockDim.x + threadIdx.x; i < n3; i += nb * blockDim.x) {
        const double a = (double)acc[i];
        if (part) part[i] = a;
        if (out) out[i] = (a + (double)add_t[i]) + add_d[i];
    }
}

template <typename T>
__global__ void k_interp_sum(int n3, const T* __restrict__ acc, const double* __restrict__ add_d,
                             const double* __restrict__ add_t, double* __restrict__ out, double* __restrict__ part)
{
    k_interp_sum_body<T>(n3, acc, add_d, add_t, out, part, blockIdx.x, gridDim.x);
}

template <typename T>
__global__ void k_interp_sum_b(const SumD<T>* __restrict__ d, const int* __restrict__ bs, int n)
{
    int bid, nb;
    const SumD<T>& a = d[batch_member(bs, n, bid, nb)];
    k_interp_sum_body<T>(a.n3, a.acc, a.add_d, a.add_t, a.out, nullptr, bid, nb);
}

template <typename T>
cudaError_t launch_interp_sum_b(const BatchL& L, cudaStream_t s)
{
    if (L.total > 0) k_interp_sum_b<T><<<L.total, 256, 0, s>>>((const SumD<T>*)L.desc, L.bstart, L.n);
    return cudaGetLastError();
}

template cudaError_t launch_interp_sum_b<float>(const BatchL&, cudaStream_t);
template cudaError_t launch_interp_sum_b<double>(const BatchL&, cudaStream_t);

template <typename T>
cudaError_t launch_interp_sum(int N, const Work& w, int what, double* out, double* part_long, cudaStream_t s)
{
    if (N <= 0) return cudaSuccess;
    const int n3 = 3 * N;
    int g = (n3 + 255) / 256;
    if (g > 4096) g = 4096;
    k_interp_sum<T><<<g, 256, 0, s>>>(n3, (const T*)w.vacc, w.vls, w.vsr, what == 2 ? nullptr : out,
                                      part_long);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_to_double(const void* in, double* out, int n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    int g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    k_to_double<T><<<g, 256, 0, s>>>((const T*)in, out, n);
    return cudaGetLastError();
}

template cudaError_t launch_spread<float>(const SpreadP&, const Work&, int, cudaStream_t);
template cudaError_t launch_spread<double>(const SpreadP&, const Work&, int, cudaStream_t);
template cudaError_t launch_kspace<float>(const KspaceP&, const Work&, cudaStream_t);
template cudaError_t launch_kspace<double>(const KspaceP&, const Work&, cudaStream_t);
template cudaError_t launch_interp<float>(const InterpP&, const double*, const Work&, const void*, int, double*,
                                          double*, cudaStream_t);
template cudaError_t launch_interp<double>(const InterpP&, const double*, const Work&, const void*, int, double*,
                                           double*, cudaStream_t);
template cudaError_t launch_interp_sum<float>(int, const Work&, int, double*, double*, cudaStream_t);
template cudaError_t launch_interp_sum<double>(int, const Work&, int, double*, double*, cudaStream_t);
template cudaError_t launch_to_double<float>(const void*, double*, int, cudaStream_t);
template cudaError_t launch_to_double<double>(const void*, double*, int, cudaStream_t);

}  // namespace bsw
