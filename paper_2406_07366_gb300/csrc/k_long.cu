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
    const int tsz = T0 * T1 * T2;
    T* acc = reinterpret_cast<T*>(smem_raw);
    T* ktab = acc + 3 * tsz;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const int b = blockIdx.x;
    const int nt0 = P.ntile[0], nt1 = P.ntile[1], nt2 = P.ntile[2];
    const int t0 = b % nt0, t1 = (b / nt0) % nt1, t2 = b / (nt0 * nt1);
    const int O0 = t0 * T0, O1 = t1 * T1, O2 = t2 * T2;
    for (int i = tid; i < 3 * tsz; i += blockDim.x) acc[i] = (T)0;
    __syncthreads();

    const T zeta = (T)P.zeta;
    const T inorm = (T)(1.0 / (1.0 - exp(-2.0 * P.zeta)));
    T* kw = ktab + wid * 3 * W;
    constexpr int H = W / 2;
    for (int d2 = -1; d2 <= 1; ++d2) {
        int u2 = t2 + d2, w2 = 0;
        if (u2 < 0) { u2 += nt2; w2 = -1; } else if (u2 >= nt2) { u2 -= nt2; w2 = 1; }
        for (int d1 = -1; d1 <= 1; ++d1) {
            int u1 = t1 + d1, w1 = 0;
            if (u1 < 0) { u1 += nt1; w1 = -1; } else if (u1 >= nt1) { u1 -= nt1; w1 = 1; }
            for (int d0 = -1; d0 <= 1; ++d0) {
                int u0 = t0 + d0, w0 = 0;
                if (u0 < 0) { u0 += nt0; w0 = -1; } else if (u0 >= nt0) { u0 -= nt0; w0 = 1; }
                const int nb = u0 + nt0 * (u1 + nt1 * u2);
                const int s0 = tstart[nb], s1 = tstart[nb + 1];
                for (int k = s0 + wid; k < s1; k += nw) {
                    const LrRec<T> R = pts[k];
                    const int ib0 = R.base & 1023, ib1 = (R.base >> 10) & 1023, ib2 = (R.base >> 20) & 1023;
                    // first support cell relative to the tile origin (unwrapped image)
                    const int r0 = ib0 + w0 * P.ng[0] - O0 - H + 1;
                    const int r1 = ib1 + w1 * P.ng[1] - O1 - H + 1;
                    const int r2 = ib2 + w2 * P.ng[2] - O2 - H + 1;
                    const int a0 = max(r0, 0), e0 = min(r0 + W - 1, T0 - 1);
                    const int a1 = max(r1, 0), e1 = min(r1 + W - 1, T1 - 1);
                    const int a2 = max(r2, 0), e2 = min(r2 + W - 1, T2 - 1);
                    if (a0 > e0 || a1 > e1 || a2 > e2) continue;  // warp-uniform
                    __syncwarp();
                    for (int i = lane; i < 3 * W; i += 32) {
                        const int d = i / W, t = i - d * W;
                        const T z = (R.f[d] + (T)(H - 1 - t)) * ((T)2 / (T)W);
                        kw[i] = kb_eval(z, zeta, inorm);
                    }
                    __syncwarp();
                    const int n0 = e0 - a0 + 1, n1 = e1 - a1 + 1, n2 = e2 - a2 + 1;
                    const int tot = n0 * n1 * n2;
                    for (int e = lane; e < tot; e += 32) {
                        const int c2 = e % n2;
                        const int rest = e / n2;
                        const int c1 = rest % n1, c0 = rest / n1;
                        const int x0 = a0 + c0, x1 = a1 + c1, x2 = a2 + c2;
                        const T wv = kw[x0 - r0] * kw[W + x1 - r1] * kw[2 * W + x2 - r2];
                        const int cell = (x0 * T1 + x1) * T2 + x2;
                        atomicAdd(&acc[cell], wv * R.q[0]);
                        atomicAdd(&acc[tsz + cell], wv * R.q[1]);
                        atomicAdd(&acc[2 * tsz + cell], wv * R.q[2]);
                    }
                }
            }
        }
    }
    __syncthreads();
    const size_t gsz = (size_t)P.ng[0] * P.ng[1] * P.ng[2];
    for (int i = tid; i < tsz; i += blockDim.x) {
        const int x2 = i % T2, x1 = (i / T2) % T1, x0 = i / (T1 * T2);
        const size_t gi = ((size_t)(O0 + x0) * P.ng[1] + (O1 + x1)) * P.ng[2] + (O2 + x2);
        grid[gi] = acc[i];
        grid[gsz + gi] = acc[tsz + i];
        grid[2 * gsz + gi] = acc[2 * tsz + i];
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
}

// Type-2 interpolation at the nodes, plus the epilogue sum
//   out = add_d (float64: local - self) + add_t (short range, T) + interp.
// part (optional) receives the interpolated long-range part alone.
template <typename T, int W>
__global__ void __launch_bounds__(128) k_interp(InterpP P, const double* __restrict__ nodes, const T* __restrict__ grid,
                                                const double* __restrict__ add_d, const T* __restrict__ add_t,
                                                double* __restrict__ out, double* __restrict__ part)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.N) return;
    constexpr int H = W / 2;
    const T zeta = (T)P.zeta;
    const T inorm = (T)(1.0 / (1.0 - exp(-2.0 * P.zeta)));
    T kv[3][W];
    int ix[3][W];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double x = nodes[3 * j + d];
        if (!isfinite(x)) x = 0.0;
        double xw = x - P.L[d] * floor(x / P.L[d]);
        if (xw >= P.L[d]) xw -= P.L[d];
        if (xw < 0.0) xw = 0.0;
        const double g = xw / P.hg[d];
        int ib = (int)floor(g);
        ib = ib < 0 ? 0 : (ib >= P.ng[d] ? P.ng[d] - 1 : ib);
        double fr = g - (double)ib;
        fr = fr < 0.0 ? 0.0 : (fr > 1.0 ? 1.0 : fr);
        const T f = (T)fr;
#pragma unroll
        for (int t = 0; t < W; ++t) {
            kv[d][t] = kb_eval((f + (T)(H - 1 - t)) * ((T)2 / (T)W), zeta, inorm);
            int gi = ib - H + 1 + t;
            gi = gi < 0 ? gi + P.ng[d] : (gi >= P.ng[d] ? gi - P.ng[d] : gi);
            ix[d][t] = gi;
        }
    }
    const size_t gsz = (size_t)P.ng[0] * P.ng[1] * P.ng[2];
    T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll 1
    for (int p = 0; p < W; ++p) {
        for (int q = 0; q < W; ++q) {
            const T wpq = kv[0][p] * kv[1][q];
            const size_t row = ((size_t)ix[0][p] * P.ng[1] + ix[1][q]) * P.ng[2];
#pragma unroll
            for (int r = 0; r < W; ++r) {
                const size_t gi = row + ix[2][r];
                const T wv = wpq * kv[2][r];
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
    return sizeof(T) * (3 * (size_t)P.tile[0] * P.tile[1] * P.tile[2] + (kThreads / 32) * 3 * (size_t)P.w);
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
static cudaError_t interp_w(const InterpP& P, const double* nodes, const void* grid, const double* add_d, const T* add_t,
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
    const T* add_t = nullptr;
    if (what == 0) { add_d = w.vls; add_t = (const T*)w.vsr; }
    if (what == 1) { add_d = w.pls; add_t = (const T*)w.psr; }
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
template cudaError_t launch_to_double<float>(const void*, double*, int, cudaStream_t);
template cudaError_t launch_to_double<double>(const void*, double*, int, cudaStream_t);

}  // namespace bsw
