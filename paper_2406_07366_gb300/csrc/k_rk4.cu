// Classical fourth-order Runge-Kutta update of the node positions
// (Sec. 5.2: ds_i/dt = v(s_i), advanced with RK4, the spline refitted at
// every stage because every velocity evaluation refits it).
//   stage:  out = x0 + c k
//   final:  x  += h/6 (k1 + 2 k2 + 2 k3 + k4)
#include "bs_internal.cuh"

namespace bsw {

__global__ void k_rk4_stage(const double* __restrict__ x0, const double* __restrict__ k, double c,
                            double* __restrict__ out, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = x0[i] + c * k[i];
}

__global__ void k_rk4_final(double* __restrict__ x, const double* __restrict__ k1, const double* __restrict__ k2,
                            const double* __restrict__ k3, const double* __restrict__ k4, double h6, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] += h6 * (k1[i] + 2.0 * (k2[i] + k3[i]) + k4[i]);
}

static int rk4_blocks(long long n)
{
    const long long b = (n + 255) / 256;
    return (int)(b < 152 * 8 ? (b > 0 ? b : 1) : 152 * 8);
}

cudaError_t launch_rk4_stage(const double* x0, const double* k, double c, double* out, long long n, cudaStream_t s)
{
    k_rk4_stage<<<rk4_blocks(n), 256, 0, s>>>(x0, k, c, out, n);
    return cudaGetLastError();
}

cudaError_t launch_rk4_final(double* x, const double* k1, const double* k2, const double* k3, const double* k4,
                             double h, long long n, cudaStream_t s)
{
    k_rk4_final<<<rk4_blocks(n), 256, 0, s>>>(x, k1, k2, k3, k4, h / 6.0, n);
    return cudaGetLastError();
}

}  // namespace bsw
