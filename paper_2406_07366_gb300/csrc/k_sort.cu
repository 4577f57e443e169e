// Counting sorts that bin the quadrature sources: by short-range cell (the
// cell lists of Sec. 5.3) and by spreading tile (the long-range spread).
// count (atomics) -> exclusive scan (three launches, no inter-block waits)
// -> scatter of the records into their bins.
#include "bs_internal.cuh"

namespace bsw {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

int scan_blocks(int n) { return (n + 1 + kScanTile - 1) / kScanTile; }

__device__ __forceinline__ void count_body(const int* __restrict__ key, int n, int* __restrict__ cnt, int bid, int nb)
{
    for (int i = bid * blockDim.x + threadIdx.x; i < n; i += nb * blockDim.x) atomicAdd(&cnt[key[i]], 1);
}

__global__ void k_count(const int* __restrict__ key, int n, int* __restrict__ cnt)
{
    count_body(key, n, cnt, blockIdx.x, gridDim.x);
}

// Block-wide inclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ int block_scan_incl(int v, int* sh_warp, int& total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) sh_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int w = (lane < (int)(blockDim.x >> 5)) ? sh_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        sh_warp[lane] = w;
    }
    __syncthreads();
    total = sh_warp[(blockDim.x >> 5) - 1];
    int add = (wid > 0) ? sh_warp[wid - 1] : 0;
    __syncthreads();
    return v + add;
}

// Phase 1: per-tile sums of cnt[0..n] (entry n counts as 0).
__device__ __forceinline__ void scan_reduce_body(const int* __restrict__ cnt, int n, int* __restrict__ part, int bid)
{
    __shared__ int sh[32];
    const int base = bid * kScanTile + threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int i = base + k;
        if (i < n) s += cnt[i];
    }
    int total;
    block_scan_incl(s, sh, total);
    if (threadIdx.x == 0) part[bid] = total;
}

__global__ void k_scan_reduce(const int* __restrict__ cnt, int n, int* __restrict__ part)
{
    scan_reduce_body(cnt, n, part, blockIdx.x);
}

// Phase 2: exclusive scan of the tile sums, one block, looping.
__device__ __forceinline__ void scan_parts_body(int* __restrict__ part, int nb)
{
    __shared__ int sh[32];
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int i = b0 + threadIdx.x;
        const int v = (i < nb) ? part[i] : 0;
        int total;
        const int inc = block_scan_incl(v, sh, total);
        if (i < nb) part[i] = carry + inc - v;
        carry += total;
        __syncthreads();
    }
}

__global__ void k_scan_parts(int* __restrict__ part, int nb) { scan_parts_body(part, nb); }

// Phase 3: exclusive scan within each tile plus its offset, in place over
// cnt[0..n]; cnt[n] becomes the grand total.
__device__ __forceinline__ void scan_apply_body(int* __restrict__ cnt, int n, const int* __restrict__ part, int bid)
{
    __shared__ int sh[32];
    const int base = bid * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int i = base + k;
        v[k] = (i < n) ? cnt[i] : 0;
        s += v[k];
    }
    int total;
    const int inc = block_scan_incl(s, sh, total);
    int run = part[bid] + inc - s;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int i = base + k;
        if (i <= n) cnt[i] = run;
        run += v[k];
    }
}

__global__ void k_scan_apply(int* __restrict__ cnt, int n, const int* __restrict__ part)
{
    scan_apply_body(cnt, n, part, blockIdx.x);
}

cudaError_t scan_exclusive(int* cnt, int n, int* tmp, cudaStream_t s)
{
    const int nb = scan_blocks(n);
    k_scan_reduce<<<nb, kScanThreads, 0, s>>>(cnt, n, tmp);
    k_scan_parts<<<1, kScanThreads, 0, s>>>(tmp, nb);
    k_scan_apply<<<nb, kScanThreads, 0, s>>>(cnt, n, tmp);
    return cudaGetLastError();
}

// The order inside a bin follows the atomics; idx_out (if non-null) records
// each copy's source index so that the bins can be re-ordered by it.
template <typename R>
__device__ __forceinline__ void scatter_body(const int* __restrict__ key, const R* __restrict__ in, int n,
                                             int* __restrict__ cur, R* __restrict__ out, int* __restrict__ idx_out,
                                             int bid, int nb)
{
    for (int i = bid * blockDim.x + threadIdx.x; i < n; i += nb * blockDim.x) {
        const int p = atomicAdd(&cur[key[i]], 1);
        out[p] = in[i];
        if (idx_out) idx_out[p] = i;
    }
}

template <typename R>
__global__ void k_scatter(const int* __restrict__ key, const R* __restrict__ in, int n, int* __restrict__ cur,
                          R* __restrict__ out, int* __restrict__ idx_out)
{
    scatter_body<R>(key, in, n, cur, out, idx_out, blockIdx.x, gridDim.x);
}

// ---- batched forms (one launch for every member of a batch) ----
__global__ void k_zero_b(const ZeroD* __restrict__ d, const int* __restrict__ bs, int n)
{
    int bid, nb;
    const ZeroD& a = d[batch_member(bs, n, bid, nb)];
    for (int i = bid * blockDim.x + threadIdx.x; i < a.n; i += nb * blockDim.x) a.p[i] = 0;
}

__global__ void k_copy_b(const CopyD* __restrict__ d, const int* __restrict__ bs, int n)
{
    int bid, nb;
    const CopyD& a = d[batch_member(bs, n, bid, nb)];
    for (int i = bid * blockDim.x + threadIdx.x; i < a.n; i += nb * blockDim.x) a.dst[i] = a.src[i];
}

__global__ void k_count_b(const CountD* __restrict__ d, const int* __restrict__ bs, int n)
{
    int bid, nb;
    const CountD& a = d[batch_member(bs, n, bid, nb)];
    count_body(a.key, a.n, a.cnt, bid, nb);
}

__global__ void k_scan_reduce_b(const ScanD* __restrict__ d, const int* __restrict__ bs, int n)
{
    int bid, nb;
    const ScanD& a = d[batch_member(bs, n, bid, nb)];
    scan_reduce_body(a.cnt, a.n, a.part, bid);
}

__global__ void k_scan_parts_b(const ScanD* __restrict__ d, int n)
{
    const ScanD& a = d[blockIdx.x];
    scan_parts_body(a.part, a.nb);
}

__global__ void k_scan_apply_b(const ScanD* __restrict__ d, const int* __restrict__ bs, int n)
{
    int bid, nb;
    const ScanD& a = d[batch_member(bs, n, bid, nb)];
    scan_apply_body(a.cnt, a.n, a.part, bid);
}

template <typename R>
__global__ void k_scatter_b(const ScatterD<R>* __restrict__ d, const int* __restrict__ bs, int n)
{
    int bid, nb;
    const ScatterD<R>& a = d[batch_member(bs, n, bid, nb)];
    scatter_body<R>(a.key, a.in, a.n, a.cur, a.out, nullptr, bid, nb);
}

cudaError_t launch_zero_b(const BatchL& L, cudaStream_t s)
{
    if (L.total > 0) k_zero_b<<<L.total, L.threads, 0, s>>>((const ZeroD*)L.desc, L.bstart, L.n);
    return cudaGetLastError();
}

cudaError_t launch_copy_b(const BatchL& L, cudaStream_t s)
{
    if (L.total > 0) k_copy_b<<<L.total, L.threads, 0, s>>>((const CopyD*)L.desc, L.bstart, L.n);
    return cudaGetLastError();
}

cudaError_t launch_count_b(const BatchL& L, cudaStream_t s)
{
    if (L.total > 0) k_count_b<<<L.total, L.threads, 0, s>>>((const CountD*)L.desc, L.bstart, L.n);
    return cudaGetLastError();
}

cudaError_t launch_scan_b(const BatchL& L1, const BatchL& L2, cudaStream_t s)
{
    if (L1.total <= 0) return cudaSuccess;
    k_scan_reduce_b<<<L1.total, kScanThreads, 0, s>>>((const ScanD*)L1.desc, L1.bstart, L1.n);
    k_scan_parts_b<<<L2.n, kScanThreads, 0, s>>>((const ScanD*)L2.desc, L2.n);
    k_scan_apply_b<<<L1.total, kScanThreads, 0, s>>>((const ScanD*)L1.desc, L1.bstart, L1.n);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_scatter_b(const BatchL& L, cudaStream_t s)
{
    if (L.total > 0) k_scatter_b<R><<<L.total, L.threads, 0, s>>>((const ScatterD<R>*)L.desc, L.bstart, L.n);
    return cudaGetLastError();
}

template cudaError_t launch_scatter_b<SrRec<float>>(const BatchL&, cudaStream_t);
template cudaError_t launch_scatter_b<SrRec<double>>(const BatchL&, cudaStream_t);

// Warp per segment [start[s], start[s+1]): the copy with the r-th smallest key
// goes to position start[s] + r (keys are distinct within a segment), records
// moved as 16-byte words.
__global__ void k_segsort(const int* __restrict__ start, int nseg, const int4* __restrict__ in,
                          const int* __restrict__ key, int4* __restrict__ out, int words)
{
    const int lane = threadIdx.x & 31;
    const int sg = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (sg >= nseg) return;
    const int s0 = start[sg], n = start[sg + 1] - s0;
    for (int a = lane; a < n; a += 32) {
        const int ka = key[s0 + a];
        int rank = 0;
        for (int b = 0; b < n; ++b) rank += key[s0 + b] < ka;
        const int4* src = in + (size_t)(s0 + a) * words;
        int4* dst = out + (size_t)(s0 + rank) * words;
        for (int k = 0; k < words; ++k) dst[k] = src[k];
    }
}

cudaError_t launch_segsort_bytes(const int* start, int nseg, const void* in, const int* key, void* out,
                                 size_t rec_bytes, cudaStream_t s)
{
    if (nseg <= 0) return cudaSuccess;
    const int tb = 256;
    const long long threads = 32LL * nseg;
    k_segsort<<<(unsigned)((threads + tb - 1) / tb), tb, 0, s>>>(start, nseg, (const int4*)in, key, (int4*)out,
                                                                 (int)(rec_bytes / 16));
    return cudaGetLastError();
}

// Warp per segment [start[s], start[s+1]): its pairs in increasing order of
// .x (distinct within a segment).
__global__ void k_segsort_int2(const int* __restrict__ start, int nseg, const int2* __restrict__ in,
                               int2* __restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int sg = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (sg >= nseg) return;
    const int s0 = start[sg], n = start[sg + 1] - s0;
    for (int a = lane; a < n; a += 32) {
        const int2 ea = in[s0 + a];
        int rank = 0;
        for (int b = 0; b < n; ++b) rank += in[s0 + b].x < ea.x;
        out[s0 + rank] = ea;
    }
}

cudaError_t launch_segsort_int2(const int* start, int nseg, const int2* in, int2* out, cudaStream_t s)
{
    if (nseg <= 0) return cudaSuccess;
    const int tb = 256;
    const long long threads = 32LL * nseg;
    k_segsort_int2<<<(unsigned)((threads + tb - 1) / tb), tb, 0, s>>>(start, nseg, in, out);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_segsort(const int* start, int nseg, const R* in, const int* key, R* out, cudaStream_t s)
{
    static_assert(sizeof(R) % 16 == 0, "records are moved as 16-byte words");
    return launch_segsort_bytes(start, nseg, in, key, out, sizeof(R), s);
}

template <typename R>
static cudaError_t sort_records(const int* key, const R* in, R* out, int n, int* cnt, int* cur, int nbins, int* tmp,
                                cudaStream_t s, int* idx_out = nullptr)
{
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)(nbins + 1), s);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        const int g = (n + kThreads - 1) / kThreads;
        k_count<<<g, kThreads, 0, s>>>(key, n, cnt);
    }
    e = scan_exclusive(cnt, nbins, tmp, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(cur, cnt, sizeof(int) * (size_t)nbins, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        const int g = (n + kThreads - 1) / kThreads;
        k_scatter<R><<<g, kThreads, 0, s>>>(key, in, n, cur, out, idx_out);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sort_sr(const Work& w, int NQ, int ncells, cudaStream_t s, bool det)
{
    if (!det)
        return sort_records<SrRec<T>>(w.sr_key, (const SrRec<T>*)w.sr_rec, (SrRec<T>*)w.sr_sorted, NQ, w.cell_cnt,
                                      w.cell_cur, ncells, w.scan_tmp, s);
    // deterministic: bin into the second buffer with the source indices, then
    // order every cell by source index
    cudaError_t e = sort_records<SrRec<T>>(w.sr_key, (const SrRec<T>*)w.sr_rec, (SrRec<T>*)w.sr_sorted2, NQ,
                                           w.cell_cnt, w.cell_cur, ncells, w.scan_tmp, s, w.sr_idx);
    if (e != cudaSuccess) return e;
    return launch_segsort<SrRec<T>>(w.cell_cnt, ncells, (const SrRec<T>*)w.sr_sorted2, w.sr_idx,
                                    (SrRec<T>*)w.sr_sorted, s);
}

template <typename T>
cudaError_t launch_sort_lr(const Work& w, int NQ, int ntiles, cudaStream_t s)
{
    return sort_records<LrRec<T>>(w.lr_key, (const LrRec<T>*)w.lr_rec, (LrRec<T>*)w.lr_sorted, NQ, w.tile_cnt,
                                  w.tile_cur, ntiles, w.scan_tmp2, s);
}

template cudaError_t launch_sort_sr<float>(const Work&, int, int, cudaStream_t, bool);
template cudaError_t launch_sort_sr<double>(const Work&, int, int, cudaStream_t, bool);
template cudaError_t launch_sort_lr<float>(const Work&, int, int, cudaStream_t);
template cudaError_t launch_sort_lr<double>(const Work&, int, int, cudaStream_t);

}  // namespace bsw
