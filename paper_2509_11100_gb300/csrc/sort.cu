// sort.cu -- integer kernels of the per-step cell sort: exclusive scan,
// key histogram, stable LSD radix sort (load path and long-move fallback),
// and the neighbour-move counting sort tables.
//
// The per-step sort exploits that a particle moves at most one cell per
// step (c dt <= min(dx, dy)): the particles of old cell c split into nine
// direction groups; new cell k receives the groups of its nine neighbours,
// ordered by source-cell index, so that equal keys keep their previous
// relative order (a stable counting sort by new cell).
#include "launch.cuh"

namespace relsim {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;   // 4096
constexpr int kMaxScanBlocks = 16384;

// exclusive block scan of one int per thread; *total = block sum.
__device__ int block_scan_excl(int v, int* smem, int* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = lane < nw ? smem[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        smem[lane] = s;
    }
    __syncthreads();
    int prefix = wid > 0 ? smem[wid - 1] : 0;
    *total = smem[nw - 1];
    __syncthreads();
    return prefix + x - v;
}

__global__ void k_scan_reduce(const int32_t* __restrict__ in, int64_t n, int32_t* partial)
{
    __shared__ int smem[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int s = 0;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r)
        if (base + r < n) s += in[base + r];
    int tot;
    block_scan_excl(s, smem, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void k_scan_partials(int32_t* partial, int nb, int32_t* total)
{
    __shared__ int smem[32];
    const int per = (nb + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per;
    int s = 0;
    for (int r = 0; r < per; ++r)
        if (b0 + r < nb) s += partial[b0 + r];
    int tot;
    int run = block_scan_excl(s, smem, &tot);
    for (int r = 0; r < per; ++r)
        if (b0 + r < nb) {
            int v = partial[b0 + r];
            partial[b0 + r] = run;
            run += v;
        }
    if (threadIdx.x == 0 && total) *total = tot;
}

__global__ void k_scan_apply(const int32_t* in, int32_t* out, int64_t n,
                             const int32_t* __restrict__ partial)
{
    __shared__ int smem[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int r = 0; r < kScanItems; ++r) {
        v[r] = base + r < n ? in[base + r] : 0;
        s += v[r];
    }
    int tot;
    int run = block_scan_excl(s, smem, &tot) + partial[blockIdx.x];
#pragma unroll
    for (int r = 0; r < kScanItems; ++r)
        if (base + r < n) {
            out[base + r] = run;
            run += v[r];
        }
}

// ---------------------------------------------------------------------------
// stable LSD radix sort, 4-bit digits

constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 16;
constexpr int kRadixTile = kRadixThreads * kRadixItems;   // 4096
constexpr int kRadix = 16;

__global__ void k_radix_up(const int32_t* __restrict__ keys, int64_t n, int shift, int nb,
                           int32_t* hist)
{
    __shared__ int cnt[kRadix];
    if (threadIdx.x < kRadix) cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int r = threadIdx.x; r < kRadixTile; r += blockDim.x) {
        int64_t i = base + r;
        if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & (kRadix - 1)], 1);
    }
    __syncthreads();
    if (threadIdx.x < kRadix) hist[(int64_t)threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(kRadixThreads)
k_radix_down(const int32_t* __restrict__ kin, const int32_t* __restrict__ vin, int32_t* kout,
             int32_t* vout, int64_t n, int shift, int nb, const int32_t* __restrict__ hist)
{
    __shared__ int cnt[kRadix * kRadixThreads];   // cnt[d*256 + t]
    __shared__ int base[kRadix];
    __shared__ int smem[32];
    const int t = threadIdx.x;
    int64_t i0 = (int64_t)blockIdx.x * kRadixTile + (int64_t)t * kRadixItems;
    int k[kRadixItems], v[kRadixItems];
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        bool ok = i0 + r < n;
        k[r] = ok ? kin[i0 + r] : 0;
        v[r] = ok ? vin[i0 + r] : 0;
    }
#pragma unroll
    for (int d = 0; d < kRadix; ++d) cnt[d * kRadixThreads + t] = 0;
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r)
        if (i0 + r < n) cnt[((k[r] >> shift) & (kRadix - 1)) * kRadixThreads + t]++;
    __syncthreads();
    // exclusive scan of the 4096 counters in digit-major order
    int loc[kRadixItems];
    int s = 0;
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        loc[r] = cnt[t * kRadixItems + r];
        s += loc[r];
    }
    int tot;
    int run = block_scan_excl(s, smem, &tot);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        cnt[t * kRadixItems + r] = run;
        run += loc[r];
    }
    __syncthreads();
    if (t < kRadix) base[t] = hist[(int64_t)t * nb + blockIdx.x] - cnt[t * kRadixThreads];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        if (i0 + r < n) {
            int d = (k[r] >> shift) & (kRadix - 1);
            int pos = base[d] + cnt[d * kRadixThreads + t]++;
            kout[pos] = k[r];
            vout[pos] = v[r];
        }
    }
}

__global__ void k_hist(const int32_t* __restrict__ keys, int64_t n, int32_t* counts)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i - threadIdx.x < n; i += stride) {
        bool ok = i < n;
        int key = ok ? keys[i] : -1;
        unsigned act = __ballot_sync(0xffffffffu, ok);
        if (!ok) continue;
        unsigned peers = __match_any_sync(act, key);
        int leader = __ffs(peers) - 1;
        if ((threadIdx.x & 31) == leader) atomicAdd(&counts[key], __popc(peers));
    }
}

__global__ void k_iota(int32_t* a, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride) a[i] = (int32_t)i;
}

// direction d = (sy+1)*3 + (sx+1) of a move by (sx, sy) cells
__device__ __forceinline__ int src_cell(int i, int j, int d, const GridP& g)
{
    int sx = d % 3 - 1, sy = d / 3 - 1;
    return wrap1(j - sy, g.ny) * g.nx + wrap1(i - sx, g.nx);
}

__global__ void k_move_counts(const int32_t* __restrict__ n9, int32_t* count_new, GridP g)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.ncell) return;
    int i = k % g.nx, j = k / g.nx;
    int c = 0;
#pragma unroll
    for (int d = 0; d < kNDir; ++d) c += n9[(int64_t)src_cell(i, j, d, g) * kNDir + d];
    count_new[k] = c;
}

// zero n4 16-byte words, then ntail 4-byte words after them
__global__ void k_zero(uint4* __restrict__ p4, int64_t n4, uint32_t* __restrict__ tail, int ntail)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride)
        p4[i] = make_uint4(0u, 0u, 0u, 0u);
    if (blockIdx.x == 0 && (int)threadIdx.x < ntail) tail[threadIdx.x] = 0u;
}

}  // namespace

cudaError_t zero_fill(void* p, size_t bytes, cudaStream_t st)
{
    if (bytes == 0) return cudaSuccess;
    if (((uintptr_t)p & 15) != 0 || (bytes & 3) != 0) return cudaErrorInvalidValue;
    const int64_t n4 = (int64_t)(bytes / 16);
    const int ntail = (int)((bytes % 16) / 4);
    int64_t blocks = (n4 + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    count_launches(1);
    k_zero<<<(unsigned)blocks, 256, 0, st>>>((uint4*)p, n4, (uint32_t*)((char*)p + n4 * 16), ntail);
    return cudaGetLastError();
}

size_t scan_tmp_ints(int64_t n)
{
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    return (size_t)(nb + 1);
}

cudaError_t scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* total,
                               int32_t* tmp, cudaStream_t st)
{
    if (n <= 0) {
        if (total) return cudaMemsetAsync(total, 0, sizeof(int32_t), st);
        return cudaSuccess;
    }
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb > kMaxScanBlocks) return cudaErrorInvalidValue;
    count_launches(1);
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, tmp);
    count_launches(1);
    k_scan_partials<<<1, kScanThreads, 0, st>>>(tmp, (int)nb, total);
    count_launches(1);
    k_scan_apply<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, tmp);
    return cudaGetLastError();
}

size_t radix_tmp_ints(int64_t n)
{
    int64_t nb = (n + kRadixTile - 1) / kRadixTile;
    return (size_t)(kRadix * nb) + scan_tmp_ints(kRadix * nb);
}

cudaError_t radix_sort_pairs(int32_t* k0, int32_t* v0, int32_t* k1, int32_t* v1, int64_t n,
                             int key_bits, int32_t* tmp, bool* result_in_1, cudaStream_t st)
{
    *result_in_1 = false;
    if (n <= 1) return cudaSuccess;
    int64_t nb = (n + kRadixTile - 1) / kRadixTile;
    int32_t* hist = tmp;
    int32_t* stmp = tmp + kRadix * nb;
    int32_t *ki = k0, *vi = v0, *ko = k1, *vo = v1;
    for (int shift = 0; shift < key_bits; shift += 4) {
        count_launches(1);
        k_radix_up<<<(unsigned)nb, kRadixThreads, 0, st>>>(ki, n, shift, (int)nb, hist);
        cudaError_t e = scan_exclusive_i32(hist, hist, kRadix * nb, nullptr, stmp, st);
        if (e != cudaSuccess) return e;
        count_launches(1);
        k_radix_down<<<(unsigned)nb, kRadixThreads, 0, st>>>(ki, vi, ko, vo, n, shift, (int)nb, hist);
        int32_t* t;
        t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
        *result_in_1 = !*result_in_1;
    }
    return cudaGetLastError();
}

cudaError_t histogram_keys(const int32_t* keys, int64_t n, int32_t* counts, int nkeys,
                           cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)nkeys, st);
    if (e != cudaSuccess || n <= 0) return e;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    count_launches(1);
    k_hist<<<(unsigned)blocks, 256, 0, st>>>(keys, n, counts);
    return cudaGetLastError();
}

cudaError_t move_counts(const int32_t* n9, int32_t* count_new, GridP g, cudaStream_t st)
{
    count_launches(1);
    k_move_counts<<<(g.ncell + 255) / 256, 256, 0, st>>>(n9, count_new, g);
    return cudaGetLastError();
}

cudaError_t iota_i32(int32_t* a, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    count_launches(1);
    k_iota<<<(unsigned)blocks, 256, 0, st>>>(a, n);
    return cudaGetLastError();
}

}  // namespace relsim
