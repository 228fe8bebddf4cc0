// scan.cu -- device-wide exclusive prefix sum of uint32 values (reduce, scan the block
// totals, scan again with the block offsets).  Used for the radix-sort digit offsets and
// for the cell table (Sec. 4.1: each cell's first particle is the count of particles in
// the cells before it in Morton order).
#include "mps_internal.cuh"

namespace mps {

namespace {
constexpr int kBT = 256;
constexpr int kItems = 8;
constexpr int kTile = kBT * kItems;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    const int lane = threadIdx.x & 31;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive block scan of one value per thread; returns exclusive prefix, *total = sum
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
    __shared__ uint32_t s_w[kBT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = warp_incl_scan(v);
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t x = (lane < kBT / 32) ? s_w[lane] : 0u;
        uint32_t xi = warp_incl_scan(x);
        if (lane < kBT / 32) s_w[lane] = xi - x;
        if (lane == kBT / 32 - 1) *total = xi;
    }
    __syncthreads();
    uint32_t r = s_w[w] + inc - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kBT) k_scan_reduce(const uint32_t* in, int64_t m, uint32_t* sums) {
    const int64_t base = (int64_t)blockIdx.x * kTile;
    uint32_t s = 0;
    for (int k = 0; k < kItems; k++) {
        int64_t i = base + (int64_t)k * kBT + threadIdx.x;
        if (i < m) s += in[i];
    }
    __shared__ uint32_t tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// single block: exclusive scan of nb block sums in place, in chunks of kBT with a carry
__global__ void __launch_bounds__(kBT) k_scan_top(uint32_t* sums, int nb, uint32_t* total_out) {
    __shared__ uint32_t tot;
    uint32_t carry = 0;
    for (int b0 = 0; b0 < nb; b0 += kBT) {
        int b = b0 + threadIdx.x;
        uint32_t v = (b < nb) ? sums[b] : 0u;
        uint32_t ex = block_excl_scan(v, &tot);
        if (b < nb) sums[b] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total_out) *total_out = carry;
}

// each thread owns kItems consecutive values of the tile
__global__ void __launch_bounds__(kBT) k_scan_down(const uint32_t* in, uint32_t* out, int64_t m,
                                                   const uint32_t* sums) {
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kItems;
    uint32_t v[kItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kItems; k++) {
        v[k] = (base + k < m) ? in[base + k] : 0u;
        s += v[k];
    }
    __shared__ uint32_t tot;
    uint32_t ex = block_excl_scan(s, &tot) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kItems; k++) {
        if (base + k < m) out[base + k] = ex;
        ex += v[k];
    }
}
}  // namespace

int64_t scan_scratch_words(int64_t m) { return (m + kTile - 1) / kTile + 1; }

int scan_exclusive(const uint32_t* in, uint32_t* out, int64_t m, bool write_total,
                   uint32_t* scratch, cudaStream_t s) {
    int nb = (int)((m + kTile - 1) / kTile);
    if (nb == 0) {
        if (write_total) cudaMemsetAsync(out, 0, sizeof(uint32_t), s);
        return 0;
    }
    k_scan_reduce<<<nb, kBT, 0, s>>>(in, m, scratch);
    k_scan_top<<<1, kBT, 0, s>>>(scratch, nb, write_total ? out + m : nullptr);
    k_scan_down<<<nb, kBT, 0, s>>>(in, out, m, scratch);
    return 3;
}

}  // namespace mps
