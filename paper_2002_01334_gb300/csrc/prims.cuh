// Device primitives: exclusive scan of uint32 and a stable LSD radix sort of (uint64 key,
// uint32 value) pairs, written for this library (no library kernels).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace lpb {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// block-wide exclusive scan of one value per thread; returns the block total in *total
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *smem, uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t w = lane < nw ? smem[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) smem[lane] = w;
  }
  __syncthreads();
  const uint32_t before = (warp > 0 ? smem[warp - 1] : 0u) + x - v;
  *total = smem[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

__global__ void k_scan_tiles(const uint32_t *in, uint32_t *out, uint32_t *tile_sums, int64_t n) {
  __shared__ uint32_t sm[32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  uint32_t v[SCAN_ITEMS];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0u;
    s += v[k];
  }
  uint32_t tot;
  uint32_t run = block_exclusive_scan(s, sm, &tot);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// single block: exclusive scan of the tile sums in place, total to *total
__global__ void k_scan_sums(uint32_t *sums, int64_t m, uint32_t *total) {
  __shared__ uint32_t sm[32];
  uint32_t carry = 0;
  for (int64_t c = 0; c < m; c += blockDim.x) {
    const int64_t i = c + threadIdx.x;
    const uint32_t v = i < m ? sums[i] : 0u;
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan(v, sm, &tot);
    if (i < m) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_add(uint32_t *out, const uint32_t *sums, int64_t n) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  const uint32_t add = sums[blockIdx.x];
  for (int k = threadIdx.x; k < SCAN_TILE; k += blockDim.x)
    if (base + k < n) out[base + k] += add;
}

// one block for short arrays: chunks of blockDim * SCAN_ITEMS with a running carry; the exclusive
// scan of in[0..n) into out (in place allowed), the total into *total (may be null)
__global__ void k_scan_one(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total) {
  __shared__ uint32_t sm[32];
  uint32_t carry = 0;
  const int64_t chunk = (int64_t)blockDim.x * SCAN_ITEMS;
  for (int64_t c0 = 0; c0 < n; c0 += chunk) {
    const int64_t base = c0 + (int64_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
      v[k] = (base + k < n) ? in[base + k] : 0u;
      s += v[k];
    }
    uint32_t tot;
    uint32_t run = carry + block_exclusive_scan(s, sm, &tot);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
      if (base + k < n) out[base + k] = run;
      run += v[k];
    }
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

// ---------------------------------------------------------------------------------------
// Stable LSD radix sort, 8-bit digits.  Tile = 256 threads x 8 rounds; within a tile the
// items are visited round-major (item = round*256 + thread), so ranks follow the input order.
// ---------------------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_ROUNDS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;

__global__ void k_radix_hist(const uint64_t *keys, int64_t n, int shift, uint32_t *hist, int nblocks) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const int64_t i = base + r * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_radix_scatter(const uint64_t *keys, const uint32_t *vals, uint64_t *okeys, uint32_t *ovals,
                                int64_t n, int shift, const uint32_t *offs, int nblocks) {
  __shared__ uint32_t cnt[RS_THREADS / 32][256];
  __shared__ uint32_t base_d[256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  base_d[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
  for (int w = 0; w < RS_THREADS / 32; ++w) cnt[w][threadIdx.x] = 0;
  __syncthreads();
  const int64_t tbase = (int64_t)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const int64_t i = tbase + r * RS_THREADS + threadIdx.x;
    const bool valid = i < n;
    uint64_t k = valid ? keys[i] : 0ull;
    uint32_t v = valid ? vals[i] : 0u;
    const uint32_t d = valid ? (uint32_t)((k >> shift) & 255u) : 256u;  // 256: padding, ranked last
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t lt = peers & ((1u << lane) - 1u);
    const uint32_t rank = __popc(lt);
    if (valid && lt == 0u) cnt[warp][d] = __popc(peers);
    __syncthreads();
    {  // exclusive prefix over warps for digit threadIdx.x, advancing the running base
      const int dd = threadIdx.x;
      uint32_t run = base_d[dd];
      for (int w = 0; w < RS_THREADS / 32; ++w) {
        const uint32_t t = cnt[w][dd];
        cnt[w][dd] = run;
        run += t;
      }
      base_d[dd] = run;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = cnt[warp][d] + rank;
      okeys[pos] = k;
      ovals[pos] = v;
    }
    __syncthreads();
    for (int w = 0; w < RS_THREADS / 32; ++w) cnt[w][threadIdx.x] = 0;
    __syncthreads();
  }
}

}  // namespace lpb
