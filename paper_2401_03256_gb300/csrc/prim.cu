// prim.cu - data-parallel primitives used by graph construction and batch updates:
// an exclusive scan of uint32 values and a stable LSD radix sort of 64-bit keys
// (one-block bitonic sort for small inputs).
#include <algorithm>
#include <utility>

#include "prdf_common.cuh"

namespace prdf {

// ------------------------------------------------------------------------ scan ---

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive scan of one tile per block (blocked arrangement); writes the tile total to
// sums[blockIdx.x] when sums != nullptr.
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const uint32_t *in, uint32_t *out, uint64_t n,
                                                             uint32_t *sums) {
  __shared__ uint32_t warp_tot[kScanThreads / 32];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t run = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    uint64_t idx = base + i;
    uint32_t x = idx < n ? in[idx] : 0u;
    v[i] = run;
    run += x;
  }
  // exclusive scan of per-thread totals across the block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0u;
    uint32_t ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = ti - t;  // exclusive
    if (lane == kScanThreads / 32 - 1 && sums) sums[blockIdx.x] = ti;
  }
  __syncthreads();
  const uint32_t offset = warp_tot[warp] + (incl - run);
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    uint64_t idx = base + i;
    if (idx < n) out[idx] = v[i] + offset;
  }
}

__global__ void k_scan_add(uint32_t *out, uint64_t n, const uint32_t *tile_off) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += tile_off[i / kScanTile];
}

size_t scan_tmp_words(uint64_t n) {
  if (n <= (uint64_t)kScanTile) return 0;
  uint64_t nb = (n + kScanTile - 1) / kScanTile;
  return nb + scan_tmp_words(nb);
}

void exclusive_scan_u32(const uint32_t *in, uint32_t *out, uint64_t n, uint32_t *tmp, cudaStream_t st) {
  if (n == 0) return;
  if (n <= (uint64_t)kScanTile) {
    k_scan_tiles<<<1, kScanThreads, 0, st>>>(in, out, n, nullptr); count_launch();
    return;
  }
  uint64_t nb = (n + kScanTile - 1) / kScanTile;
  k_scan_tiles<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, tmp); count_launch();
  exclusive_scan_u32(tmp, tmp, nb, tmp + nb, st);
  k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n, tmp); count_launch();
}

// ------------------------------------------------------------------ small sort ---

// Bitonic sort of up to kSmallSort keys by one block of 1024 threads, in place.
__global__ void __launch_bounds__(1024) k_block_sort(uint64_t *keys, uint32_t n) {
  __shared__ uint64_t s[kSmallSort];
  uint32_t p = 2;
  while (p < n) p <<= 1;
  for (uint32_t i = threadIdx.x; i < p; i += blockDim.x) s[i] = i < n ? keys[i] : kSentinel;
  __syncthreads();
  for (uint32_t k = 2; k <= p; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < p; i += blockDim.x) {
        uint32_t l = i ^ j;
        if (l > i) {
          uint64_t a = s[i], b = s[l];
          bool up = (i & k) == 0;
          if ((a > b) == up) {
            s[i] = b;
            s[l] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) keys[i] = s[i];
}

// ------------------------------------------------------------------ radix sort ---

// A block sorts a tile of ITEMS keys per thread: 16 (4096 keys) for large sorts, 4 (1024
// keys) below kSmallTileKeys, where 4096-key tiles leave most SMs idle and every pass is
// bound by one block's serial work (the sorts of a graph update are of this size).
constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixItemsSmall = 4, kRadixItemsLarge = 16;
constexpr uint64_t kSmallTileKeys = 2500000;

template <int ITEMS>
__global__ void __launch_bounds__(kRadixThreads) k_radix_hist(const uint64_t *keys, uint64_t n, int shift,
                                                              uint32_t *hist, uint32_t nblocks) {
  constexpr int kRadixTile = kRadixThreads * ITEMS;
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kRadixTile;
  for (int i = threadIdx.x; i < kRadixTile; i += kRadixThreads) {
    uint64_t idx = base + i;
    if (idx < n) atomicAdd(&cnt[(keys[idx] >> shift) & 0xFF], 1u);
  }
  __syncthreads();
  hist[(uint64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: warp w ranks its 32 * ITEMS consecutive keys round by round with
// __match_any_sync; per-warp digit counts are then offset across warps (warp order =
// index order) and by the block's global digit base.
template <int ITEMS>
__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(const uint64_t *keys, uint64_t *out, uint64_t n,
                                                                 int shift, const uint32_t *hist, uint32_t nblocks) {
  constexpr int kRadixItems = ITEMS, kRadixTile = kRadixThreads * ITEMS, kWarpKeys = kRadixTile / kRadixWarps;
  __shared__ uint32_t wcnt[kRadixWarps][256];
  __shared__ uint32_t gbase[256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int w = 0; w < kRadixWarps; w++) wcnt[w][threadIdx.x] = 0;
  gbase[threadIdx.x] = hist[(uint64_t)threadIdx.x * nblocks + blockIdx.x];
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kRadixTile + (uint64_t)warp * kWarpKeys;
  uint64_t k[kRadixItems];
  uint32_t local[kRadixItems];
#pragma unroll
  for (int r = 0; r < kRadixItems; r++) {
    uint64_t idx = base + (uint64_t)r * 32 + lane;
    bool valid = idx < n;
    k[r] = valid ? keys[idx] : 0ull;
    uint32_t d = valid ? (uint32_t)((k[r] >> shift) & 0xFF) : 0xFFFFu;
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t rank = __popc(peers & lanemask_lt());
    uint32_t b = valid ? wcnt[warp][d] : 0u;
    __syncwarp();
    if (valid && rank == 0) wcnt[warp][d] = b + __popc(peers);
    __syncwarp();
    local[r] = b + rank;
  }
  __syncthreads();
  {
    uint32_t run = 0;
    for (int w = 0; w < kRadixWarps; w++) {
      uint32_t c = wcnt[w][threadIdx.x];
      wcnt[w][threadIdx.x] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRadixItems; r++) {
    uint64_t idx = base + (uint64_t)r * 32 + lane;
    if (idx < n) {
      uint32_t d = (uint32_t)((k[r] >> shift) & 0xFF);
      out[gbase[d] + wcnt[warp][d] + local[r]] = k[r];
    }
  }
}

// Key-value variants: equal keys keep the order of their values (the values enter in
// ascending order), so a stable sort by key is also a sort by (key, value).
__global__ void __launch_bounds__(1024) k_block_sort_kv(uint64_t *keys, uint32_t *vals, uint32_t n) {
  __shared__ uint64_t sk[kSmallSort / 2];
  __shared__ uint32_t sv[kSmallSort / 2];
  uint32_t p = 2;
  while (p < n) p <<= 1;
  for (uint32_t i = threadIdx.x; i < p; i += blockDim.x) {
    sk[i] = i < n ? keys[i] : kSentinel;
    sv[i] = i < n ? vals[i] : 0xFFFFFFFFu;
  }
  __syncthreads();
  for (uint32_t k = 2; k <= p; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < p; i += blockDim.x) {
        uint32_t l = i ^ j;
        if (l > i) {
          uint64_t a = sk[i], b = sk[l];
          uint32_t va = sv[i], vb = sv[l];
          bool gt = a > b || (a == b && va > vb);
          bool up = (i & k) == 0;
          if (gt == up) {
            sk[i] = b;
            sk[l] = a;
            sv[i] = vb;
            sv[l] = va;
          }
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    keys[i] = sk[i];
    vals[i] = sv[i];
  }
}

template <int ITEMS>
__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter_kv(const uint64_t *keys, const uint32_t *vals,
                                                                    uint64_t *out, uint32_t *vout, uint64_t n,
                                                                    int shift, const uint32_t *hist,
                                                                    uint32_t nblocks) {
  constexpr int kRadixItems = ITEMS, kRadixTile = kRadixThreads * ITEMS, kWarpKeys = kRadixTile / kRadixWarps;
  __shared__ uint32_t wcnt[kRadixWarps][256];
  __shared__ uint32_t gbase[256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int w = 0; w < kRadixWarps; w++) wcnt[w][threadIdx.x] = 0;
  gbase[threadIdx.x] = hist[(uint64_t)threadIdx.x * nblocks + blockIdx.x];
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kRadixTile + (uint64_t)warp * kWarpKeys;
  uint64_t k[kRadixItems];
  uint32_t local[kRadixItems];
#pragma unroll
  for (int r = 0; r < kRadixItems; r++) {
    uint64_t idx = base + (uint64_t)r * 32 + lane;
    bool valid = idx < n;
    k[r] = valid ? keys[idx] : 0ull;
    uint32_t d = valid ? (uint32_t)((k[r] >> shift) & 0xFF) : 0xFFFFu;
    uint32_t peers = __match_any_sync(0xffffffffu, d);
    uint32_t rank = __popc(peers & lanemask_lt());
    uint32_t b = valid ? wcnt[warp][d] : 0u;
    __syncwarp();
    if (valid && rank == 0) wcnt[warp][d] = b + __popc(peers);
    __syncwarp();
    local[r] = b + rank;
  }
  __syncthreads();
  {
    uint32_t run = 0;
    for (int w = 0; w < kRadixWarps; w++) {
      uint32_t c = wcnt[w][threadIdx.x];
      wcnt[w][threadIdx.x] = run;
      run += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRadixItems; r++) {
    uint64_t idx = base + (uint64_t)r * 32 + lane;
    if (idx < n) {
      uint32_t d = (uint32_t)((k[r] >> shift) & 0xFF);
      uint32_t at = gbase[d] + wcnt[warp][d] + local[r];
      out[at] = k[r];
      vout[at] = vals[idx];
    }
  }
}

template <int ITEMS>
void radix_kv(uint64_t **keys, uint32_t **vals, uint64_t *alt_k, uint32_t *alt_v, uint64_t n, int bits,
              uint32_t *hist, uint32_t *scan_tmp, cudaStream_t st) {
  constexpr int kRadixTile = kRadixThreads * ITEMS;
  const uint32_t nblocks = (uint32_t)((n + kRadixTile - 1) / kRadixTile);
  uint64_t *sk = *keys, *dk = alt_k;
  uint32_t *sv = *vals, *dv = alt_v;
  for (int shift = 0; shift < bits; shift += 8) {
    k_radix_hist<ITEMS><<<nblocks, kRadixThreads, 0, st>>>(sk, n, shift, hist, nblocks);
    count_launch();
    exclusive_scan_u32(hist, hist, (uint64_t)256 * nblocks, scan_tmp, st);
    k_radix_scatter_kv<ITEMS><<<nblocks, kRadixThreads, 0, st>>>(sk, sv, dk, dv, n, shift, hist, nblocks);
    count_launch();
    std::swap(sk, dk);
    std::swap(sv, dv);
  }
  *keys = sk;
  *vals = sv;
}

void sort_u64_kv(uint64_t **keys, uint32_t **vals, uint64_t *alt_k, uint32_t *alt_v, uint64_t n, int bits,
                 uint32_t *hist, uint32_t *scan_tmp, cudaStream_t st) {
  if (n < 2) return;
  if (n <= kSmallSort / 2) {
    k_block_sort_kv<<<1, 1024, 0, st>>>(*keys, *vals, (uint32_t)n);
    count_launch();
    return;
  }
  if (n < kSmallTileKeys) radix_kv<kRadixItemsSmall>(keys, vals, alt_k, alt_v, n, bits, hist, scan_tmp, st);
  else radix_kv<kRadixItemsLarge>(keys, vals, alt_k, alt_v, n, bits, hist, scan_tmp, st);
}

size_t radix_hist_words(uint64_t n) {
  // the most tiles n keys can need: small tiles below kSmallTileKeys, large ones above
  const uint64_t small = std::min<uint64_t>(n, kSmallTileKeys);
  const uint64_t tiles = std::max<uint64_t>((small + kRadixThreads * kRadixItemsSmall - 1) / (kRadixThreads * kRadixItemsSmall),
                                            (n + kRadixThreads * kRadixItemsLarge - 1) / (kRadixThreads * kRadixItemsLarge));
  return 256 * tiles;
}

int bits_for(uint32_t n) {
  int b = 1;
  while (b < 32 && (1ull << b) < (uint64_t)n) b++;
  return b;
}

template <int ITEMS>
uint64_t *radix_keys(uint64_t *keys, uint64_t *alt, uint64_t n, int bits, uint32_t *hist, uint32_t *scan_tmp,
                     cudaStream_t st) {
  constexpr int kRadixTile = kRadixThreads * ITEMS;
  const uint32_t nblocks = (uint32_t)((n + kRadixTile - 1) / kRadixTile);
  uint64_t *src = keys, *dst = alt;
  for (int shift = 0; shift < bits; shift += 8) {
    k_radix_hist<ITEMS><<<nblocks, kRadixThreads, 0, st>>>(src, n, shift, hist, nblocks); count_launch();
    exclusive_scan_u32(hist, hist, (uint64_t)256 * nblocks, scan_tmp, st);
    k_radix_scatter<ITEMS><<<nblocks, kRadixThreads, 0, st>>>(src, dst, n, shift, hist, nblocks); count_launch();
    uint64_t *t = src;
    src = dst;
    dst = t;
  }
  return src;
}

uint64_t *sort_u64(uint64_t *keys, uint64_t *alt, uint64_t n, int bits, uint32_t *hist, uint32_t *scan_tmp,
                   cudaStream_t st) {
  if (n < 2) return keys;
  if (n <= kSmallSort) {
    k_block_sort<<<1, 1024, 0, st>>>(keys, (uint32_t)n); count_launch();
    return keys;
  }
  return n < kSmallTileKeys ? radix_keys<kRadixItemsSmall>(keys, alt, n, bits, hist, scan_tmp, st)
                            : radix_keys<kRadixItemsLarge>(keys, alt, n, bits, hist, scan_tmp, st);
}

}  // namespace prdf
