// Stable LSD radix sort of 64-bit keys with device-resident key counts.
//
// Each pass handles one 8-bit window of the key. A pass whose window holds no
// bit that varies between keys (known from the OR and AND over all keys,
// accumulated by the kernel that produced them) is skipped on the device, so
// the host launches a fixed sequence and never waits for a count. Each pass is
// reduce-then-scan: per-tile digit counts, an exclusive scan over
// (digit, tile), then a stable scatter staged through shared memory so that
// each digit's keys leave the tile as one contiguous run. No block ever waits
// for another block.
#include <atomic>

#include "aiwc_internal.cuh"
#include "common.cuh"

namespace aiwc {

static std::atomic<unsigned long long> g_launches{0};
void count_launches(u64 n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
u64 launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

namespace {

// The sort's own tile: 256 threads x 8 keys (fewer registers per thread, so
// more blocks per SM than the 16-key tiles of the run kernels).
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kWarps = kSortThreads / 32;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;

__device__ __forceinline__ u64 eff_mask(const SortDesc& d) { return d.dmask ? (d.mask & *d.dmask) : d.mask; }

// Tiles holding keys: the device count decides, so that a sort sized for a
// capacity (the overflow list, the pattern words) works on what is there. The
// digit counts are laid out digit-major over these tiles.
__device__ __forceinline__ u32 live_tiles(const SortDesc& d) {
  const u64 n = umin64(*d.n, d.n_cap);
  const u64 t = (n + kSortTile - 1) / kSortTile;
  return (u32)(t < (u64)d.ntiles ? t : (u64)d.ntiles);
}

__device__ __forceinline__ bool pass_shift(const SortDesc& d, int pass, int* shift) {
  int sh = d.lo_bit + 8 * pass;
  *shift = sh;
  if (sh >= 64 || !gate_open(d.gate, d.gate_want)) return false;
  u64 varying = ((*d.key_or) ^ (*d.key_and)) & eff_mask(d);
  return ((varying >> sh) & 0xFFull) != 0;
}

__global__ void __launch_bounds__(kSortThreads) k_hist(SortDesc d, int pass) {
  int shift;
  if (!pass_shift(d, pass, &shift)) return;
  const u32 nt = live_tiles(d);
  if (blockIdx.x >= nt) return;
  __shared__ u32 h[kWarps][256];
  for (int i = threadIdx.x; i < kWarps * 256; i += kSortThreads) (&h[0][0])[i] = 0;
  __syncthreads();
  const u64 n = umin64(*d.n, d.n_cap);
  const u64* src = *d.cur ? d.b : d.a;
  const u64 base = (u64)blockIdx.x * kSortTile;
  const int w = threadIdx.x >> 5;
  const u64 m = eff_mask(d);
#pragma unroll 4
  for (int k = 0; k < kSortItems; ++k) {
    u64 i = base + (u64)k * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[w][((src[i] & m) >> shift) & 0xFF], 1u);
  }
  __syncthreads();
  u32 s = 0;
#pragma unroll
  for (int q = 0; q < kWarps; ++q) s += h[q][threadIdx.x];
  d.counts[(u64)threadIdx.x * nt + blockIdx.x] = s;
}

template <typename T>
__device__ __forceinline__ T block_excl_scan(T x, T* total, T* warp_tot) {
  // Exclusive prefix sum over the block; *total receives the block sum.
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[w] = inc;
  __syncthreads();
  if (w == 0) {
    T v = lane < nw ? warp_tot[lane] : T(0);
    T vi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, vi, o);
      if (lane >= o) vi += y;
    }
    if (lane < nw) warp_tot[lane] = vi - v;
    if (lane == 31) warp_tot[32] = vi;
  }
  __syncthreads();
  T r = warp_tot[w] + inc - x;
  *total = warp_tot[32];
  __syncthreads();
  return r;
}

// Exclusive scan of the counts of the live tiles, gated on the same pass
// predicate.
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(SortDesc d, int pass) {
  int shift;
  if (!pass_shift(d, pass, &shift)) return;
  const u64 len = 256ull * live_tiles(d);
  if ((u64)blockIdx.x * kScanBlock >= len) return;
  __shared__ u32 wt[33];
  u64 base = (u64)blockIdx.x * kScanBlock + (u64)threadIdx.x * kScanItems;
  u32 s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < len) s += d.counts[base + k];
  u32 tot;
  block_excl_scan<u32>(s, &tot, wt);
  if (threadIdx.x == 0) d.block_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(SortDesc d, int pass) {
  int shift;
  if (!pass_shift(d, pass, &shift)) return;
  const u32 nb = (u32)((256ull * live_tiles(d) + kScanBlock - 1) / kScanBlock);
  __shared__ u32 wt[33];
  u32 carry = 0;
  for (u32 c0 = 0; c0 < nb; c0 += kScanBlock) {
    u32 v[kScanItems];
    u32 s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      u32 i = c0 + threadIdx.x * kScanItems + k;
      v[k] = i < nb ? d.block_sums[i] : 0u;
      s += v[k];
    }
    u32 tot;
    u32 ex = block_excl_scan<u32>(s, &tot, wt) + carry;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      u32 i = c0 + threadIdx.x * kScanItems + k;
      if (i < nb) d.block_sums[i] = ex;
      ex += v[k];
    }
    carry += tot;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(SortDesc d, int pass) {
  int shift;
  if (!pass_shift(d, pass, &shift)) return;
  const u64 len = 256ull * live_tiles(d);
  if ((u64)blockIdx.x * kScanBlock >= len) return;
  __shared__ u32 wt[33];
  u64 base = (u64)blockIdx.x * kScanBlock + (u64)threadIdx.x * kScanItems;
  u32 v[kScanItems];
  u32 s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < len ? d.counts[base + k] : 0u;
    s += v[k];
  }
  u32 tot;
  u32 ex = block_excl_scan<u32>(s, &tot, wt) + d.block_sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < len) d.counts[base + k] = ex;
    ex += v[k];
  }
}

__global__ void __launch_bounds__(kSortThreads) k_scatter(SortDesc d, int pass) {
  int shift;
  if (!pass_shift(d, pass, &shift)) return;
  const u32 nt = live_tiles(d);
  if (blockIdx.x >= nt) return;
  __shared__ u32 wcnt[kWarps][256];
  __shared__ u32 dofs[256];
  __shared__ u32 gofs[256];
  __shared__ u32 wt[33];
  __shared__ u64 stage[kSortTile];
  for (int i = threadIdx.x; i < kWarps * 256; i += kSortThreads) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const u64 n = umin64(*d.n, d.n_cap);
  const u32 cur = *d.cur;
  const u64* src = cur ? d.b : d.a;
  u64* dst = cur ? d.a : d.b;
  const u64 base = (u64)blockIdx.x * kSortTile;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const u32 lt_mask = (1u << lane) - 1u;
  const u64 m = eff_mask(d);
  u64 key[kSortItems];
  u32 rank[kSortItems];
  // Warp w ranks positions base + w*512 + k*32 + lane in that order, which
  // keeps the scatter stable.
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    u64 i = base + (u64)w * (32 * kSortItems) + (u64)k * 32 + lane;
    bool valid = i < n;
    key[k] = valid ? src[i] : 0ull;
    u32 dig = valid ? (u32)(((key[k] & m) >> shift) & 0xFF) : 256u + lane;
    u32 peers = __match_any_sync(0xffffffffu, dig);
    u32 before = valid ? wcnt[w][dig] : 0u;
    rank[k] = before + __popc(peers & lt_mask);
    __syncwarp();
    if (valid && lane == 31 - __clz(peers)) wcnt[w][dig] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    const int dg = threadIdx.x;  // one thread per digit
    u32 tot = 0;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) {
      u32 c = wcnt[q][dg];
      wcnt[q][dg] = tot;
      tot += c;
    }
    u32 all;
    u32 ex = block_excl_scan<u32>(tot, &all, wt);
    dofs[dg] = ex;
    gofs[dg] = d.counts[(u64)dg * nt + blockIdx.x];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    u64 i = base + (u64)w * (32 * kSortItems) + (u64)k * 32 + lane;
    if (i < n) {
      u32 dig = (u32)(((key[k] & m) >> shift) & 0xFF);
      stage[dofs[dig] + wcnt[w][dig] + rank[k]] = key[k];
    }
  }
  __syncthreads();
  const u64 tile_n = n > base ? (n - base < (u64)kSortTile ? n - base : (u64)kSortTile) : 0ull;
  for (u32 j = threadIdx.x; j < tile_n; j += kSortThreads) {
    u64 kv = stage[j];
    u32 dig = (u32)(((kv & m) >> shift) & 0xFF);
    dst[(u64)gofs[dig] + (j - dofs[dig])] = kv;
  }
}

// A sort of a few tiles (at most kFewTiles): two launches per pass instead of
// six. The pass reads the buffer its parity gives -- the live buffer when the
// sort starts, flipped by every pass that runs (launched and with a varying
// window) -- so no pass writes `cur`; one launch at the end flips it by the
// parity of the passes that ran. The scatter computes each digit's global
// offset for its tile from all tiles' counts itself (256 x ntiles reads).
constexpr u32 kFewTiles = 64;

__device__ __forceinline__ bool few_pass(const SortDesc& d, int pass, u32 host_passes, int* shift, int* parity) {
  if (!gate_open(d.gate, d.gate_want)) return false;
  const u64 varying = ((*d.key_or) ^ (*d.key_and)) & eff_mask(d);
  int before = 0;
  for (int q = 0; q < pass; ++q) {
    const int sq = d.lo_bit + 8 * q;
    if (sq < 64 && ((host_passes >> q) & 1u) && ((varying >> sq) & 0xFFull)) ++before;
  }
  *shift = d.lo_bit + 8 * pass;
  *parity = before & 1;
  return *shift < 64 && ((varying >> *shift) & 0xFFull) != 0;
}

__global__ void __launch_bounds__(kSortThreads) k_hist_few(SortDesc d, int pass, u32 host_passes) {
  int shift, parity;
  if (!few_pass(d, pass, host_passes, &shift, &parity)) return;
  const u32 nt = live_tiles(d);
  if (blockIdx.x >= nt) return;
  __shared__ u32 h[kWarps][256];
  for (int i = threadIdx.x; i < kWarps * 256; i += kSortThreads) (&h[0][0])[i] = 0;
  __syncthreads();
  const u64 n = umin64(*d.n, d.n_cap);
  const u64* src = (*d.cur ^ (u32)parity) ? d.b : d.a;
  const u64 base = (u64)blockIdx.x * kSortTile;
  const int w = threadIdx.x >> 5;
  const u64 m = eff_mask(d);
#pragma unroll 4
  for (int k = 0; k < kSortItems; ++k) {
    const u64 i = base + (u64)k * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[w][((src[i] & m) >> shift) & 0xFF], 1u);
  }
  __syncthreads();
  u32 s = 0;
#pragma unroll
  for (int q = 0; q < kWarps; ++q) s += h[q][threadIdx.x];
  d.counts[(u64)threadIdx.x * nt + blockIdx.x] = s;
}

__global__ void __launch_bounds__(kSortThreads) k_scatter_few(SortDesc d, int pass, u32 host_passes) {
  int shift, parity;
  if (!few_pass(d, pass, host_passes, &shift, &parity)) return;
  const u32 nt = live_tiles(d);
  if (blockIdx.x >= nt) return;
  __shared__ u32 wcnt[kWarps][256];
  __shared__ u32 dofs[256];
  __shared__ u32 gofs[256];
  __shared__ u32 wt[33];
  __shared__ u64 stage[kSortTile];
  for (int i = threadIdx.x; i < kWarps * 256; i += kSortThreads) (&wcnt[0][0])[i] = 0;
  {
    // this tile's global offset for digit dg: the keys of smaller digits, then
    // those of digit dg in earlier tiles
    const int dg = threadIdx.x;
    u32 before = 0, total = 0;
    for (u32 t = 0; t < nt; ++t) {
      const u32 c = d.counts[(u64)dg * nt + t];
      if (t < blockIdx.x) before += c;
      total += c;
    }
    u32 all;
    gofs[dg] = block_excl_scan<u32>(total, &all, wt) + before;
  }
  __syncthreads();
  const u64 n = umin64(*d.n, d.n_cap);
  const u32 cur = *d.cur ^ (u32)parity;
  const u64* src = cur ? d.b : d.a;
  u64* dst = cur ? d.a : d.b;
  const u64 base = (u64)blockIdx.x * kSortTile;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const u32 lt_mask = (1u << lane) - 1u;
  const u64 m = eff_mask(d);
  u64 key[kSortItems];
  u32 rank[kSortItems];
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const u64 i = base + (u64)w * (32 * kSortItems) + (u64)k * 32 + lane;
    const bool valid = i < n;
    key[k] = valid ? src[i] : 0ull;
    const u32 dig = valid ? (u32)(((key[k] & m) >> shift) & 0xFF) : 256u + lane;
    const u32 peers = __match_any_sync(0xffffffffu, dig);
    const u32 before = valid ? wcnt[w][dig] : 0u;
    rank[k] = before + __popc(peers & lt_mask);
    __syncwarp();
    if (valid && lane == 31 - __clz(peers)) wcnt[w][dig] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    const int dg = threadIdx.x;
    u32 tot = 0;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) {
      const u32 c = wcnt[q][dg];
      wcnt[q][dg] = tot;
      tot += c;
    }
    u32 all;
    dofs[dg] = block_excl_scan<u32>(tot, &all, wt);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const u64 i = base + (u64)w * (32 * kSortItems) + (u64)k * 32 + lane;
    if (i < n) {
      const u32 dig = (u32)(((key[k] & m) >> shift) & 0xFF);
      stage[dofs[dig] + wcnt[w][dig] + rank[k]] = key[k];
    }
  }
  __syncthreads();
  const u64 tile_n = n > base ? (n - base < (u64)kSortTile ? n - base : (u64)kSortTile) : 0ull;
  for (u32 j = threadIdx.x; j < tile_n; j += kSortThreads) {
    const u64 kv = stage[j];
    const u32 dig = (u32)(((kv & m) >> shift) & 0xFF);
    dst[(u64)gofs[dig] + (j - dofs[dig])] = kv;
  }
}

// After the passes: the live buffer is the other one when an odd number ran.
__global__ void k_flip_few(SortDesc d, u32 host_passes) {
  if (!gate_open(d.gate, d.gate_want)) return;
  const u64 varying = ((*d.key_or) ^ (*d.key_and)) & eff_mask(d);
  int ran = 0;
  for (int q = 0; 8 * q + d.lo_bit < 64; ++q)
    if (((host_passes >> q) & 1u) && ((varying >> (d.lo_bit + 8 * q)) & 0xFFull)) ++ran;
  if (ran & 1) *d.cur ^= 1u;
}

// A sort that fits one tile (at most kSortTile keys): every pass in one block,
// ranking as k_scatter does (stable), the keys held in shared memory between
// passes and written back to the live buffer at the end (so `cur` does not
// change). One launch instead of six per pass.
__global__ void __launch_bounds__(kSortThreads) k_sort_tile(SortDesc d, u32 host_passes) {
  if (!gate_open(d.gate, d.gate_want)) return;
  __shared__ u32 wcnt[kWarps][256];
  __shared__ u32 dofs[256];
  __shared__ u32 wt[33];
  __shared__ u64 buf[2][kSortTile];
  const u64 n = umin64(umin64(*d.n, d.n_cap), (u64)kSortTile);
  u64* live = *d.cur ? d.b : d.a;
  for (u32 j = threadIdx.x; j < n; j += kSortThreads) buf[0][j] = live[j];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const u32 lt_mask = (1u << lane) - 1u;
  const u64 m = eff_mask(d);
  const u64 varying = ((*d.key_or) ^ (*d.key_and)) & m;
  int src = 0;
  bool ran = false;
  const int passes = (64 - d.lo_bit + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    const int shift = d.lo_bit + 8 * p;
    if (!((host_passes >> p) & 1u) || ((varying >> shift) & 0xFFull) == 0) continue;
    for (int i = threadIdx.x; i < kWarps * 256; i += kSortThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    u64 key[kSortItems];
    u32 rank[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
      const u32 i = (u32)w * (32 * kSortItems) + (u32)k * 32 + lane;
      const bool valid = i < n;
      key[k] = valid ? buf[src][i] : 0ull;
      const u32 dig = valid ? (u32)(((key[k] & m) >> shift) & 0xFF) : 256u + lane;
      const u32 peers = __match_any_sync(0xffffffffu, dig);
      const u32 before = valid ? wcnt[w][dig] : 0u;
      rank[k] = before + __popc(peers & lt_mask);
      __syncwarp();
      if (valid && lane == 31 - __clz(peers)) wcnt[w][dig] = before + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    {
      const int dg = threadIdx.x;  // one thread per digit
      u32 tot = 0;
#pragma unroll
      for (int q = 0; q < kWarps; ++q) {
        const u32 c = wcnt[q][dg];
        wcnt[q][dg] = tot;
        tot += c;
      }
      u32 all;
      dofs[dg] = block_excl_scan<u32>(tot, &all, wt);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
      const u32 i = (u32)w * (32 * kSortItems) + (u32)k * 32 + lane;
      if (i < n) {
        const u32 dig = (u32)(((key[k] & m) >> shift) & 0xFF);
        buf[src ^ 1][dofs[dig] + wcnt[w][dig] + rank[k]] = key[k];
      }
    }
    __syncthreads();
    src ^= 1;
    ran = true;
  }
  if (ran)
    for (u32 j = threadIdx.x; j < n; j += kSortThreads) live[j] = buf[src][j];
}

__global__ void k_flip(SortDesc d, int pass) {
  int shift;
  if (pass_shift(d, pass, &shift)) *d.cur ^= 1u;
}

}  // namespace

size_t sort_counts_words(u64 n_max) {
  u64 nt = (n_max + kSortTile - 1) / kSortTile;
  return (size_t)(256 * (nt ? nt : 1));
}

size_t sort_block_sums_words(u64 n_max) {
  u64 len = sort_counts_words(n_max);
  return (size_t)((len + kScanBlock - 1) / kScanBlock + 1);
}

u32 sort_tiles(u64 n) { return (u32)((n + kSortTile - 1) / kSortTile); }

void sort_keys(const SortDesc& d, cudaStream_t s, u32 host_passes) {
  if (d.ntiles == 0) return;
  const int npass = (64 - d.lo_bit + 7) / 8;
  if (d.ntiles == 1) {  // one tile: every pass in one launch
    if (host_passes & ((1u << npass) - 1u)) {
      k_sort_tile<<<1, kSortThreads, 0, s>>>(d, host_passes);
      count_launches(1);
    }
    return;
  }
  if (d.ntiles <= kFewTiles) {  // a few tiles: two launches per pass, one flip
    int launched = 0;
    for (int p = 0; p < npass; ++p) {
      if (!((host_passes >> p) & 1u)) continue;
      ++launched;
      k_hist_few<<<d.ntiles, kSortThreads, 0, s>>>(d, p, host_passes);
      k_scatter_few<<<d.ntiles, kSortThreads, 0, s>>>(d, p, host_passes);
    }
    if (launched) {
      k_flip_few<<<1, 1, 0, s>>>(d, host_passes);
      count_launches(2ull * launched + 1);
    }
    return;
  }
  const u64 len = 256ull * d.ntiles;
  const u32 nb = (u32)((len + kScanBlock - 1) / kScanBlock);
  const int passes = (64 - d.lo_bit + 7) / 8;
  int launched = 0;
  for (int p = 0; p < passes; ++p) {
    if (!((host_passes >> p) & 1u)) continue;
    ++launched;
    k_hist<<<d.ntiles, kSortThreads, 0, s>>>(d, p);
    k_scan_reduce<<<nb, kScanThreads, 0, s>>>(d, p);
    k_scan_top<<<1, kScanThreads, 0, s>>>(d, p);
    k_scan_down<<<nb, kScanThreads, 0, s>>>(d, p);
    k_scatter<<<d.ntiles, kSortThreads, 0, s>>>(d, p);
    k_flip<<<1, 1, 0, s>>>(d, p);
  }
  count_launches(6ull * launched);
}

}  // namespace aiwc
