// Stable LSD radix sort of 64-bit keys with device-resident key counts.
//
// Each pass handles one 8-bit window of the key. Only bits that vary between
// keys need ordering (known from the OR and AND over all keys, accumulated by
// the kernel that produced them), and the device decides which passes run, so
// the host launches a fixed sequence and never waits for a count. Three forms:
// one tile (every pass in one block, in shared memory); fewer than 2^30 keys
// (one-sweep passes: one launch each, the tiles' digit offsets found by a
// bounded look-back over earlier tiles); more (reduce-then-scan passes:
// per-tile digit counts, an exclusive scan over (digit, tile), a stable
// scatter staged through shared memory). The first two place each window at
// the lowest bit still to be ordered; the last uses the key's bytes and skips
// bytes without a varying bit. In every form each digit's keys leave a tile
// as one contiguous run.
#include <algorithm>
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

__device__ __forceinline__ u64 eff_mask(const SortDesc& d) {
  u64 m = d.dmask ? (d.mask & *d.dmask) : d.mask;
  // work-item ids in push order: a stable sort by site keeps (work-item, program order)
  if (d.unsorted) m &= *d.unsorted ? ~1ull : 0xFFFFFFFF00000000ull;
  return m;
}

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

// One-sweep form (sorts of more than one tile and fewer than 2^30 keys): one
// launch counts the digits of every window at once (k_hist_all), then one
// launch per window ranks each tile, publishes the tile's digit counts and
// finds the counts of the tiles before it by decoupled look-back (each tile
// waits only for tiles that took their tickets earlier, so every wait ends),
// and scatters. Window p reads the buffer its parity gives (the live buffer
// for p = 0), so no pass writes `cur`; one launch at the end flips it when
// the number of windows is odd.
//
// Scratch: block_sums holds the digit totals of the eight windows (8 x 256)
// and eight tile tickets, zeroed before the sort; counts holds two regions of
// look-back words (ntiles x 256 each), the pass of parity q using region q & 1
// and clearing its tile's words of the other region for the next pass. A
// look-back word is state << 30 | count: 0 not yet published, kLbAgg the
// tile's own count, kLbInc the count of this and every earlier tile.
constexpr u32 kLbAgg = 1u << 30, kLbInc = 2u << 30, kLbCount = (1u << 30) - 1u;
constexpr u32 kSpinLimit = 1u << 20;  // polls of one word (with a short sleep each) before giving up
constexpr u32 kTotWords = 8 * 256;    // digit totals; the eight tickets follow

// Look-back words are read and written at GPU scope (not from a stale L1 line).
__device__ __forceinline__ u32 ld_gpu(const u32* p) {
  u32 v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_gpu(u32* p, u32 v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bits a sort must order: those that vary between keys, inside the mask and
// inside the byte windows the host left on.
__device__ __forceinline__ u64 sort_bits(const SortDesc& d, u32 host_passes) {
  u64 allowed = 0;
  for (int q = 0; q < 8 && d.lo_bit + 8 * q < 64; ++q)
    if ((host_passes >> q) & 1u) allowed |= 0xFFull << (d.lo_bit + 8 * q);
  return ((*d.key_or) ^ (*d.key_and)) & eff_mask(d) & allowed;
}

// Start bit of the p-th 8-bit window, or -1 past the last. Each window starts
// at the lowest bit still to be ordered, so the windows are the fewest that
// cover every such bit (never more than the bytes holding one), and ordering
// them from low to high is a stable LSD sort on the bits that matter.
__device__ __forceinline__ int window_shift(u64 bits, int p) {
  for (int k = 0;; ++k) {
    if (!bits) return -1;
    const int b = __ffsll((long long)bits) - 1;
    if (k == p) return b;
    bits = b >= 56 ? 0ull : bits & (~0ull << (b + 8));
  }
}

// Digit totals of every pass that will run, and the first pass's look-back region cleared.
__global__ void __launch_bounds__(kSortThreads) k_hist_all(SortDesc d, u32 host_passes) {
  if (!gate_open(d.gate, d.gate_want)) return;
  __shared__ u32 h[4][8][256];  // one copy per pair of warps
  for (int i = threadIdx.x; i < 4 * 8 * 256; i += kSortThreads) (&h[0][0][0])[i] = 0u;
  __syncthreads();
  const u64 n = umin64(*d.n, d.n_cap);
  const u64* src = *d.cur ? d.b : d.a;
  const u64 m = eff_mask(d);
  const u64 bits = sort_bits(d, host_passes);
  int sh[8];
  u32 act = 0;  // windows that exist
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    sh[p] = window_shift(bits, p);
    if (sh[p] >= 0) act |= 1u << p;
  }
  u32 (*hh)[256] = h[(threadIdx.x >> 6) & 3];
  const u64 stride = (u64)gridDim.x * kSortThreads;
  // eight keys per thread in flight
  for (u64 i0 = (u64)blockIdx.x * kSortThreads + threadIdx.x; i0 < n; i0 += 8 * stride) {
    u64 k[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) k[q] = i0 + q * stride < n ? src[i0 + q * stride] & m : 0ull;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (i0 + q * stride >= n) break;
#pragma unroll
      for (int p = 0; p < 8; ++p)
        if ((act >> p) & 1u) atomicAdd(&hh[p][(u32)(k[q] >> sh[p]) & 0xFFu], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 8 * 256; i += kSortThreads) {
    const u32 c = (&h[0][0][0])[i] + (&h[1][0][0])[i] + (&h[2][0][0])[i] + (&h[3][0][0])[i];
    if (c) atomicAdd(&d.block_sums[i], c);
  }
  const u64 words = 256ull * live_tiles(d);
  for (u64 i = (u64)blockIdx.x * kSortThreads + threadIdx.x; i < words; i += stride) d.counts[i] = 0u;
}

__global__ void __launch_bounds__(kSortThreads) k_onesweep(SortDesc d, int pass, u32 host_passes) {
  if (!gate_open(d.gate, d.gate_want)) return;
  const int shift = window_shift(sort_bits(d, host_passes), pass);
  if (shift < 0) return;
  const int parity = pass & 1;  // windows 0 .. pass-1 ran before this one
  __shared__ u32 wcnt[kWarps][256];
  __shared__ u32 dofs[256];
  __shared__ u32 gofs[256];
  __shared__ u32 wt[33];
  __shared__ u32 s_tile;
  __shared__ u64 stage[kSortTile];
  const u32 nt = live_tiles(d);
  if (threadIdx.x == 0) s_tile = atomicAdd(&d.block_sums[kTotWords + pass], 1u);
  for (int i = threadIdx.x; i < kWarps * 256; i += kSortThreads) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const u32 t = s_tile;
  if (t >= nt) return;
  const u64 n = umin64(*d.n, d.n_cap);
  const u32 cur = *d.cur ^ (u32)parity;
  const u64* src = cur ? d.b : d.a;
  u64* dst = cur ? d.a : d.b;
  const u64 base = (u64)t * kSortTile;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const u32 lt_mask = (1u << lane) - 1u;
  const u64 m = eff_mask(d);
  u64 key[kSortItems];
  u32 rank[kSortItems];
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {  // every load in flight before the ranking
    const u64 i = base + (u64)w * (32 * kSortItems) + (u64)k * 32 + lane;
    key[k] = i < n ? src[i] : 0ull;
  }
  // warp w ranks positions base + w*256 + k*32 + lane in that order (stable)
#pragma unroll
  for (int k = 0; k < kSortItems; ++k) {
    const u64 i = base + (u64)w * (32 * kSortItems) + (u64)k * 32 + lane;
    const bool valid = i < n;
    const u32 dig = valid ? (u32)(((key[k] & m) >> shift) & 0xFF) : 256u + lane;
    const u32 peers = __match_any_sync(0xffffffffu, dig);
    const u32 before = valid ? wcnt[w][dig] : 0u;
    rank[k] = before + __popc(peers & lt_mask);
    __syncwarp();
    if (valid && lane == 31 - __clz(peers)) wcnt[w][dig] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
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
  const u32 dstart = block_excl_scan<u32>(d.block_sums[pass * 256 + dg], &all, wt);
  u32* look = d.counts + (size_t)(parity & 1) * 256u * d.ntiles;
  u32* mine = look + (size_t)t * 256 + dg;
  u32 excl = 0;
  if (t == 0) {
    st_gpu(mine, kLbInc | tot);
  } else {
    st_gpu(mine, kLbAgg | tot);
    for (u32 j = t - 1;; --j) {
      const u32* pw = look + (size_t)j * 256 + dg;
      u32 v = ld_gpu(pw);
      for (u32 spin = 0; !(v >> 30); ++spin) {
        if (spin == kSpinLimit) {
          // every earlier tile has its ticket and runs, so this does not
          // happen; should it, the counts so far keep every position in range
          if (d.err) atomicOr(d.err, kErrSort);
          v = kLbInc;
          break;
        }
        __nanosleep(64);
        v = ld_gpu(pw);
      }
      excl += v & kLbCount;
      if ((v & kLbInc) || j == 0) break;
    }
    st_gpu(mine, kLbInc | (excl + tot));
  }
  gofs[dg] = dstart + excl;
  // the next pass's region: this tile's words start unpublished
  d.counts[(size_t)((parity + 1) & 1) * 256u * d.ntiles + (size_t)t * 256 + dg] = 0u;
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
  const u64 tile_n = n > base ? umin64(n - base, (u64)kSortTile) : 0ull;
  for (u32 j = threadIdx.x; j < tile_n; j += kSortThreads) {
    const u64 kv = stage[j];
    const u32 dig = (u32)(((kv & m) >> shift) & 0xFF);
    dst[(u64)gofs[dig] + (j - dofs[dig])] = kv;
  }
}

// After the passes: the live buffer is the other one when an odd number ran.
__global__ void k_flip_windows(SortDesc d, u32 host_passes) {
  if (!gate_open(d.gate, d.gate_want)) return;
  const u64 bits = sort_bits(d, host_passes);
  int ran = 0;
  while (window_shift(bits, ran) >= 0) ++ran;
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
  const u64 bits = sort_bits(d, host_passes);
  int src = 0;
  bool ran = false;
  for (int p = 0; p < 8; ++p) {
    const int shift = window_shift(bits, p);
    if (shift < 0) break;
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
  return (size_t)(512 * (nt ? nt : 1));  // two look-back regions of the one-sweep form
}

size_t sort_block_sums_words(u64 n_max) {
  u64 len = 256 * ((n_max + kSortTile - 1) / kSortTile + 1);
  return std::max<size_t>((size_t)((len + kScanBlock - 1) / kScanBlock + 1), kTotWords + 8);
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
  if (d.n_cap < (1ull << 30)) {  // one sweep per window, one histogram launch, one flip
    // at most one window per byte the host left on; the device finds how many there are
    const int windows = __builtin_popcount(host_passes & ((1u << npass) - 1u));
    if (!windows) return;
    cudaMemsetAsync(d.block_sums, 0, (kTotWords + 8) * sizeof(u32), s);
    k_hist_all<<<std::min<u32>(d.ntiles, 152u * 4), kSortThreads, 0, s>>>(d, host_passes);
    for (int p = 0; p < windows; ++p) k_onesweep<<<d.ntiles, kSortThreads, 0, s>>>(d, p, host_passes);
    k_flip_windows<<<1, 1, 0, s>>>(d, host_passes);
    count_launches(windows + 2ull);
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
