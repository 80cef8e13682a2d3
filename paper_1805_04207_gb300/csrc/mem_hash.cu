// Memory path without a sort ("hash" plan).
//
// Every group of skip level n <= 10 (key >> n, Sec. III) lies inside one
// superblock of 2^11 addresses (key >> 11). So instead of sorting 64-bit
// words we:
//   1. count the events of each superblock in an open-addressing table that
//      stays in L2 (done during ingest, see mem.cu),
//   2. scan the counts into segment offsets and scatter each event's low 12
//      bits (11 address bits and the store bit) into its superblock's
//      segment as a u16,
//   3. build each segment's dense 4096-bin histogram in shared memory and sum
//      it hierarchically: level n groups are aligned runs of 2^n addresses.
// Superblocks and segments are processed in any order: every output is a sum
// of exact integers, so the result does not depend on scheduling.
#include "aiwc_internal.cuh"
#include "common.cuh"

namespace aiwc {
namespace {

constexpr int kScanT = 1024;
constexpr int kScanI = 4;
constexpr int kScanB = kScanT * kScanI;

__global__ void __launch_bounds__(kScanT) k_sbt_reduce(const u32* cnt, u64 len, u32* bsum) {
  __shared__ u32 red[32];
  const u64 base = (u64)blockIdx.x * kScanB + (u64)threadIdx.x * kScanI;
  u32 s = 0;
#pragma unroll
  for (int k = 0; k < kScanI; ++k)
    if (base + k < len) s += cnt[base + k];
  s = block_reduce(s, OpAdd(), 0u, red);
  if (threadIdx.x == 0) bsum[blockIdx.x] = s;
}

__device__ __forceinline__ u32 block_excl_u32(u32 x, u32* total, u32* wt) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  u32 inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    u32 y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  __syncthreads();
  if (lane == 31) wt[w] = inc;
  __syncthreads();
  if (w == 0) {
    u32 v = lane < nw ? wt[lane] : 0u, vi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      u32 y = __shfl_up_sync(0xffffffffu, vi, o);
      if (lane >= o) vi += y;
    }
    if (lane < nw) wt[lane] = vi - v;
    if (lane == 31) wt[32] = vi;
  }
  __syncthreads();
  const u32 r = wt[w] + inc - x;
  *total = wt[32];
  return r;
}

__global__ void __launch_bounds__(kScanT) k_sbt_top(u32* bsum, u32 nb) {
  __shared__ u32 wt[33];
  u32 carry = 0;
  for (u32 c0 = 0; c0 < nb; c0 += kScanB) {
    u32 v[kScanI], s = 0;
#pragma unroll
    for (int k = 0; k < kScanI; ++k) {
      const u32 i = c0 + threadIdx.x * kScanI + k;
      v[k] = i < nb ? bsum[i] : 0u;
      s += v[k];
    }
    u32 tot;
    u32 ex = block_excl_u32(s, &tot, wt) + carry;
#pragma unroll
    for (int k = 0; k < kScanI; ++k) {
      const u32 i = c0 + threadIdx.x * kScanI + k;
      if (i < nb) bsum[i] = ex;
      ex += v[k];
    }
    carry += tot;
  }
}

// Offsets (exclusive) into off[] and cur[]; the occupied slots are appended
// to `used_list` (in no particular order) and counted in *n_used.
__global__ void __launch_bounds__(kScanT) k_sbt_down(const u32* cnt, u64 len, const u32* bsum, u32* off, u32* cur,
                                                    u64* n_used, u32* used_list) {
  __shared__ u32 wt[33];
  __shared__ u32 wt2[33];
  __shared__ u64 s_base;
  const u64 base = (u64)blockIdx.x * kScanB + (u64)threadIdx.x * kScanI;
  u32 v[kScanI], s = 0, used = 0;
#pragma unroll
  for (int k = 0; k < kScanI; ++k) {
    v[k] = base + k < len ? cnt[base + k] : 0u;
    s += v[k];
    used += v[k] != 0u;
  }
  u32 tot;
  u32 ex = block_excl_u32(s, &tot, wt) + bsum[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanI; ++k) {
    if (base + k < len) {
      off[base + k] = ex;
      cur[base + k] = ex;
    }
    ex += v[k];
  }
  u32 utot;
  u32 uex = block_excl_u32(used, &utot, wt2);
  if (threadIdx.x == 0) s_base = utot ? atomicAdd(n_used, (u64)utot) : 0ull;
  __syncthreads();
  u64 p = s_base + uex;
#pragma unroll
  for (int k = 0; k < kScanI; ++k)
    if (v[k]) used_list[p++] = (u32)(base + k);
}

constexpr int kScThreads = 256;
constexpr int kScItems = 8;

// Scatter each word's low 12 bits into its superblock's segment.
__global__ void __launch_bounds__(kScThreads) k_mem_scatter(HashArgs a) {
  const u64 n = umin64(a.arena->st.n_words, a.n_cap);
  const int lane = threadIdx.x & 31;
  const u32 lt = (1u << lane) - 1u;
  const u64 per_block = (u64)kScThreads * kScItems;
  for (u64 t0 = (u64)blockIdx.x * per_block; t0 < n; t0 += (u64)gridDim.x * per_block) {
    u64 w[kScItems];
#pragma unroll
    for (int k = 0; k < kScItems; ++k) {
      const u64 i = t0 + (u64)k * kScThreads + threadIdx.x;
      w[k] = i < n ? __ldcs(a.words + i) : 0ull;
    }
    u32 slot[kScItems];
    u64 pos[kScItems], first[kScItems];
#pragma unroll
    for (int k = 0; k < kScItems; ++k) {
      const u64 i = t0 + (u64)k * kScThreads + threadIdx.x;
      pos[k] = sbt_hash((w[k] >> 12) + 1ull) & a.tab.mask;
      first[k] = i < n ? a.tab.keys[pos[k]] : 0ull;
    }
#pragma unroll
    for (int k = 0; k < kScItems; ++k) {
      const u64 i = t0 + (u64)k * kScThreads + threadIdx.x;
      const u64 key = (w[k] >> 12) + 1ull;
      slot[k] = i >= n ? kNoSlot : (first[k] == key ? (u32)pos[k] : sbt_find(a.tab, key));
    }
#pragma unroll
    for (int k = 0; k < kScItems; ++k) {
      const bool valid = slot[k] != kNoSlot;
      const u32 key = valid ? slot[k] : (0xFFFFFFE0u | (u32)lane);
      const u32 peers = __match_any_sync(0xffffffffu, key);
      const int leader = __ffs(peers) - 1;
      u32 base = 0;
      if (valid && lane == leader) base = atomicAdd(&a.tab.cur[slot[k]], (u32)__popc(peers));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (valid) a.low[base + __popc(peers & lt)] = (uint16_t)(w[k] & 0xFFFull);
    }
  }
}

constexpr int kSgThreads = 256;
constexpr int kCocSmem = 256;  // group sizes below this are counted in shared memory

// Emits one group size of skip level `lev`: shared bins, then the global
// dense bins, then the overflow list.
__device__ __forceinline__ void emit_group(u32 (*coc)[kCocSmem], int lev, u32 c, u64* over, u64 cap,
                                           Arena* ar) {
  if (c == 0) return;
  if (c < (u32)kCocSmem) atomicAdd(&coc[lev][c], 1u);
  else if (c < (u32)kCocDense) atomicAdd(&ar->mem_coc[lev][c], 1ull);
  else overflow_append(over, cap, &ar->st, lev, c);
}

// One block per superblock segment at a time (grid-stride over the occupied slots).
__global__ void __launch_bounds__(kSgThreads) k_mem_segments(HashArgs a) {
  __shared__ u32 hist[4096];
  __shared__ u32 coc[kLevels][kCocSmem];
  __shared__ u32 wsum[kSgThreads / 32];
  __shared__ u64 red64[32];
  DevState* st = &a.arena->st;
  for (int i = threadIdx.x; i < kLevels * kCocSmem; i += kSgThreads) (&coc[0][0])[i] = 0u;
  for (int i = threadIdx.x; i < 4096; i += kSgThreads) hist[i] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  u64 fp = 0, ur = 0, uw = 0;
  const u64 n_used = umin64(*a.n_used, a.tab.mask + 1);
  for (u64 u = blockIdx.x; u < n_used; u += gridDim.x) {
    const u32 s = a.used_list[u];
    const u32 cnt = a.tab.cnt[s];
    const u32 off = a.tab.off[s];
    const uint16_t* seg = a.low + off;
    for (u32 j = threadIdx.x; j < cnt; j += kSgThreads) atomicAdd(&hist[seg[j]], 1u);
    __syncthreads();
    // thread t owns addresses 8t .. 8t+7 (bins 16t .. 16t+15: read, write pairs)
    u32 c0[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const u32 r = hist[16 * threadIdx.x + 2 * k], wv = hist[16 * threadIdx.x + 2 * k + 1];
      c0[k] = r + wv;
      fp += c0[k] != 0u;
      ur += r != 0u;
      uw += wv != 0u;
      emit_group(coc, 0, c0[k], a.over, a.over_cap, a.arena);
    }
    u32 c1[4], c2[2];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      c1[k] = c0[2 * k] + c0[2 * k + 1];
      emit_group(coc, 1, c1[k], a.over, a.over_cap, a.arena);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      c2[k] = c1[2 * k] + c1[2 * k + 1];
      emit_group(coc, 2, c2[k], a.over, a.over_cap, a.arena);
    }
    u32 g = c2[0] + c2[1];
    emit_group(coc, 3, g, a.over, a.over_cap, a.arena);
    // levels 4..8: pairs, quads, ... of threads inside the warp
#pragma unroll
    for (int lev = 4; lev <= 8; ++lev) {
      const int span = 1 << (lev - 3);  // threads per group
      g += __shfl_xor_sync(0xffffffffu, g, span >> 1);
      if ((lane & (span - 1)) == 0) emit_group(coc, lev, g, a.over, a.over_cap, a.arena);
    }
    if (lane == 0) wsum[wp] = g;  // 256 addresses per warp
    __syncthreads();
    if (threadIdx.x < 4) {  // level 9: pairs of warps
      const u32 v = wsum[2 * threadIdx.x] + wsum[2 * threadIdx.x + 1];
      emit_group(coc, 9, v, a.over, a.over_cap, a.arena);
    }
    if (threadIdx.x < 2) {  // level 10: quads of warps
      const u32 v = wsum[4 * threadIdx.x] + wsum[4 * threadIdx.x + 1] + wsum[4 * threadIdx.x + 2] +
                    wsum[4 * threadIdx.x + 3];
      emit_group(coc, 10, v, a.over, a.over_cap, a.arena);
    }
    // clear the bins this segment touched (all of them when it is large)
    if (cnt >= 2048) {
      for (int i = threadIdx.x; i < 4096; i += kSgThreads) hist[i] = 0u;
    } else {
      for (u32 j = threadIdx.x; j < cnt; j += kSgThreads) hist[seg[j]] = 0u;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < kLevels * kCocSmem; i += kSgThreads) {
    const u32 c = (&coc[0][0])[i];
    if (c) atomicAdd(&a.arena->mem_coc[i / kCocSmem][i % kCocSmem], (u64)c);
  }
  fp = block_reduce(fp, OpAdd(), 0ull, red64);
  ur = block_reduce(ur, OpAdd(), 0ull, red64);
  uw = block_reduce(uw, OpAdd(), 0ull, red64);
  if (threadIdx.x == 0) {
    if (fp) atomicAdd(&st->footprint, fp);
    if (ur) atomicAdd(&st->unique_reads, ur);
    if (uw) atomicAdd(&st->unique_writes, uw);
  }
}

}  // namespace

size_t sbt_scan_words(u64 cap) { return (size_t)((cap + kScanB - 1) / kScanB + 1); }

void launch_mem_hash(const HashArgs& a, cudaStream_t s) {
  const u64 C = a.tab.mask + 1;
  const u32 nb = (u32)((C + kScanB - 1) / kScanB);
  k_sbt_reduce<<<nb, kScanT, 0, s>>>(a.tab.cnt, C, a.scan_tmp);
  k_sbt_top<<<1, kScanT, 0, s>>>(a.scan_tmp, nb);
  k_sbt_down<<<nb, kScanT, 0, s>>>(a.tab.cnt, C, a.scan_tmp, a.tab.off, a.tab.cur, a.n_used, a.used_list);
  k_mem_scatter<<<a.grid_scatter, kScThreads, 0, s>>>(a);
  k_mem_segments<<<a.grid_segments, kSgThreads, 0, s>>>(a);
  count_launches(5);
}

}  // namespace aiwc
