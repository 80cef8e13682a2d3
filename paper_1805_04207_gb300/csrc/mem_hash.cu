// Memory path without a sort ("hash" plan).
//
// Every group of skip level n <= 10 (key >> n, Sec. III) lies inside one
// superblock of 2^11 addresses (key >> 11). So instead of sorting 64-bit
// words we:
//   1. count the events of each superblock in an open-addressing table that
//      stays in L2 (done during ingest, see mem.cu),
//   2. scan the counts into segment offsets and scatter each event's low 12
//      bits (11 address bits and the store bit), taken from the 32-bit slot
//      word the ingest wrote, into its superblock's segment as a u16,
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

__global__ void __launch_bounds__(kScanT) k_sbt_reduce(const u32* cnt, u64 len, u32* bsum, const u32* gate,
                                                      u32 want) {
  if (!gate_open(gate, want)) return;
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

__global__ void __launch_bounds__(kScanT) k_sbt_top(u32* bsum, u32 nb, const u32* gate, u32 want) {
  if (!gate_open(gate, want)) return;
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
                                                    u64* n_used, u32* used_list, const u32* gate, u32 want) {
  if (!gate_open(gate, want)) return;
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
constexpr int kScItems = 16;

// Scatter each event's low 12 bits into its superblock's segment.
__global__ void __launch_bounds__(kScThreads) k_mem_scatter(HashArgs a) {
  if (!gate_open(a.gate, a.gate_want)) return;
  const u64 n = umin64(a.arena->st.n_words, a.n_cap);
  const int lane = threadIdx.x & 31;
  const u32 lt = (1u << lane) - 1u;
  const u64 per_block = (u64)kScThreads * kScItems;
  for (u64 t0 = (u64)blockIdx.x * per_block; t0 < n; t0 += (u64)gridDim.x * per_block) {
    u32 sw[kScItems];
#pragma unroll
    for (int k = 0; k < kScItems; ++k) {
      const u64 i = t0 + (u64)k * kScThreads + threadIdx.x;
      sw[k] = i < n ? __ldcs(a.slotw + i) : kSlotWordNone;
    }
    u32 peers[kScItems], base[kScItems];
#pragma unroll
    for (int k = 0; k < kScItems; ++k) {
      const bool valid = sw[k] != kSlotWordNone;
      peers[k] = __match_any_sync(0xffffffffu, valid ? (sw[k] >> 12) : (0xFFFFFFE0u | (u32)lane));
      base[k] = 0;
      if (valid && lane == __ffs(peers[k]) - 1) base[k] = atomicAdd(&a.tab.cur[sw[k] >> 12], (u32)__popc(peers[k]));
    }
#pragma unroll
    for (int k = 0; k < kScItems; ++k) {
      const u32 b = __shfl_sync(0xffffffffu, base[k], __ffs(peers[k]) - 1);
      if (sw[k] != kSlotWordNone) a.low[b + __popc(peers[k] & lt)] = (uint16_t)(sw[k] & 0xFFFu);
    }
  }
}

constexpr int kRbThreads = 256;
constexpr int kRbItems = 8;

// Sort-plan fallback: 64-bit words rebuilt from slot words and table keys,
// appended after the spilled words (order is irrelevant to the sort).
__global__ void __launch_bounds__(kRbThreads) k_rebuild_words(const u32* slotw, SbTable tab, u64* words,
                                                             Arena* arena, const u32* gate, u32 want) {
  if (!gate_open(gate, want)) return;
  __shared__ u32 scan_tot[33];
  __shared__ u64 s_base;
  DevState* st = &arena->st;
  const u64 n = st->n_words;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const u64 per_block = (u64)kRbThreads * kRbItems;
  for (u64 t0 = (u64)blockIdx.x * per_block; t0 < n; t0 += (u64)gridDim.x * per_block) {
    u32 sw[kRbItems];
    u32 cnt = 0;
#pragma unroll
    for (int k = 0; k < kRbItems; ++k) {
      const u64 i = t0 + (u64)k * kRbThreads + threadIdx.x;
      sw[k] = i < n ? slotw[i] : kSlotWordNone;
      cnt += sw[k] != kSlotWordNone;
    }
    u32 inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      u32 y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) scan_tot[w] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
      u32 t = 0;
      for (int q = 0; q < kRbThreads / 32; ++q) { u32 c = scan_tot[q]; scan_tot[q] = t; t += c; }
      s_base = atomicAdd(&st->n_spill, (u64)t);  // appends after the spilled words
    }
    __syncthreads();
    u64 pos = s_base + scan_tot[w] + inc - cnt;
#pragma unroll
    for (int k = 0; k < kRbItems; ++k)
      if (sw[k] != kSlotWordNone) words[pos++] = ((tab.keys[sw[k] >> 12] - 1ull) << 12) | (sw[k] & 0xFFFu);
    __syncthreads();
  }
}

constexpr int kSgThreads = 256;
constexpr int kCocSmem = 256;  // group sizes below this are counted in shared memory

// Adds `times` groups of size c at skip level `lev`: shared bins below
// kCocSmem, global dense bins below kCocDense, the overflow list above.
__device__ __forceinline__ void emit_n(u32 (*coc)[kCocSmem], int lev, u32 c, u32 times, const HashArgs& a) {
  if (c == 0u || times == 0u) return;
  if (c < (u32)kCocSmem) atomicAdd(&coc[lev][c], times);
  else if (c < (u32)kCocDense) atomicAdd(&a.arena->mem_coc[lev][c], (u64)times);
  else
    for (u32 t = 0; t < times; ++t) overflow_append(a.over, a.over_cap, &a.arena->st, lev, c);
}

// Emits this thread's K group sizes of one level: equal neighbours are
// merged first, and when every lane of the warp holds K copies of one size
// the warp adds them with a single atomic. All 32 lanes must call it.
template <int K>
__device__ __forceinline__ void emit_level(u32 (*coc)[kCocSmem], int lev, const u32 (&c)[K], const HashArgs& a) {
  const int lane = threadIdx.x & 31;
  bool same = true;
#pragma unroll
  for (int k = 1; k < K; ++k) same &= c[k] == c[0];
  const u32 c0 = __shfl_sync(0xffffffffu, c[0], 0);
  if (__all_sync(0xffffffffu, same && c[0] == c0)) {
    if (lane == 0) emit_n(coc, lev, c0, 32u * K, a);
    return;
  }
  u32 cur = c[0], run = 1;
#pragma unroll
  for (int k = 1; k < K; ++k) {
    if (c[k] == cur) {
      ++run;
    } else {
      emit_n(coc, lev, cur, run, a);
      cur = c[k];
      run = 1;
    }
  }
  emit_n(coc, lev, cur, run, a);
}

// One block per superblock segment at a time (grid-stride over the occupied slots).
__global__ void __launch_bounds__(kSgThreads) k_mem_segments(HashArgs a) {
  if (!gate_open(a.gate, a.gate_want)) return;
  __shared__ __align__(16) u32 hist[4096];
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
    const uint4* hv = reinterpret_cast<const uint4*>(hist + 16 * threadIdx.x);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4 v = hv[q];
      c0[2 * q] = v.x + v.y;
      c0[2 * q + 1] = v.z + v.w;
      fp += (v.x + v.y != 0u) + (v.z + v.w != 0u);
      ur += (v.x != 0u) + (v.z != 0u);
      uw += (v.y != 0u) + (v.w != 0u);
    }
    emit_level<8>(coc, 0, c0, a);
    u32 c1[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) c1[k] = c0[2 * k] + c0[2 * k + 1];
    emit_level<4>(coc, 1, c1, a);
    u32 c2[2] = {c1[0] + c1[1], c1[2] + c1[3]};
    emit_level<2>(coc, 2, c2, a);
    u32 g = c2[0] + c2[1];
    {
      const u32 c3[1] = {g};
      emit_level<1>(coc, 3, c3, a);
    }
    // levels 4..8: pairs, quads, ... of threads inside the warp; the group's
    // first lane holds the sum, the others emit nothing
#pragma unroll
    for (int lev = 4; lev <= 8; ++lev) {
      const int span = 1 << (lev - 3);  // threads per group
      g += __shfl_xor_sync(0xffffffffu, g, span >> 1);
      if ((lane & (span - 1)) == 0) emit_n(coc, lev, g, 1u, a);
    }
    if (lane == 0) wsum[wp] = g;  // 256 addresses per warp
    __syncthreads();
    if (threadIdx.x < 4) emit_n(coc, 9, wsum[2 * threadIdx.x] + wsum[2 * threadIdx.x + 1], 1u, a);
    if (threadIdx.x < 2)
      emit_n(coc, 10, wsum[4 * threadIdx.x] + wsum[4 * threadIdx.x + 1] + wsum[4 * threadIdx.x + 2] +
                          wsum[4 * threadIdx.x + 3], 1u, a);
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
  k_sbt_reduce<<<nb, kScanT, 0, s>>>(a.tab.cnt, C, a.scan_tmp, a.gate, a.gate_want);
  k_sbt_top<<<1, kScanT, 0, s>>>(a.scan_tmp, nb, a.gate, a.gate_want);
  k_sbt_down<<<nb, kScanT, 0, s>>>(a.tab.cnt, C, a.scan_tmp, a.tab.off, a.tab.cur, a.n_used, a.used_list, a.gate,
                                   a.gate_want);
  k_mem_scatter<<<a.grid_scatter, kScThreads, 0, s>>>(a);
  k_mem_segments<<<a.grid_segments, kSgThreads, 0, s>>>(a);
  count_launches(5);
}

void launch_rebuild_words(const u32* slotw, SbTable tab, u64* words, Arena* arena, int grid, cudaStream_t s,
                          const u32* gate, u32 gate_want) {
  k_rebuild_words<<<grid, kRbThreads, 0, s>>>(slotw, tab, words, arena, gate, gate_want);
  count_launches(1);
}

}  // namespace aiwc
