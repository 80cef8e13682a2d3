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
constexpr u32 kBigSeg = 16384;  // segments with at least this many events are split into chunks

__global__ void __launch_bounds__(kScanT) k_sbt_reduce(const u32* cnt, u64 len, u32* bsum, const u32* gate,
                                                      u32 want) {
  if (!gate_open(gate, want)) return;
  __shared__ u32 red[32];
  const u64 base = (u64)blockIdx.x * kScanB + (u64)threadIdx.x * kScanI;
  u32 s = 0;
#pragma unroll
  for (int k = 0; k < kScanI; ++k)
    if (base + k < len) {
#pragma unroll
      for (int q = 0; q < kSbtStripes; ++q) s += cnt[(u64)q * len + base + k];
    }
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

// Segment offsets (exclusive prefix of the counts) into off[]. Occupied slots are listed (in no
// particular order): those with fewer than kBigSeg events from the front of
// used_list (count in n_used[0]), the others from the back (n_used[1]). The
// counter stripes become each slot's total (stripe 0) and, in stripe s > 0,
// the offset where stripe s's events start in the slot's segment.
__global__ void __launch_bounds__(kScanT) k_sbt_down(u32* cnt, u64 len, const u32* bsum, u32* off,
                                                    u64* n_used, u32* used_list, const u32* gate, u32 want) {
  if (!gate_open(gate, want)) return;
  __shared__ u32 wt[33];
  __shared__ u32 wt2[33];
  __shared__ u32 wt3[33];
  __shared__ u64 s_base, b_base;
  const u64 base = (u64)blockIdx.x * kScanB + (u64)threadIdx.x * kScanI;
  u32 v[kScanI], c[kScanI][kSbtStripes], s = 0, small = 0, big = 0;
#pragma unroll
  for (int k = 0; k < kScanI; ++k) {
    v[k] = 0u;
#pragma unroll
    for (int q = 0; q < kSbtStripes; ++q) {
      c[k][q] = base + k < len ? cnt[(u64)q * len + base + k] : 0u;
      v[k] += c[k][q];
    }
    s += v[k];
    small += v[k] != 0u && v[k] < kBigSeg;
    big += v[k] >= kBigSeg;
  }
  u32 tot;
  u32 ex = block_excl_u32(s, &tot, wt) + bsum[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanI; ++k) {
    if (base + k < len) {
      off[base + k] = ex;
      if (v[k]) {
        cnt[base + k] = v[k];
        u32 at = ex + c[k][0];
#pragma unroll
        for (int q = 1; q < kSbtStripes; ++q) {
          cnt[(u64)q * len + base + k] = at;
          at += c[k][q];
        }
      }
    }
    ex += v[k];
  }
  u32 stot, btot;
  const u32 sex = block_excl_u32(small, &stot, wt2);
  const u32 bex = block_excl_u32(big, &btot, wt3);
  if (threadIdx.x == 0) {
    s_base = stot ? atomicAdd(&n_used[0], (u64)stot) : 0ull;
    b_base = btot ? atomicAdd(&n_used[1], (u64)btot) : 0ull;
  }
  __syncthreads();
  u64 ps = s_base + sex, pb = b_base + bex;
#pragma unroll
  for (int k = 0; k < kScanI; ++k) {
    if (v[k] != 0u && v[k] < kBigSeg) used_list[ps++] = (u32)(base + k);
    else if (v[k] >= kBigSeg) used_list[len - 1 - pb++] = (u32)(base + k);
  }
}

constexpr int kScThreads = 256;
constexpr int kScItems = 8;

// Scatter each event's low 12 bits into its superblock's segment, at the
// offset where its counter stripe starts in the segment plus its rank within
// the stripe (from the ingest).
__global__ void __launch_bounds__(kScThreads, 4) k_mem_scatter(HashArgs a) {
  if (!gate_open(a.gate, a.gate_want)) return;
  const u64 n = umin64(a.arena->st.n_words, a.n_cap);
  const u64 per_block = (u64)kScThreads * kScItems;
  for (u64 t0 = (u64)blockIdx.x * per_block; t0 < n; t0 += (u64)gridDim.x * per_block) {
    u64 sw[kScItems];
#pragma unroll
    for (int k = 0; k < kScItems; ++k) {
      const u64 i = t0 + (u64)k * kScThreads + threadIdx.x;
      sw[k] = i < n ? __ldcs(a.slotw + i) : (u64)kSlotWordNone;
    }
    const u64 C = a.tab.mask + 1;
    u32 off[kScItems];
#pragma unroll
    for (int k = 0; k < kScItems; ++k) {
      const u32 w = (u32)sw[k];
      const u32 stripe = (u32)(sw[k] >> 32) & (u32)(kSbtStripes - 1);
      off[k] = w == kSlotWordNone ? 0u
               : stripe ? __ldg(a.tab.cnt + (u64)stripe * C + (w >> 12))
                        : __ldg(a.tab.off + (w >> 12));
    }
#pragma unroll
    for (int k = 0; k < kScItems; ++k) {
      const u32 w = (u32)sw[k];
      if (w != kSlotWordNone) a.low[off[k] + (u32)(sw[k] >> kRankShift)] = (uint16_t)(w & 0xFFFu);
    }
  }
}

constexpr int kRbThreads = 256;
constexpr int kRbItems = 8;

// Sort-plan fallback: 64-bit words rebuilt from slot words and table keys,
// appended after the spilled words (order is irrelevant to the sort).
__global__ void __launch_bounds__(kRbThreads) k_rebuild_words(const u64* slotw, SbTable tab, u64* words,
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
      sw[k] = i < n ? (u32)slotw[i] : kSlotWordNone;
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

constexpr int kCocSmem = 128;  // group sizes below this are counted in shared memory (more resident blocks than 256)

// Adds `times` groups of size c at skip levels lo..lev (lo < lev only when the
// low address bits are all zero, so that those levels group identically):
// shared bins below kCocSmem (level lev only: the block copies that row to
// levels lo..lev when it flushes), global dense bins below kCocDense, the
// overflow list above (one entry per group, reserved with a single atomic).
__device__ __forceinline__ void emit_n(u32 (*coc)[kCocSmem], int lo, int lev, u32 c, u32 times, const HashArgs& a) {
  if (c == 0u || times == 0u) return;
  if (c < (u32)kCocSmem) {
    atomicAdd(&coc[lev][c], times);
    return;
  }
  for (int l = lo; l <= lev; ++l) {
    if (c < (u32)kCocDense) {
      atomicAdd(&a.arena->mem_coc[l][c], (u64)times);
    } else {
      DevState* st = &a.arena->st;
      const u64 e = ((u64)l << 56) | ((u64)c & kValueMask);
      const u64 idx = atomicAdd(&st->n_over, (u64)times);
      for (u32 t = 0; t < times && idx + t < a.over_cap; ++t) a.over[idx + t] = e;
      if (idx + times > a.over_cap) atomicOr(&st->err, kErrOverflow);
      atomicOr(&st->over_or, e);
      atomicAnd(&st->over_and, e);
    }
  }
}

// Emits this thread's K group sizes of one level: equal neighbours are
// merged first, and when every lane of the warp holds K copies of one size
// the warp adds them with a single atomic. All 32 lanes must call it.
template <int K>
__device__ __forceinline__ void emit_level(u32 (*coc)[kCocSmem], int lo, int lev, const u32 (&c)[K],
                                           const HashArgs& a) {
  const int lane = threadIdx.x & 31;
  bool same = true;
#pragma unroll
  for (int k = 1; k < K; ++k) same &= c[k] == c[0];
  const u32 c0 = __shfl_sync(0xffffffffu, c[0], 0);
  if (__all_sync(0xffffffffu, same && c[0] == c0)) {
    if (lane == 0) emit_n(coc, lo, lev, c0, 32u * K, a);
    return;
  }
  u32 cur = c[0], run = 1;
#pragma unroll
  for (int k = 1; k < K; ++k) {
    if (c[k] == cur) {
      ++run;
    } else {
      emit_n(coc, lo, lev, cur, run, a);
      cur = c[k];
      run = 1;
    }
  }
  emit_n(coc, lo, lev, cur, run, a);
}

// Segment geometry when the S low address bits of every event are zero: a
// superblock (2048 addresses) holds NA = 2048 >> S possible addresses; T =
// NA / 8 threads walk it, 8 consecutive ones each. Compressed level k (groups
// of 2^k possible addresses) is skip level S + k, and skip levels 0..S group
// exactly like level S.
template <int S>
struct SegShape {
  static constexpr int NA = 2048 >> S;
  static constexpr int T = NA / 8;
  static constexpr int W = T / 32;
};

// Walks one superblock histogram (reads in [0, NA), writes in [NA, 2 NA),
// compressed address order; shared or global memory) and emits the group
// sizes of every skip level. Called by all THREADS threads of the block; the
// first T walk. The caller synchronises before wsum or hist is reused.
template <int S, int THREADS>
__device__ __forceinline__ void walk_superblock(const u32* hist, u32 (*coc)[kCocSmem], u32* wsum, const HashArgs& a,
                                                u64& fp, u64& ur, u64& uw) {
  using Sh = SegShape<S>;
  constexpr int NA = Sh::NA, T = Sh::T, W = Sh::W;
  constexpr int KMAX = 10 - S;  // highest compressed level
  static_assert(THREADS >= T && THREADS % 32 == 0, "block too small for the walk");
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  if (threadIdx.x < T) {
    // thread t owns compressed addresses 8t .. 8t+7
    const uint4* hr = reinterpret_cast<const uint4*>(hist + 8 * threadIdx.x);
    const uint4* hw = reinterpret_cast<const uint4*>(hist + NA + 8 * threadIdx.x);
    const uint4 r0 = hr[0], r1 = hr[1], w0 = hw[0], w1 = hw[1];
    const u32 rd[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
    const u32 wr[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
    u32 c0[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      c0[j] = rd[j] + wr[j];
      fp += c0[j] != 0u;
      ur += rd[j] != 0u;
      uw += wr[j] != 0u;
    }
    emit_level<8>(coc, 0, S, c0, a);
    u32 c1[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) c1[k] = c0[2 * k] + c0[2 * k + 1];
    emit_level<4>(coc, S + 1, S + 1, c1, a);
    const u32 c2[2] = {c1[0] + c1[1], c1[2] + c1[3]};
    emit_level<2>(coc, S + 2, S + 2, c2, a);
    u32 g = c2[0] + c2[1];
    {
      const u32 c3[1] = {g};
      emit_level<1>(coc, S + 3, S + 3, c3, a);
    }
    // compressed levels 4..8: pairs, quads, ... of threads inside the warp;
    // the group's first lane holds the sum
#pragma unroll
    for (int k = 4; k <= 8; ++k) {
      if (k > KMAX) break;
      const int span = 1 << (k - 3);  // threads per group
      g += __shfl_xor_sync(0xffffffffu, g, span >> 1);
      if ((lane & (span - 1)) == 0) emit_n(coc, S + k, S + k, g, 1u, a);
    }
    if (W > 1 && lane == 0) wsum[wp] = g;  // 256 possible addresses per warp
  }
  __syncthreads();
  // compressed levels 9 and 10: pairs and quads of warps
  if (KMAX >= 9 && threadIdx.x < W / 2)
    emit_n(coc, S + 9, S + 9, wsum[2 * threadIdx.x] + wsum[2 * threadIdx.x + 1], 1u, a);
  if (KMAX >= 10 && threadIdx.x < W / 4)
    emit_n(coc, 10, 10, wsum[4 * threadIdx.x] + wsum[4 * threadIdx.x + 1] + wsum[4 * threadIdx.x + 2] +
                           wsum[4 * threadIdx.x + 3], 1u, a);
}

// End of a walking block: shared count-of-counts to the arena (the level-S
// row also counts for levels 0..S-1) and the footprint counters.
template <int S>
__device__ __forceinline__ void flush_walks(u32 (*coc)[kCocSmem], u64 fp, u64 ur, u64 uw, u64* red64,
                                            const HashArgs& a) {
  __syncthreads();
  for (int i = threadIdx.x; i < kLevels * kCocSmem; i += blockDim.x) {
    const u32 c = (&coc[0][0])[i];
    const int lev = i / kCocSmem, bin = i % kCocSmem;
    if (c)
      for (int l = (lev == S ? 0 : lev); l <= lev; ++l) atomicAdd(&a.arena->mem_coc[l][bin], (u64)c);
  }
  fp = block_reduce(fp, OpAdd(), 0ull, red64);
  ur = block_reduce(ur, OpAdd(), 0ull, red64);
  uw = block_reduce(uw, OpAdd(), 0ull, red64);
  if (threadIdx.x == 0) {
    DevState* st = &a.arena->st;
    if (fp) atomicAdd(&st->footprint, fp);
    if (ur) atomicAdd(&st->unique_reads, ur);
    if (uw) atomicAdd(&st->unique_writes, uw);
  }
}

template <int S>
__device__ __forceinline__ u32 hist_index(u32 v) {
  return (v & 1u) * (u32)SegShape<S>::NA + ((v >> 1) >> S);
}

// Adds the events seg[b0, b1) to a shared histogram, THREADS at a time.
template <int S, int THREADS>
__device__ __forceinline__ void fill_hist(u32* hist, const uint16_t* seg, u32 b0, u32 b1) {
  u32 j = b0 + threadIdx.x;
  for (; j + 3 * THREADS < b1; j += 4 * THREADS) {
    u32 v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = seg[j + q * THREADS];
#pragma unroll
    for (int q = 0; q < 4; ++q) atomicAdd(&hist[hist_index<S>(v[q])], 1u);
  }
  for (; j < b1; j += THREADS) atomicAdd(&hist[hist_index<S>(seg[j])], 1u);
}

// Small segments (fewer than kBigSeg events): one block of T threads per
// segment at a time, grid-stride over the front of the used list.
template <int S>
__global__ void __launch_bounds__(SegShape<S>::T) k_mem_segments(HashArgs a) {
  constexpr int NA = SegShape<S>::NA, T = SegShape<S>::T;
  if (!gate_open(a.gate, a.gate_want)) return;
  __shared__ __align__(16) u32 hist[2 * NA];
  __shared__ u32 coc[kLevels][kCocSmem];
  __shared__ u32 wsum[8];
  __shared__ u64 red64[32];
  const u64 n_list = umin64(a.n_used[0], a.tab.mask + 1);
  if (blockIdx.x >= n_list) return;  // no segment for this block
  for (int i = threadIdx.x; i < kLevels * kCocSmem; i += T) (&coc[0][0])[i] = 0u;
  for (int i = threadIdx.x; i < 2 * NA; i += T) hist[i] = 0u;
  __syncthreads();
  u64 fp = 0, ur = 0, uw = 0;
  for (u64 u = blockIdx.x; u < n_list; u += gridDim.x) {
    const u32 s = a.used_list[u];
    const u32 cnt = a.tab.cnt[s];
    const uint16_t* seg = a.low + a.tab.off[s];
    fill_hist<S, T>(hist, seg, 0u, cnt);
    __syncthreads();
    walk_superblock<S, T>(hist, coc, wsum, a, fp, ur, uw);
    // clear the bins this segment touched (all of them when it is large)
    if (cnt >= (u32)NA) {
      for (int i = threadIdx.x; i < 2 * NA; i += T) hist[i] = 0u;
    } else {
      for (u32 j = threadIdx.x; j < cnt; j += T) hist[hist_index<S>(seg[j])] = 0u;
    }
    __syncthreads();
  }
  flush_walks<S>(coc, fp, ur, uw, red64, a);
}

constexpr int kBfThreads = 256;
constexpr u32 kChunk = 4096;  // events per work item of a wide segment

// Wide segments (kBigSeg events or more, at the back of the used list):
// their events are cut into chunks of kChunk, dealt round-robin to all
// blocks; each block adds its chunk's histogram to the segment's global
// histogram in big_hist (zeroed beforehand, 2 NA words per wide segment).
template <int S>
__global__ void __launch_bounds__(kBfThreads) k_mem_big_fill(HashArgs a) {
  constexpr int NA = SegShape<S>::NA;
  if (!gate_open(a.gate, a.gate_want)) return;
  __shared__ __align__(16) u32 hist[2 * NA];
  __shared__ u32 m_off[kBfThreads], m_cnt[kBfThreads], m_pre[kBfThreads];
  __shared__ u32 wt[33];
  const u64 C = a.tab.mask + 1;
  const u64 n_big = umin64(umin64(a.n_used[1], C), a.big_cap);
  if (n_big == 0) return;
  for (int i = threadIdx.x; i < 2 * NA; i += kBfThreads) hist[i] = 0u;
  const u64 G = gridDim.x;
  u64 qbase = 0;  // chunks in earlier batches
  for (u64 i0 = 0; i0 < n_big; i0 += kBfThreads) {
    const u64 i = i0 + threadIdx.x;
    u32 nch = 0;
    __syncthreads();  // the previous batch's entries are no longer read
    if (i < n_big) {
      const u32 s = a.used_list[C - 1 - i];
      const u32 cnt = a.tab.cnt[s];
      m_off[threadIdx.x] = a.tab.off[s];
      m_cnt[threadIdx.x] = cnt;
      nch = (cnt + kChunk - 1) / kChunk;
    }
    u32 tot;
    m_pre[threadIdx.x] = block_excl_u32(nch, &tot, wt);
    __syncthreads();
    const u32 nvalid = (u32)umin64(n_big - i0, (u64)kBfThreads);
    // this block takes the batch's chunks q with (qbase + q) % G == blockIdx.x
    for (u64 q = (blockIdx.x + G - qbase % G) % G; q < tot; q += G) {
      u32 lo = 0, hi = nvalid - 1;  // last entry whose first chunk is <= q
      while (lo < hi) {
        const u32 mid = (lo + hi + 1) >> 1;
        if (m_pre[mid] <= q) lo = mid; else hi = mid - 1;
      }
      const u32 b0 = (u32)(q - m_pre[lo]) * kChunk;
      const u32 b1 = min(m_cnt[lo], b0 + kChunk);
      fill_hist<S, kBfThreads>(hist, a.low + m_off[lo], b0, b1);
      __syncthreads();
      u32* gh = a.big_hist + (i0 + lo) * (u64)(2 * NA);
      for (int k = threadIdx.x; k < 2 * NA; k += kBfThreads) {
        const u32 v = hist[k];
        if (v) {
          atomicAdd(&gh[k], v);
          hist[k] = 0u;
        }
      }
      __syncthreads();
    }
    qbase += tot;
  }
}

// Walks the global histogram of every wide segment (grid-stride).
template <int S>
__global__ void __launch_bounds__(SegShape<S>::T) k_mem_big_walk(HashArgs a) {
  constexpr int NA = SegShape<S>::NA, T = SegShape<S>::T;
  if (!gate_open(a.gate, a.gate_want)) return;
  __shared__ u32 coc[kLevels][kCocSmem];
  __shared__ u32 wsum[8];
  __shared__ u64 red64[32];
  const u64 n_big = umin64(umin64(a.n_used[1], a.tab.mask + 1), a.big_cap);
  if (blockIdx.x == 0 && threadIdx.x == 0 && a.n_used[1] > a.big_cap) atomicOr(&a.arena->st.err, kErrOverflow);
  if (blockIdx.x >= n_big) return;  // no wide segment for this block
  for (int i = threadIdx.x; i < kLevels * kCocSmem; i += T) (&coc[0][0])[i] = 0u;
  __syncthreads();
  u64 fp = 0, ur = 0, uw = 0;
  for (u64 i = blockIdx.x; i < n_big; i += gridDim.x) {
    walk_superblock<S, T>(a.big_hist + i * (u64)(2 * NA), coc, wsum, a, fp, ur, uw);
    __syncthreads();
  }
  flush_walks<S>(coc, fp, ur, uw, red64, a);
}

template <typename K>
int resident_blocks(K kernel, int threads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  return per_sm < 1 ? 1 : per_sm;
}

template <int S>
void launch_segments_shift(const HashArgs& a, cudaStream_t s) {
  constexpr int T = SegShape<S>::T;
  const int sm = a.sm_count;
  k_mem_big_fill<S><<<sm * resident_blocks(k_mem_big_fill<S>, kBfThreads), kBfThreads, 0, s>>>(a);
  k_mem_big_walk<S><<<sm * 2, T, 0, s>>>(a);
  k_mem_segments<S><<<sm * resident_blocks(k_mem_segments<S>, T), T, 0, s>>>(a);
  count_launches(3);
}

}  // namespace

size_t sbt_scan_words(u64 cap) { return (size_t)((cap + kScanB - 1) / kScanB + 1); }

void launch_mem_hash_scatter(const HashArgs& a, cudaStream_t s) {
  const u64 C = a.tab.mask + 1;
  const u32 nb = (u32)((C + kScanB - 1) / kScanB);
  k_sbt_reduce<<<nb, kScanT, 0, s>>>(a.tab.cnt, C, a.scan_tmp, a.gate, a.gate_want);
  k_sbt_top<<<1, kScanT, 0, s>>>(a.scan_tmp, nb, a.gate, a.gate_want);
  k_sbt_down<<<nb, kScanT, 0, s>>>(a.tab.cnt, C, a.scan_tmp, a.tab.off, a.n_used, a.used_list, a.gate,
                                   a.gate_want);
  k_mem_scatter<<<a.grid_scatter, kScThreads, 0, s>>>(a);
  count_launches(4);
}

u64 mem_hash_big_segments(u64 n_words, size_t bytes, int seg_shift) {
  const u64 per = 2ull * (u64)(2048 >> seg_shift) * 4;
  return std::min<u64>(n_words / kBigSeg, bytes / per);
}

void launch_mem_hash_segments(const HashArgs& a, cudaStream_t s) {
  if (a.big_cap) cudaMemsetAsync(a.big_hist, 0, a.big_cap * 2ull * (u64)(2048 >> a.seg_shift) * 4, s);
  switch (a.seg_shift) {
    case 1: launch_segments_shift<1>(a, s); break;
    case 2: launch_segments_shift<2>(a, s); break;
    case 3: launch_segments_shift<3>(a, s); break;
    default: launch_segments_shift<0>(a, s); break;
  }
}

void launch_mem_hash(const HashArgs& a, cudaStream_t s) {
  launch_mem_hash_scatter(a, s);
  launch_mem_hash_segments(a, s);
}

void launch_rebuild_words(const u64* slotw, SbTable tab, u64* words, Arena* arena, int grid, cudaStream_t s,
                          const u32* gate, u32 gate_want) {
  k_rebuild_words<<<grid, kRbThreads, 0, s>>>(slotw, tab, words, arena, gate, gate_want);
  count_launches(1);
}

}  // namespace aiwc
