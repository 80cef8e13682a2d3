// Memory-event path: ingest (one 16-byte event -> one 64-bit sort word) and
// the per-skip-level run lengths over the sorted words.
//
// Sort word of an access: (space << 62) | (addr << 1) | store, i.e. the key
// (space, address) of Table I's memory rows with the read/write bit below
// it. Sorting the words groups equal addresses and, inside an address, reads
// before writes; the group of skip level n (Sec. III: n = 0 global entropy,
// n = 1..10 local entropies) is word >> (n + 1).
#include <algorithm>

#include "aiwc_internal.cuh"
#include "common.cuh"
#include "runs.cuh"

namespace aiwc {
namespace {

constexpr int kIngestThreads = 256;
constexpr int kHashItems = 4;  // events per thread and block-tile in the hash plan (8 in the sort plan)

// Hash plan: places the kept words' superblocks in the table, counts them in
// this warp's counter stripe and forms their slot words (sentinel for words
// the table cannot place, whose full words go to the spill list). All lanes
// of the warp call it.
template <int ITEMS>
__device__ __forceinline__ void place_words(const MemIngestArgs& a, DevState* st, const u64 (&word)[ITEMS],
                                            const bool (&keep)[ITEMS], u64 (&sw)[ITEMS], u32* sbt_fail) {
  const int lane = threadIdx.x & 31;
  // batch the home-slot loads, then resolve
  u32 pos[ITEMS];
  u64 first[ITEMS];
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    pos[k] = (u32)(sbt_hash((word[k] >> 12) + 1ull) & a.tab.mask);
    // an L1-cached copy may still read 0 for a slot another SM just
    // claimed; sbt_place then loses the CAS and reads the real key
    first[k] = keep[k] ? a.tab.keys[pos[k]] : 0ull;
  }
  u32 slot[ITEMS];
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    slot[k] = kNoSlot;
    if (keep[k]) {
      slot[k] = sbt_place(a.tab, (word[k] >> 12) + 1ull, pos[k], first[k]);
      if (slot[k] == kNoSlot) {
        *sbt_fail = 1u;
        a.spill[atomicAdd(&st->n_spill, 1ull)] = word[k];
      }
    }
  }
  // all counting atomics in flight before any result is needed; this warp's
  // counter stripe
  const u32 stripe = (blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5)) & (u32)(kSbtStripes - 1);
  u32* cnt_s = a.tab.cnt + (u64)stripe * (a.tab.mask + 1);
  u32 peers[ITEMS], rb[ITEMS];
#pragma unroll
  for (int k = 0; k < ITEMS; ++k)
    peers[k] = __match_any_sync(0xffffffffu, slot[k] != kNoSlot ? slot[k] : (0xFFFFFFE0u | (u32)lane));
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    rb[k] = 0u;
    if (slot[k] != kNoSlot && lane == __ffs(peers[k]) - 1) rb[k] = atomicAdd(&cnt_s[slot[k]], (u32)__popc(peers[k]));
  }
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const u32 r = __shfl_sync(0xffffffffu, rb[k], __ffs(peers[k]) - 1) + (u32)__popc(peers[k] & ((1u << lane) - 1u));
    if (slot[k] != kNoSlot && r >= kRankLimit) *sbt_fail = 1u;
    sw[k] = slot[k] != kNoSlot ? (((u64)r << kRankShift) | ((u64)stripe << 32) | (slot[k] << 12) |
                                  (u32)(word[k] & 0xFFFull))
                               : (u64)kSlotWordNone;
  }
}

// One pass over the 16-byte events. Sort plan (HASH = false): writes the
// 64-bit sort word of every kept event. Hash plan (HASH = true): places the
// event's superblock (word >> 12) in the table, counts it there and writes
// the 32-bit slot word (slot << 12) | (word & 0xFFF) -- the table keeps the
// superblock, so the word can be rebuilt from the slot word -- with, in the
// high half, the warp's counter stripe and the event's rank among its
// superblock's events in that stripe (the count before it, from the same
// atomic), which with the stripes before it fixes its place in the
// superblock's segment. An event the table cannot place gets the sentinel slot word and
// its full word goes to the spill list. FILTER: the space mask drops events,
// so outputs are compacted behind one atomicAdd per block-tile. FULL: a.n is
// a multiple of the block tile, so every event slot is valid (no tests).
// Hash plan: six blocks per SM (40 registers, a few spilled) hide more of the
// table-probe and atomic latency than four blocks of 64 registers.
template <bool FILTER, bool HASH, bool FULL>
__global__ void __launch_bounds__(kIngestThreads, HASH ? 6 : 3) k_mem_ingest(MemIngestArgs a) {
  constexpr int ITEMS = HASH ? kHashItems : 8;
  __shared__ u64 red64[32];
  __shared__ u32 red32[32];
  __shared__ u32 scan_tot[33];
  __shared__ u64 s_base;
  DevState* st = &a.arena->st;
  const uint4* ev = reinterpret_cast<const uint4*>(a.ev);
  const int lane = threadIdx.x & 31;
  // per thread: counts fit 32 bits; the hash plan keeps no AND over the words
  // (the sort fallback then treats every set bit as varying, a superset)
  u32 writes = 0, kept = 0;
  u64 wor = 0, wand = HASH ? 0ull : ~0ull;
  u32 wmin = 0xFFFFFFFFu, wmax = 0u, err = 0u, sbt_fail = 0u;
  const u64 per_block = (u64)kIngestThreads * ITEMS;
  for (u64 t0 = (u64)blockIdx.x * per_block; t0 < a.n; t0 += (u64)gridDim.x * per_block) {
    uint4 e[ITEMS];
    bool valid[ITEMS];
    u64 word[ITEMS];
    bool keep[ITEMS];
    u32 nkeep = 0;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const u64 i = t0 + (u64)k * kIngestThreads + threadIdx.x;
      valid[k] = FULL || i < a.n;
      e[k] = valid[k] ? __ldcs(ev + i) : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
      const u64 addr = (u64)e[k].x | ((u64)e[k].y << 32);
      const u32 wi = e[k].z;
      const u32 flags = (e[k].w >> 8) & 0xFFu;
      const u32 space = (flags >> 1) & 3u;
      const u32 store = flags & 1u;
      mark_work_items(a.wi_bitmap, a.max_wi, wi, valid[k], &err);
      if (valid[k]) {
        if ((u64)wi < a.max_wi) {
          wmin = min(wmin, wi);
          wmax = max(wmax, wi);
        }
        if (addr >> 61) err |= kErrAddr;
      }
      keep[k] = valid[k] && (!FILTER || ((a.space_mask >> space) & 1u));
      word[k] = ((u64)space << 62) | ((addr & ((1ull << 61) - 1)) << 1) | store;
      if (keep[k]) {
        ++nkeep;
        writes += store;  // reads follow from the kept count
        wor |= word[k];
        if (!HASH) wand &= word[k];
      }
    }
    kept += nkeep;
    u64 sw[ITEMS];
    if (HASH) place_words<ITEMS>(a, st, word, keep, sw, &sbt_fail);
    if (FILTER) {
      // compact the kept outputs of this block-tile behind one atomicAdd
      const int w = threadIdx.x >> 5;
      u32 inc = nkeep;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        u32 y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      if (lane == 31) scan_tot[w] = inc;
      __syncthreads();
      if (threadIdx.x == 0) {
        u32 s = 0;
        for (int q = 0; q < kIngestThreads / 32; ++q) { u32 c = scan_tot[q]; scan_tot[q] = s; s += c; }
        s_base = atomicAdd(&st->n_words, (u64)s);
      }
      __syncthreads();
      u64 pos = s_base + scan_tot[w] + inc - nkeep;
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        if (keep[k]) {
          if (HASH) a.slotw[pos++] = sw[k];
          else a.words[pos++] = word[k];
        }
      }
      __syncthreads();
    } else {
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        const u64 i = t0 + (u64)k * kIngestThreads + threadIdx.x;
        if (valid[k]) {
          if (HASH) a.slotw[a.word_base + i] = sw[k];
          else a.words[a.word_base + i] = word[k];
        }
      }
    }
  }
  const u64 b_writes = block_reduce((u64)writes, OpAdd(), 0ull, red64);
  wor = block_reduce(wor, OpOr(), 0ull, red64);
  if (!HASH) wand = block_reduce(wand, OpAnd(), ~0ull, red64);
  const u64 b_kept = block_reduce((u64)kept, OpAdd(), 0ull, red64);
  const u64 reads = b_kept - b_writes;
  wmin = block_reduce(wmin, OpMin(), 0xFFFFFFFFu, red32);
  wmax = block_reduce(wmax, OpMax(), 0u, red32);
  err = block_reduce(err, OpOr(), 0u, red32);
  sbt_fail = block_reduce(sbt_fail, OpOr(), 0u, red32);
  if (threadIdx.x == 0) {
    if (sbt_fail) atomicOr(&st->sbt_overflow, 1u);
    if (reads) atomicAdd(&st->total_reads, reads);
    if (b_writes) atomicAdd(&st->total_writes, b_writes);
    if (b_kept) {
      atomicOr(&st->mem_or, wor);
      atomicAnd(&st->mem_and, wand);
      if (!FILTER) atomicAdd(&st->n_words, b_kept);
    }
    if (wmin <= wmax) {
      atomicMin(&st->wi_min, wmin);
      atomicMax(&st->wi_max, wmax);
    }
    if (err) atomicOr(&st->err, err);
  }
}

// Byte-granular addresses. A tile of kExpandTile events: k_expand_count sums
// the sizes of its kept events (and marks every event's work-item),
// k_expand_scan turns the tile sums into the tiles' offsets, and
// k_mem_ingest_bytes (below) ingests the tile's one-byte accesses there.
constexpr int kExpThreads = 256;
constexpr int kExpItems = (int)kExpandTile / kExpThreads;

__global__ void __launch_bounds__(kExpThreads) k_expand_count(ExpandArgs a) {
  __shared__ u32 red32[32];
  DevState* st = &a.arena->st;
  const uint4* ev = reinterpret_cast<const uint4*>(a.ev);
  const u32 ntiles = (u32)((a.n + kExpandTile - 1) / kExpandTile);
  u32 err = 0u, wmin = 0xFFFFFFFFu, wmax = 0u;
  for (u32 tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    u32 sum = 0u;
#pragma unroll
    for (int k = 0; k < kExpItems; ++k) {
      const u64 i = (u64)tile * kExpandTile + (u64)k * kExpThreads + threadIdx.x;
      const bool valid = i < a.n;
      const uint4 e = valid ? __ldg(ev + i) : make_uint4(0u, 0u, 0u, 0u);
      const u32 space = (e.w >> 9) & 3u;
      if ((a.space_mask >> space) & 1u) sum += e.w & 0xFFu;
      if (valid && (e.y >> 29)) err |= kErrAddr;  // start address outside the 61-bit domain
      mark_work_items(a.wi_bitmap, a.max_wi, e.z, valid, &err);
      if (valid && (u64)e.z < a.max_wi) {
        wmin = min(wmin, e.z);
        wmax = max(wmax, e.z);
      }
    }
    sum = block_reduce(sum, OpAdd(), 0u, red32);
    if (threadIdx.x == 0) a.tile_sum[tile] = sum;
  }
  err = block_reduce(err, OpOr(), 0u, red32);
  wmin = block_reduce(wmin, OpMin(), 0xFFFFFFFFu, red32);
  wmax = block_reduce(wmax, OpMax(), 0u, red32);
  if (threadIdx.x == 0) {
    if (err) atomicOr(&st->err, err);
    if (wmin <= wmax) {
      atomicMin(&st->wi_min, wmin);
      atomicMax(&st->wi_max, wmax);
    }
  }
}

__global__ void __launch_bounds__(1024) k_expand_scan(ExpandArgs a) {
  __shared__ u64 wsum[32];
  __shared__ u64 s_carry;
  const u32 ntiles = (u32)((a.n + kExpandTile - 1) / kExpandTile);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0ull;
  __syncthreads();
  for (u32 c0 = 0; c0 < ntiles; c0 += 1024) {
    const u32 t = c0 + threadIdx.x;
    const u64 v = t < ntiles ? (u64)a.tile_sum[t] : 0ull;
    u64 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u64 y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
      u64 s = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const u64 y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      wsum[lane] = s;
    }
    __syncthreads();
    if (t < ntiles) a.tile_off[t] = s_carry + (w ? wsum[w - 1] : 0ull) + x - v;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += wsum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *a.total = s_carry;
}

// Byte-granular ingest: a block stages a tile of kExpandTile events in
// shared memory -- each event's word at its start byte and the offset of its
// first byte among the tile's kept bytes, as k_expand_count laid them out --
// and forms the words of the tile's one-byte accesses on the fly,
// kIngestThreads * ITEMS at a time in offset order, so that consecutive lanes
// take consecutive bytes (a thread finds the event of byte q by binary search
// over the offsets); the words go through the same placement as the event
// ingest's and land at the tile's offset. Work-items and start addresses were
// handled by k_expand_count.
template <bool HASH>
__global__ void __launch_bounds__(kIngestThreads, HASH ? 6 : 3) k_mem_ingest_bytes(MemIngestArgs a, const u64* tile_off) {
  constexpr int ITEMS = HASH ? kHashItems : 8;
  constexpr int EV = (int)kExpandTile / kIngestThreads;  // events each thread stages
  __shared__ u64 s_word[kExpandTile];
  __shared__ u32 s_off[kExpandTile + 1];
  __shared__ u32 s_wsum[kIngestThreads / 32];
  __shared__ u64 red64[32];
  __shared__ u32 red32[32];
  DevState* st = &a.arena->st;
  const uint4* ev = reinterpret_cast<const uint4*>(a.ev);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  u64 writes = 0, wor = 0, wand = ~0ull, kept = 0;
  u32 err = 0u, sbt_fail = 0u;
  const u32 ntiles = (u32)((a.n + kExpandTile - 1) / kExpandTile);
  for (u32 tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const u64 base = (u64)tile * kExpandTile;
    u32 sz[EV];
    u32 mine = 0u;
#pragma unroll
    for (int k = 0; k < EV; ++k) {
      const u32 j = threadIdx.x * EV + k;
      const uint4 e = base + j < a.n ? __ldcs(ev + base + j) : make_uint4(0u, 0u, 0u, 0u);
      const u32 space = (e.w >> 9) & 3u, store = (e.w >> 8) & 1u;
      const u64 addr = (u64)e.x | ((u64)e.y << 32);
      s_word[j] = ((u64)space << 62) | (addr << 1) | store;  // address bits above 60 are dropped here
      sz[k] = ((a.space_mask >> space) & 1u) ? (e.w & 0xFFu) : 0u;
      mine += sz[k];
    }
    u32 x = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u32 y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_wsum[w] = x;
    __syncthreads();
    u32 run = x - mine;
    for (int q = 0; q < w; ++q) run += s_wsum[q];
#pragma unroll
    for (int k = 0; k < EV; ++k) {
      s_off[threadIdx.x * EV + k] = run;
      run += sz[k];
    }
    if (threadIdx.x == kIngestThreads - 1) s_off[kExpandTile] = run;
    __syncthreads();
    const u32 T = s_off[kExpandTile];
    const u64 o0 = a.word_base + tile_off[tile];
    for (u32 r0 = 0; r0 < T; r0 += kIngestThreads * ITEMS) {
      u64 word[ITEMS];
      bool keep[ITEMS];
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        const u32 q = r0 + k * kIngestThreads + threadIdx.x;
        keep[k] = q < T;
        word[k] = 0ull;
        if (keep[k]) {
          // the last event whose offset is <= q; it touches at least one byte
          u32 lo = 0u, hi = (u32)kExpandTile - 1u;
          while (lo < hi) {
            const u32 mid = (lo + hi + 1u) >> 1;
            if (s_off[mid] <= q) lo = mid;
            else hi = mid - 1u;
          }
          // one byte further is 2 in word units; the sum stays within 62
          // bits unless the byte leaves the 61-bit domain
          const u64 w0 = s_word[lo];
          word[k] = w0 + 2ull * (u64)(q - s_off[lo]);
          if ((word[k] ^ w0) >> 62) err |= kErrAddr;
          ++kept;
          writes += word[k] & 1ull;
          wor |= word[k];
          wand &= word[k];
        }
      }
      u64 sw[ITEMS];
      if (HASH) place_words<ITEMS>(a, st, word, keep, sw, &sbt_fail);
#pragma unroll
      for (int k = 0; k < ITEMS; ++k) {
        const u32 q = r0 + k * kIngestThreads + threadIdx.x;
        if (keep[k]) {
          if (HASH) a.slotw[o0 + q] = sw[k];
          else a.words[o0 + q] = word[k];
        }
      }
    }
    __syncthreads();  // the tile's staging is refilled next
  }
  writes = block_reduce(writes, OpAdd(), 0ull, red64);
  wor = block_reduce(wor, OpOr(), 0ull, red64);
  wand = block_reduce(wand, OpAnd(), ~0ull, red64);
  kept = block_reduce(kept, OpAdd(), 0ull, red64);
  const u64 reads = kept - writes;
  err = block_reduce(err, OpOr(), 0u, red32);
  sbt_fail = block_reduce(sbt_fail, OpOr(), 0u, red32);
  if (threadIdx.x == 0) {
    if (sbt_fail) atomicOr(&st->sbt_overflow, 1u);
    if (reads) atomicAdd(&st->total_reads, reads);
    if (writes) atomicAdd(&st->total_writes, writes);
    if (kept) {
      atomicOr(&st->mem_or, wor);
      atomicAnd(&st->mem_and, wand);
      atomicAdd(&st->n_words, kept);
    }
    if (err) atomicOr(&st->err, err);
  }
}

constexpr int kLvThreads = kTileThreads;
constexpr int kLvItems = kTileItems;

__global__ void __launch_bounds__(kLvThreads) k_mem_levels(LevelArgs a) {
  if (!gate_open(a.gate, a.gate_want)) return;
  __shared__ u32 coc[kLevels][kCocShared];
  __shared__ Seg sh[33];
  __shared__ u64 pre_slot[2];
  __shared__ u64 red64[32];
  DevState* st = &a.arena->st;
  for (int i = threadIdx.x; i < kLevels * kCocShared; i += kLvThreads) (&coc[0][0])[i] = 0u;
  __syncthreads();
  const u64 n = *a.n;
  const u64* words = *a.cur ? a.b : a.a;
  const u32 ntiles = (u32)((n + kTile - 1) / kTile);
  u64 heads0 = 0, ur = 0, uw = 0;
  for (u32 tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const u64 base = (u64)tile * kTile;
    const u64 pos0 = base + (u64)threadIdx.x * kLvItems;
    const int nvalid = pos0 < n ? (int)umin64(n - pos0, (u64)kLvItems) : 0;
    const u64 tile_n = umin64(n - base, (u64)kTile);
    u64 key[kLvItems];
    if (nvalid == kLvItems) {
      const ulonglong2* p = reinterpret_cast<const ulonglong2*>(words + pos0);
#pragma unroll
      for (int k = 0; k < kLvItems / 2; ++k) {
        ulonglong2 v = p[k];
        key[2 * k] = v.x;
        key[2 * k + 1] = v.y;
      }
    } else {
#pragma unroll
      for (int k = 0; k < kLvItems; ++k) key[k] = k < nvalid ? words[pos0 + k] : 0ull;
    }
    const u64 prev = (pos0 > 0 && nvalid > 0) ? words[pos0 - 1] : 0ull;
    // unique reads / writes: heads of the full word; footprint: heads of word >> 1
    {
      u64 pw = prev;
#pragma unroll
      for (int k = 0; k < kLvItems; ++k) {
        if (k < nvalid) {
          const bool first = pos0 + k == 0;
          if (first || key[k] != pw) { if (key[k] & 1ull) ++uw; else ++ur; }
          if (first || (key[k] >> 1) != (pw >> 1)) ++heads0;
          pw = key[k];
        }
      }
    }
    for (int l = 0; l < kLevels; ++l) {
      const int shift = l + 1;
      tile_runs<kLvItems>(
          key, nvalid, pos0, prev, tile_n, [shift](u64 x) { return x >> shift; }, [](u64) { return 0ull; },
          [&](u64 len, u64) {
            if (len < (u64)kCocShared) atomicAdd(&coc[l][len], 1u);
            else if (len < (u64)kCocDense) atomicAdd(&a.arena->mem_coc[l][len], 1ull);
            else overflow_append(a.over, a.over_cap, st, l, len);
          },
          &a.tiles[(u64)l * a.ntiles + tile], sh, pre_slot);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kLevels * kCocShared; i += kLvThreads) {
    const u32 c = (&coc[0][0])[i];
    if (c) atomicAdd(&a.arena->mem_coc[i / kCocShared][i % kCocShared], (u64)c);
  }
  heads0 = block_reduce(heads0, OpAdd(), 0ull, red64);
  ur = block_reduce(ur, OpAdd(), 0ull, red64);
  uw = block_reduce(uw, OpAdd(), 0ull, red64);
  if (threadIdx.x == 0) {
    if (heads0) atomicAdd(&st->footprint, heads0);
    if (ur) atomicAdd(&st->unique_reads, ur);
    if (uw) atomicAdd(&st->unique_writes, uw);
  }
}

}  // namespace

void launch_mem_ingest(const MemIngestArgs& a, cudaStream_t s) {
  if (a.n == 0) return;
  const u64 per_block = (u64)kIngestThreads * (a.use_tab ? kHashItems : 8);
  const u64 cap = a.use_tab ? 152ull * 16 : 152ull * 8;
  auto grid = [&](u64 n) { return (unsigned)std::min<u64>((n + per_block - 1) / per_block, cap); };
  const bool filter = a.space_mask != 0xFu;
  if (filter) {
    if (a.use_tab) k_mem_ingest<true, true, false><<<grid(a.n), kIngestThreads, 0, s>>>(a);
    else k_mem_ingest<true, false, false><<<grid(a.n), kIngestThreads, 0, s>>>(a);
    count_launches(1);
    return;
  }
  // whole block tiles without bounds tests, then the ragged tail
  const u64 n_full = a.n / per_block * per_block;
  if (n_full) {
    MemIngestArgs f = a;
    f.n = n_full;
    if (a.use_tab) k_mem_ingest<false, true, true><<<grid(n_full), kIngestThreads, 0, s>>>(f);
    else k_mem_ingest<false, false, true><<<grid(n_full), kIngestThreads, 0, s>>>(f);
    count_launches(1);
  }
  if (a.n > n_full) {
    MemIngestArgs t = a;
    t.ev = static_cast<const char*>(a.ev) + 16 * n_full;
    t.n = a.n - n_full;
    t.word_base = a.word_base + n_full;
    if (a.use_tab) k_mem_ingest<false, true, false><<<grid(t.n), kIngestThreads, 0, s>>>(t);
    else k_mem_ingest<false, false, false><<<grid(t.n), kIngestThreads, 0, s>>>(t);
    count_launches(1);
  }
}

size_t expand_meta_bytes() {
  const size_t nt = (size_t)(kExpandChunk / kExpandTile);
  return nt * 8 + nt * 4;
}

void launch_expand_count(const ExpandArgs& a, cudaStream_t s) {
  if (a.n == 0) return;
  const u64 ntiles = (a.n + kExpandTile - 1) / kExpandTile;
  const unsigned g = (unsigned)std::min<u64>(ntiles, (u64)a.sm_count * 8);
  k_expand_count<<<g, kExpThreads, 0, s>>>(a);
  k_expand_scan<<<1, 1024, 0, s>>>(a);
  count_launches(2);
}

void launch_mem_ingest_bytes(const MemIngestArgs& a, const u64* tile_off, cudaStream_t s) {
  if (a.n == 0) return;
  const u64 ntiles = (a.n + kExpandTile - 1) / kExpandTile;
  const unsigned g = (unsigned)std::min<u64>(ntiles, a.use_tab ? 152ull * 16 : 152ull * 8);
  if (a.use_tab) k_mem_ingest_bytes<true><<<g, kIngestThreads, 0, s>>>(a, tile_off);
  else k_mem_ingest_bytes<false><<<g, kIngestThreads, 0, s>>>(a, tile_off);
  count_launches(1);
}

void launch_mem_levels(const LevelArgs& a, cudaStream_t s) {
  if (a.ntiles == 0) return;
  unsigned g = (unsigned)(a.grid < (int)a.ntiles ? a.grid : (int)a.ntiles);
  k_mem_levels<<<g, kLvThreads, 0, s>>>(a);
  count_launches(1);
}

}  // namespace aiwc
