// Branch path: per-site histories (Sec. III: 16-outcome histories; Sec. V:
// outcomes appended per branch location while work-items run one after
// another) and the average linear branch entropy of De Pestel et al.
//
// Branch word: (site << 32) | (work_item << 1) | taken. A stable sort by site
// (a counting sort when work-items arrive in order and site ids are small,
// else a radix sort on the varying bits 1..63) orders events by (site,
// work-item) and keeps push (program) order inside each work-item, which is
// the per-site history order. Per-site path: one block per site counts each
// h-outcome window's (taken, total) in shared-memory bins. Global path: a
// pattern word (site << 32) | (history << 1) | outcome is emitted for every
// outcome that has `h` predecessors in its history; sorting pattern words puts
// each (site, history) pattern in one run whose length is n and whose sum of
// low bits is the number taken, t. Either way M = sum min(t, n - t), N' = sum n.
#include <algorithm>

#include "aiwc_internal.cuh"
#include "common.cuh"
#include "runs.cuh"

namespace aiwc {
namespace {

constexpr int kBrThreads = 256;
constexpr int kBrItems = 8;

// Yokota entropy inputs: one pattern predicting n outcomes, one site
// predicting n outcomes (exact count-of-counts, dense below kValDense).
__device__ __forceinline__ void emit_pattern_count(u64 n, u64* over, u64 cap, Arena* ar) {
  if (n == 0) return;
  if (n < (u64)kValDense) atomicAdd(&ar->pat_coc[n], 1ull);
  else overflow_append(over, cap, &ar->st, kTagPat, n);
}
__device__ __forceinline__ void emit_site_pred_count(u64 n, u64* over, u64 cap, Arena* ar) {
  if (n == 0) return;
  if (n < (u64)kValDense) atomicAdd(&ar->site_pat_coc[n], 1ull);
  else overflow_append(over, cap, &ar->st, kTagSitePat, n);
}
// one history per site: a site with m outcomes predicts m - h of them
__device__ __forceinline__ void emit_site_predicted(u64 m, u32 h, u64* over, u64 cap, Arena* ar) {
  if (m > h) emit_site_pred_count(m - h, over, cap, ar);
}

__global__ void __launch_bounds__(kBrThreads, 4) k_branch_ingest(BranchIngestArgs a) {
  __shared__ u64 red64[32];
  __shared__ u32 red32[32];
  DevState* st = &a.arena->st;
  const uint2* ev = reinterpret_cast<const uint2*>(a.ev);
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  u64 wor = 0, wand = ~0ull;
  u32 wmin = 0xFFFFFFFFu, wmax = 0u, err = 0u, unsorted = 0u;
  const u64 per_block = (u64)kBrThreads * kBrItems;
  // each warp takes kBrItems consecutive groups of 32 events, so an event's
  // predecessor is the lane below, or lane 31 of the group before
  for (u64 t0 = (u64)blockIdx.x * per_block; t0 < a.n; t0 += (u64)gridDim.x * per_block) {
    const u64 w0 = t0 + (u64)wp * (32 * kBrItems);
    uint2 e[kBrItems];
#pragma unroll
    for (int k = 0; k < kBrItems; ++k) {
      const u64 i = w0 + (u64)k * 32 + lane;
      e[k] = i < a.n ? __ldcs(ev + i) : make_uint2(0u, 0u);
    }
    // the event before the warp's first
    u32 carry = 0;
    if (lane == 0 && w0 < a.n) {
      if (w0 > 0) carry = ev[w0 - 1].y & 0x7FFFFFFFu;
      else carry = a.push_index ? st->br_last_wi[(a.push_index - 1) & 1] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kBrItems; ++k) {
      const u64 i = w0 + (u64)k * 32 + lane;
      const bool valid = i < a.n;
      const u32 wi = e[k].y & 0x7FFFFFFFu;
      mark_work_items(a.wi_bitmap, a.max_wi, wi, valid, &err);
      // do work-item ids arrive in non-decreasing order?
      u32 prev = __shfl_up_sync(0xffffffffu, wi, 1);
      if (lane == 0) prev = carry;
      carry = __shfl_sync(0xffffffffu, wi, 31);  // for lane 0 of the next group (used by lane 0 only)
      if (valid) {
        if (wi < prev) unsorted = 1u;  // the first push's first event compares with 0
        if (i == a.n - 1) st->br_last_wi[a.push_index & 1] = wi;
        const u64 w = ((u64)e[k].x << 32) | ((u64)wi << 1) | (u64)(e[k].y >> 31);
        a.words[a.word_base + i] = w;
        // the counting sort by site reads two bytes per event instead of eight
        if (a.compact)
          a.compact[a.word_base + i] = e[k].x < kCsSites ? (uint16_t)((e[k].x << 1) | (e[k].y >> 31)) : (uint16_t)0xFFFFu;
        wor |= w;
        wand &= w;
        if ((u64)wi < a.max_wi) {
          wmin = min(wmin, wi);
          wmax = max(wmax, wi);
        }
      }
    }
  }
  wor = block_reduce(wor, OpOr(), 0ull, red64);
  wand = block_reduce(wand, OpAnd(), ~0ull, red64);
  wmin = block_reduce(wmin, OpMin(), 0xFFFFFFFFu, red32);
  wmax = block_reduce(wmax, OpMax(), 0u, red32);
  err = block_reduce(err, OpOr(), 0u, red32);
  unsorted = block_reduce(unsorted, OpOr(), 0u, red32);
  if (threadIdx.x == 0) {
    atomicOr(&st->br_or, wor);
    atomicAnd(&st->br_and, wand);
    if (wmin <= wmax) {
      atomicMin(&st->wi_min, wmin);
      atomicMax(&st->wi_max, wmax);
    }
    if (err) atomicOr(&st->err, err);
    if (unsorted) atomicOr(&st->br_unsorted, 1u);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&st->n_branch, a.n);
}

// Sites longer than kSiteMaxLen are counted in chunks when the long-site
// tables hold them all (and their 32-bit counters cannot overflow).
__global__ void k_persite_decide(Arena* arena, u32 h, u64 sites_cap, u64 long_cap, int allow) {
  DevState* st = &arena->st;
  const bool longs_fit = st->br_site_max <= kSiteMaxLen || (st->n_long <= long_cap && st->br_site_max < (1ull << 32));
  st->br_persite = (allow && h <= kSiteMaxHist && longs_fit && st->n_sites <= sites_cap) ? 1u : 0u;
}

// Lists each site's segment of the sorted branch words: (start, length).
__global__ void __launch_bounds__(256) k_site_heads(SiteArgs a) {
  DevState* st = &a.arena->st;
  const u64* w = *a.cur ? a.b : a.a;
  const u64 n = a.n;
  u64 mx = 0;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
    const u64 site = w[i] >> 32;
    if (i > 0 && (w[i - 1] >> 32) == site) continue;
    u64 lo = i + 1, hi = n;  // first position with a larger site
    while (lo < hi) {
      const u64 mid = (lo + hi) >> 1;
      if ((w[mid] >> 32) > site) hi = mid; else lo = mid + 1;
    }
    const u64 len = lo - i;
    mx = len > mx ? len : mx;
    if (len > kSiteMaxLen) atomicAdd(&st->n_long, 1ull);
    const u64 k = atomicAdd(&st->n_sites, 1ull);
    if (k < a.sites_cap) a.sites[k] = (i << 32) | len;  // a list exists only below 2^32 events
  }
  if (mx) atomicMax(&st->br_site_max, mx);
}

// ---------------------------------------------------------------- site counting sort

constexpr int kCsThreads = 256;
constexpr int kCsWarps = kCsThreads / 32;
// Tiles of 2^tile_shift events (14 or 15; each warp ranks an eighth, a
// contiguous run): the larger tile halves the per-site offsets and counts read
// and written per event, the smaller keeps two tiles per SM on mid-size
// sorts. Either stays below 2^16, the range of the per-warp site counters.
constexpr u32 kCsMaxShift = 15;
static_assert((1u << kCsMaxShift) < 65536, "the per-warp site counters are 16-bit halves");
constexpr int kCsChunk = 64;                            // tiles per scan chunk
constexpr int kCsScanThreads = 1024;
constexpr int kCsPer = kCsSites / kCsScanThreads;       // sites per scan thread (4)
static_assert(kCsPer == 4, "the scan reads four sites as one 16-byte vector");

__host__ __device__ inline u64 cs_tiles(u64 n, u32 shift) { return (n + (1ull << shift) - 1) >> shift; }
__host__ __device__ inline u64 cs_chunks(u64 n, u32 shift) { return (cs_tiles(n, shift) + kCsChunk - 1) / kCsChunk; }

// Phase 1: per-tile site counts, counts[tile][site].
__global__ void __launch_bounds__(kCsThreads) k_cs_count(SiteSortArgs a) {
  __shared__ u32 hist[kCsSites];
  const u64 ntiles = cs_tiles(a.n, a.tile_shift);
  for (u64 t = blockIdx.x; t < ntiles; t += gridDim.x) {
    for (int i = threadIdx.x; i < (int)kCsSites; i += kCsThreads) hist[i] = 0u;
    __syncthreads();
    const u64 base = t << a.tile_shift;
    const u64 end = umin64(a.n, base + (1ull << a.tile_shift));
    for (u64 i = base + threadIdx.x; i < end; i += kCsThreads)
      atomicAdd(&hist[a.src16 ? (u32)(a.src16[i] >> 1) : (u32)(a.src[i] >> 32)], 1u);
    __syncthreads();
    uint4* out = reinterpret_cast<uint4*>(a.counts + t * kCsSites);
    for (int i = threadIdx.x; i < (int)kCsSites / 4; i += kCsThreads)
      out[i] = make_uint4(hist[4 * i], hist[4 * i + 1], hist[4 * i + 2], hist[4 * i + 3]);
    __syncthreads();
  }
}

constexpr int kCs2Threads = 256;                           // phase 2 blocks
constexpr int kCs2Sites = kCs2Threads * 4;                 // sites per phase-2a block (four per thread)

// Phase 2a: within each chunk of kCsChunk tiles, counts become exclusive
// prefixes over the chunk's tiles; chunks[chunk][site] gets the chunk total.
// Blocks: (chunk, quarter of the sites).
__global__ void __launch_bounds__(kCs2Threads) k_cs_scan_chunks(SiteSortArgs a) {
  const u64 ntiles = cs_tiles(a.n, a.tile_shift), nchunks = cs_chunks(a.n, a.tile_shift);
  const u32 col = blockIdx.y * (kCs2Sites / 4) + threadIdx.x;  // uint4 column
  for (u64 c = blockIdx.x; c < nchunks; c += gridDim.x) {
    uint4 run = make_uint4(0u, 0u, 0u, 0u);
    const u64 t1 = umin64(ntiles, (c + 1) * kCsChunk);
    // eight tiles' counts in flight at a time
    for (u64 t0 = c * kCsChunk; t0 < t1; t0 += 8) {
      uint4 v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        v[q] = t0 + q < t1 ? reinterpret_cast<const uint4*>(a.counts + (t0 + q) * kCsSites)[col]
                           : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (t0 + q < t1) reinterpret_cast<uint4*>(a.counts + (t0 + q) * kCsSites)[col] = run;
        run.x += v[q].x; run.y += v[q].y; run.z += v[q].z; run.w += v[q].w;
      }
    }
    reinterpret_cast<uint4*>(a.chunks + c * kCsSites)[col] = run;
  }
}

// Phase 2b: per site (one per thread), exclusive prefix over the chunks and
// the site's total (in the words after the chunk rows).
__global__ void __launch_bounds__(kCs2Threads) k_cs_scan_site_chunks(SiteSortArgs a) {
  const u64 nchunks = cs_chunks(a.n, a.tile_shift);
  const u32 site = blockIdx.x * kCs2Threads + threadIdx.x;
  u32 run = 0;
  for (u64 c0 = 0; c0 < nchunks; c0 += 8) {
    u32 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = c0 + q < nchunks ? a.chunks[(c0 + q) * kCsSites + site] : 0u;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (c0 + q < nchunks) a.chunks[(c0 + q) * kCsSites + site] = run;
      run += v[q];
    }
  }
  a.chunks[nchunks * kCsSites + site] = run;  // site total
}

// Phase 2c (one block): each site's start (exclusive prefix of the totals),
// the site list, the number of sites and the longest site.
__global__ void __launch_bounds__(kCsScanThreads) k_cs_scan_sites(SiteSortArgs a) {
  __shared__ u64 wt64[33];
  __shared__ u32 wt32[33];
  __shared__ u64 red64[32];
  DevState* st = &a.arena->st;
  const u64 nchunks = cs_chunks(a.n, a.tile_shift);
  const u32* totals = a.chunks + nchunks * kCsSites;
  u32* starts = a.chunks + (nchunks + 1) * kCsSites;
  const uint4 tv = reinterpret_cast<const uint4*>(totals)[threadIdx.x];
  const u64 tot[kCsPer] = {tv.x, tv.y, tv.z, tv.w};
  // site starts: block exclusive scan of the per-thread sums (sites 4i .. 4i+3)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const u64 mine = tot[0] + tot[1] + tot[2] + tot[3];
  const u32 nz = (tot[0] != 0) + (tot[1] != 0) + (tot[2] != 0) + (tot[3] != 0);
  u64 inc = mine;
  u32 inz = nz;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u64 y = __shfl_up_sync(0xffffffffu, inc, o);
    const u32 yz = __shfl_up_sync(0xffffffffu, inz, o);
    if (lane >= o) { inc += y; inz += yz; }
  }
  if (lane == 31) { wt64[w] = inc; wt32[w] = inz; }
  __syncthreads();
  if (w == 0) {
    const u64 v = wt64[lane];
    const u32 vz = wt32[lane];
    u64 vi = v;
    u32 viz = vz;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const u64 y = __shfl_up_sync(0xffffffffu, vi, o);
      const u32 yz = __shfl_up_sync(0xffffffffu, viz, o);
      if (lane >= o) { vi += y; viz += yz; }
    }
    wt64[lane] = vi - v;
    wt32[lane] = viz - vz;
  }
  __syncthreads();
  u64 start = wt64[w] + inc - mine;
  u64 k = wt32[w] + inz - nz;
  u64 mx = 0, nl = 0;
  u32 sv[kCsPer];
#pragma unroll
  for (int q = 0; q < kCsPer; ++q) {
    sv[q] = (u32)start;
    nl += tot[q] > kSiteMaxLen;
    if (tot[q]) {
      if (k < a.sites_cap) a.sites[k] = (start << 32) | tot[q];
      ++k;
      mx = tot[q] > mx ? tot[q] : mx;
    }
    start += tot[q];
  }
  reinterpret_cast<uint4*>(starts)[threadIdx.x] = make_uint4(sv[0], sv[1], sv[2], sv[3]);
  mx = block_reduce(mx, OpMax(), 0ull, red64);
  nl = block_reduce(nl, OpAdd(), 0ull, red64);
  if (threadIdx.x == kCsScanThreads - 1) st->n_sites = k;  // the last thread's count is the total
  if (threadIdx.x == 0) {
    st->br_site_max = mx;
    st->n_long = nl;
    *a.sort_cur = 1u;
  }
}

// Phase 3: each warp ranks its 2048 events in push order among the tile's
// events of the same site (per-warp 16-bit counters, two sites per word,
// turned into prefixes over the warps) and writes each word to its site's
// position: chunk offset + prefix within the chunk + rank within the tile.
constexpr size_t kCsScatterSmem = (size_t)(kCsWarps * kCsSites / 2 + kCsSites) * 4;

template <bool OUT8>
__global__ void __launch_bounds__(kCsThreads) k_cs_scatter(SiteSortArgs a) {
  extern __shared__ u32 csm[];
  u32 (*wc)[kCsSites / 2] = reinterpret_cast<u32 (*)[kCsSites / 2]>(csm);
  u32* toff = csm + kCsWarps * kCsSites / 2;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const u32 lt = (1u << lane) - 1u;
  const u64 ntiles = cs_tiles(a.n, a.tile_shift);
  for (u64 t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const u32* cc = a.chunks + (t / kCsChunk) * kCsSites;
    const u32* ct = a.counts + t * kCsSites;
    const u32* cs = a.chunks + (cs_chunks(a.n, a.tile_shift) + 1) * kCsSites;  // site starts
    for (int i = threadIdx.x; i < (int)kCsSites; i += kCsThreads) toff[i] = cs[i] + cc[i] + ct[i];
    for (int i = threadIdx.x; i < kCsWarps * (int)kCsSites / 2; i += kCsThreads) (&wc[0][0])[i] = 0u;
    __syncthreads();
    const u64 warp_events = 1ull << (a.tile_shift - 3);  // kCsWarps = 8 runs per tile
    const u64 w0 = (t << a.tile_shift) + (u64)wp * warp_events;
    const u64 w1 = umin64(a.n, w0 + warp_events);
    {
      u64 i = w0 + lane;
      for (; i + 96 < w1; i += 128) {  // four loads in flight
        u32 st4[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) st4[q] = OUT8 ? (u32)(a.src16[i + 32 * q] >> 1) : (u32)(a.src[i + 32 * q] >> 32);
#pragma unroll
        for (int q = 0; q < 4; ++q) atomicAdd(&wc[wp][st4[q] >> 1], 1u << ((st4[q] & 1u) * 16));
      }
      for (; i < w1; i += 32) {
        const u32 site = OUT8 ? (u32)(a.src16[i] >> 1) : (u32)(a.src[i] >> 32);
        atomicAdd(&wc[wp][site >> 1], 1u << ((site & 1u) * 16));
      }
    }
    __syncthreads();
    // prefixes over the warps, one site pair per thread at a time
    for (int pr = threadIdx.x; pr < (int)kCsSites / 2; pr += kCsThreads) {
      u32 run = 0;
#pragma unroll
      for (int q = 0; q < kCsWarps; ++q) {
        const u32 c = wc[q][pr];
        wc[q][pr] = run;
        run += c;  // both halves stay below 2^16: a tile has at most 32768 events
      }
    }
    __syncthreads();
    // push order is kept: groups of 32 events are ranked one after another,
    // while the loads of the next groups are already in flight
    for (u64 i0 = w0; i0 < w1; i0 += 128) {
      u64 word[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const u64 i = i0 + 32 * q + lane;
        // OUT8: the compact record in the word's place, site above bit 32 and the outcome in bit 0
        word[q] = i < w1 ? (OUT8 ? (((u64)(a.src16[i] >> 1) << 32) | (a.src16[i] & 1u)) : a.src[i]) : 0ull;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bool v = i0 + 32 * q + lane < w1;
        const u32 site = (u32)(word[q] >> 32);
        const u32 peers = __match_any_sync(0xffffffffu, v ? site : (0xFFFFF000u | (u32)lane));
        const int leader = __ffs(peers) - 1;
        u32 b = 0;
        if (v && lane == leader) {
          const u32 sh = (site & 1u) * 16;
          b = (atomicAdd(&wc[wp][site >> 1], (u32)__popc(peers) << sh) >> sh) & 0xFFFFu;
        }
        b = __shfl_sync(0xffffffffu, b, leader);
        const u64 pos = (u64)toff[site] + b + (u32)__popc(peers & lt);
        if (v) {
          if (OUT8) a.dst8[pos] = (uint8_t)(word[q] & 1ull);
          else a.dst[pos] = word[q];
        }
      }
    }
    __syncthreads();
  }
}

constexpr int kSpThreads = 1024;
constexpr int kPatSmem = 1024;  // pattern counts below this are counted in shared memory first
constexpr int kSpBinsLog = 15;
constexpr int kSpBitWords = (int)((kSiteMaxLen + 32) / 32) + 2;
constexpr u32 kLongChunk = 16384;  // predicted outcomes of a long site per block work item

// Shared memory of the window-counting kernels: the outcome bit string, the
// work-item change bit string, 2^kSpBinsLog packed counters (total in the low
// 16 bits, taken in the high 16) and the list of the bins a pass used.
struct WinSmem {
  u32* bits;
  u32* brk;
  u32* cnt;
  uint16_t* used;
  u32* n_used;
};

__device__ __forceinline__ WinSmem win_smem(u32* spm, u32* n_used) {
  WinSmem s;
  s.bits = spm;
  s.brk = spm + kSpBitWords;
  s.cnt = spm + 2 * kSpBitWords;
  s.used = reinterpret_cast<uint16_t*>(s.cnt + (1 << kSpBinsLog));
  s.n_used = n_used;
  return s;
}

// Counts the windows of the outcome positions [b0, e) of one site (positions
// relative to the site, whose words or outcome bytes start at `start`): each
// position j in [j0, e), j0 >= b0 + h, is counted under its history, the h
// outcomes before it. The positions become a bit string in shared memory;
// the packed counter of j's history gets +1 total and +outcome taken.
// Histories are binned 2^15 at a time (more passes for h > 15); the first
// increment of a bin lists it, and after each pass flush(pattern, counter)
// is called once for every bin the pass used, which is then cleared. Any
// fixed bijection of the h-bit window names the pattern equally well; here
// bit k of the pattern is the outcome k+1 places after the oldest. With one
// history per (site, work-item) a second bit string marks where the
// work-item changes (the words are sorted by work-item within a site); a
// window counts only when no change falls inside it, and the return value
// is this thread's number of such windows. Called by the whole block, which
// it leaves synchronised.
template <typename Flush>
__device__ __forceinline__ u64 count_windows(const SiteArgs& a, const u64* w, u64 start, u64 b0, u64 j0, u64 e,
                                             const WinSmem& sm, Flush&& flush) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = kSpThreads / 32;
  const u32 h = a.h;
  const int pbits = h > (u32)kSpBinsLog ? kSpBinsLog : (int)h;
  const u32 nbins = 1u << pbits;
  const u32 passes = h > (u32)kSpBinsLog ? (1u << (h - kSpBinsLog)) : 1u;
  const u64 hmask = (1ull << h) - 1ull;
  const u64 len = e - b0;
  const u32 nwords = (u32)((len + 31) / 32);
  // eight 32-position groups per warp in flight at a time
  for (u32 c0 = wp; c0 < nwords + 2; c0 += 8 * nw) {
    bool t[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const u64 l = (u64)(c0 + q * nw) * 32 + lane;
      t[q] = l < len && (a.outcomes ? (a.outcomes[start + b0 + l] & 1u) : (w[start + b0 + l] & 1ull));
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const u32 b = __ballot_sync(0xffffffffu, t[q]);
      if (lane == 0 && c0 + q * nw < nwords + 2) sm.bits[c0 + q * nw] = b;
    }
    if (a.per_wi) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const u64 l = (u64)(c0 + q * nw) * 32 + lane;
        const u64 p = b0 + l;
        const bool change = l < len && p > 0 && (w[start + p] >> 1) != (w[start + p - 1] >> 1);
        const u32 b = __ballot_sync(0xffffffffu, change);
        if (lane == 0 && c0 + q * nw < nwords + 2) sm.brk[c0 + q * nw] = b;
      }
    }
  }
  __syncthreads();
  u64 spred = 0;
  for (u32 q = 0; q < passes; ++q) {
    for (u64 j = j0 + threadIdx.x; j < e; j += kSpThreads) {
      const u64 jl = j - b0, pos = jl - h;
      const u64 two = (u64)sm.bits[pos >> 5] | ((u64)sm.bits[(pos >> 5) + 1] << 32);
      const u32 win = (u32)((two >> (pos & 31)) & hmask);
      const u32 outcome = (sm.bits[jl >> 5] >> (jl & 31)) & 1u;
      if (a.per_wi) {
        // work-item changes at positions pos + 1 .. jl end the window's history
        const u64 p1 = pos + 1;
        const u64 tb = (u64)sm.brk[p1 >> 5] | ((u64)sm.brk[(p1 >> 5) + 1] << 32);
        if ((tb >> (p1 & 31)) & hmask) continue;
        if (q == 0) ++spred;
      }
      if ((win >> pbits) == q) {
        const u32 b = win & (nbins - 1);
        if (atomicAdd(&sm.cnt[b], 1u + (outcome << 16)) == 0u) sm.used[atomicAdd(sm.n_used, 1u)] = (uint16_t)b;
      }
    }
    __syncthreads();
    const u32 nu = *sm.n_used;
    for (u32 i = threadIdx.x; i < nu; i += kSpThreads) {
      const u32 b = sm.used[i];
      const u32 v = sm.cnt[b];
      sm.cnt[b] = 0u;
      flush((q << pbits) | b, v);
    }
    __syncthreads();
    if (threadIdx.x == 0) *sm.n_used = 0;
    __syncthreads();
  }
  return spred;
}

// One block per site of at most kSiteMaxLen outcomes (longer ones are
// counted in chunks, below): every window of the site is counted in shared
// memory, and M and N' follow from the bins.
__global__ void __launch_bounds__(kSpThreads) k_site_patterns(SiteArgs a) {
  if (!gate_open(a.gate, a.gate_want)) return;
  extern __shared__ u32 spm[];
  __shared__ u32 n_used;
  __shared__ u64 red64[32];
  __shared__ u32 pcoc[kPatSmem];  // pattern count-of-counts for small counts
  const WinSmem sm = win_smem(spm, &n_used);
  DevState* st = &a.arena->st;
  if (blockIdx.x >= umin64(st->n_sites, a.sites_cap)) return;  // no site for this block
  const u64* w = *a.cur ? a.b : a.a;
  for (int i = threadIdx.x; i < kPatSmem; i += kSpThreads) pcoc[i] = 0u;
  for (int i = threadIdx.x; i < (1 << kSpBinsLog); i += kSpThreads) sm.cnt[i] = 0u;
  if (threadIdx.x == 0) n_used = 0;
  __syncthreads();
  const u32 h = a.h;
  const u64 n_sites = umin64(st->n_sites, a.sites_cap);
  u64 msum = 0, nsum = 0, nsite = 0;
  for (u64 si = blockIdx.x; si < n_sites; si += gridDim.x) {
    const u64 start = a.sites[si] >> 32, m = a.sites[si] & 0xFFFFFFFFull;
    if (m > kSiteMaxLen) continue;
    if (threadIdx.x == 0) {
      ++nsite;
      if (m < (u64)kCocDense) atomicAdd(&a.arena->site_coc[m], 1ull);
      else overflow_append(a.over, a.over_cap, st, kTagSites, m);
      if (!a.per_wi) emit_site_predicted(m, h, a.over, a.over_cap, a.arena);
    }
    u64 spred = count_windows(a, w, start, 0, h, m, sm, [&](u32, u32 v) {
      const u32 nn = v & 0xFFFFu, t = v >> 16;
      msum += t < nn - t ? t : nn - t;
      nsum += nn;
      if (nn < (u32)kPatSmem) atomicAdd(&pcoc[nn], 1u);
      else atomicAdd(&a.arena->pat_coc[nn], 1ull);  // nn <= kSiteMaxLen < kValDense
    });
    if (a.per_wi) {
      spred = block_reduce(spred, OpAdd(), 0ull, red64);
      if (threadIdx.x == 0) emit_site_pred_count(spred, a.over, a.over_cap, a.arena);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kPatSmem; i += kSpThreads)
    if (pcoc[i]) atomicAdd(&a.arena->pat_coc[i], (u64)pcoc[i]);
  msum = block_reduce(msum, OpAdd(), 0ull, red64);
  nsum = block_reduce(nsum, OpAdd(), 0ull, red64);
  nsite = block_reduce(nsite, OpAdd(), 0ull, red64);
  if (threadIdx.x == 0) {
    if (msum) atomicAdd(&st->minsum, msum);
    if (nsum) atomicAdd(&st->npat, nsum);
    if (nsite) atomicAdd(&st->branch_sites, nsite);
  }
}

// Sites longer than kSiteMaxLen (a chunk's counters still fit 16 bits, a
// site's may not): k_long_prep lists them and clears their tables,
// k_site_chunks counts each chunk of kLongChunk predicted outcomes as above
// and adds its bins to the site's dense table of 2^h (taken << 32 | total)
// counters, and k_long_walk takes M, N' and the pattern counts from the
// tables, one block per site. The chunks partition the site's predicted
// outcomes, so every (site, history) count is the same sum as in one pass.
__global__ void __launch_bounds__(256) k_long_prep(SiteArgs a) {
  if (!gate_open(a.gate, a.gate_want)) return;
  DevState* st = &a.arena->st;
  const u64 n_sites = umin64(st->n_sites, a.sites_cap);
  const u64 n_long = umin64(st->n_long, a.long_cap);
  const u64 tid = (u64)blockIdx.x * blockDim.x + threadIdx.x, nt = (u64)gridDim.x * blockDim.x;
  for (u64 i = tid; i < n_sites; i += nt) {
    const u64 m = a.sites[i] & 0xFFFFFFFFull;
    if (m > kSiteMaxLen) {
      const u64 k = atomicAdd(&st->long_next, 1ull);
      if (k < a.long_cap) {
        a.long_list[3 * k] = a.sites[i] >> 32;
        a.long_list[3 * k + 1] = m;
        a.long_list[3 * k + 2] = 0ull;
      }
    }
  }
  ulonglong2* t2 = reinterpret_cast<ulonglong2*>(a.long_tab);
  const u64 pairs = (n_long << a.h) / 2;  // h >= 1
  for (u64 i = tid; i < pairs; i += nt) t2[i] = make_ulonglong2(0ull, 0ull);
}

// Chunk q of long site i goes to block (chunks of the sites before i + q)
// mod gridDim.x.
__global__ void __launch_bounds__(kSpThreads) k_site_chunks(SiteArgs a) {
  if (!gate_open(a.gate, a.gate_want)) return;
  extern __shared__ u32 spm[];
  __shared__ u32 n_used;
  __shared__ u64 red64[32];
  const WinSmem sm = win_smem(spm, &n_used);
  DevState* st = &a.arena->st;
  const u64* w = *a.cur ? a.b : a.a;
  const u32 h = a.h;
  const u64 n_long = umin64(umin64(st->n_long, st->long_next), a.long_cap);  // the listed ones
  const u64 G = gridDim.x;
  {
    u64 chunks = 0;
    for (u64 i = 0; i < n_long; ++i) chunks += (a.long_list[3 * i + 1] + kLongChunk - 1) / kLongChunk;
    if (blockIdx.x >= chunks) return;  // no chunk for this block
  }
  for (int i = threadIdx.x; i < (1 << kSpBinsLog); i += kSpThreads) sm.cnt[i] = 0u;
  if (threadIdx.x == 0) n_used = 0;
  __syncthreads();
  u64 qbase = 0;
  for (u64 i = 0; i < n_long; ++i) {
    const u64 start = a.long_list[3 * i], m = a.long_list[3 * i + 1];
    const u64 nch = (m + kLongChunk - 1) / kLongChunk;
    u64* tab = a.long_tab + (i << h);
    u64 spred = 0;
    for (u64 q = (blockIdx.x + G - qbase % G) % G; q < nch; q += G) {
      const u64 c0 = q * kLongChunk, e = umin64(m, c0 + kLongChunk);
      const u64 j0 = c0 > (u64)h ? c0 : (u64)h;
      spred += count_windows(a, w, start, j0 - h, j0, e, sm, [&](u32 pat, u32 v) {
        atomicAdd(&tab[pat], ((u64)(v >> 16) << 32) | (u64)(v & 0xFFFFu));
      });
    }
    if (a.per_wi) {
      spred = block_reduce(spred, OpAdd(), 0ull, red64);
      if (threadIdx.x == 0 && spred) atomicAdd(&a.long_list[3 * i + 2], spred);
    }
    qbase += nch;
  }
}

constexpr int kLwThreads = 1024;

__global__ void __launch_bounds__(kLwThreads) k_long_walk(SiteArgs a) {
  if (!gate_open(a.gate, a.gate_want)) return;
  __shared__ u64 red64[32];
  __shared__ u32 pcoc[kPatSmem];
  DevState* st = &a.arena->st;
  const u32 h = a.h;
  const u64 n_long = umin64(umin64(st->n_long, st->long_next), a.long_cap);
  if (blockIdx.x >= n_long) return;
  for (int i = threadIdx.x; i < kPatSmem; i += kLwThreads) pcoc[i] = 0u;
  __syncthreads();
  u64 msum = 0, nsum = 0, nsite = 0;
  for (u64 i = blockIdx.x; i < n_long; i += gridDim.x) {
    const u64 m = a.long_list[3 * i + 1];
    if (threadIdx.x == 0) {
      ++nsite;
      if (m < (u64)kCocDense) atomicAdd(&a.arena->site_coc[m], 1ull);
      else overflow_append(a.over, a.over_cap, st, kTagSites, m);
      if (a.per_wi) emit_site_pred_count(a.long_list[3 * i + 2], a.over, a.over_cap, a.arena);
      else emit_site_predicted(m, h, a.over, a.over_cap, a.arena);
    }
    const ulonglong2* tab = reinterpret_cast<const ulonglong2*>(a.long_tab + (i << h));
    for (u32 b = threadIdx.x; b < (1u << h) / 2; b += kLwThreads) {
      const ulonglong2 v2 = tab[b];
      const u64 v[2] = {v2.x, v2.y};
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        if (!v[k]) continue;
        const u64 nn = v[k] & 0xFFFFFFFFull, t = v[k] >> 32;
        msum += umin64(t, nn - t);
        nsum += nn;
        if (nn < (u64)kPatSmem) atomicAdd(&pcoc[nn], 1u);
        else emit_pattern_count(nn, a.over, a.over_cap, a.arena);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kPatSmem; i += kLwThreads)
    if (pcoc[i]) atomicAdd(&a.arena->pat_coc[i], (u64)pcoc[i]);
  msum = block_reduce(msum, OpAdd(), 0ull, red64);
  nsum = block_reduce(nsum, OpAdd(), 0ull, red64);
  nsite = block_reduce(nsite, OpAdd(), 0ull, red64);
  if (threadIdx.x == 0) {
    if (msum) atomicAdd(&st->minsum, msum);
    if (nsum) atomicAdd(&st->npat, nsum);
    if (nsite) atomicAdd(&st->branch_sites, nsite);
  }
}

constexpr int kHalo = 32;  // history lengths are at most 31

// Reads the sorted branch words of one tile (plus the 32 words before it),
// writes the compacted pattern words of outcomes with a full history, and
// runs the per-site run lengths (site event counts) for the site metrics.
// An outcome has a full history when the word h places before it belongs to
// the same history: the same site, or with per-(site, work-item) histories
// the same site and work-item (gshift 1; the sort keeps each work-item's
// outcomes at a site together, in program order).
__global__ void __launch_bounds__(kTileThreads) k_windows(WindowArgs a) {
  if (!gate_open(a.gate, a.gate_want)) return;
  __shared__ u64 tw[kHalo + kTile];
  __shared__ u32 site_coc[kCocShared];
  __shared__ Seg sh[33];
  __shared__ u64 pre_slot[2];
  __shared__ u64 red64[32];
  __shared__ u32 scan_tot[33];
  __shared__ u64 s_base;
  DevState* st = &a.arena->st;
  for (int i = threadIdx.x; i < kCocShared; i += kTileThreads) site_coc[i] = 0u;
  const u64 n = a.n;
  const u64* words = *a.cur ? a.b : a.a;
  const u32 ntiles = (u32)((n + kTile - 1) / kTile);
  const u32 h = a.h;
  const u64 hmask = (1ull << h) - 1ull;
  u64 heads = 0, npat = 0, por = 0, pand = ~0ull;
  for (u32 tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const u64 base = (u64)tile * kTile;
    const u64 tile_n = umin64(n - base, (u64)kTile);
    __syncthreads();
    for (int i = threadIdx.x; i < kHalo + kTile; i += kTileThreads) {
      const long long p = (long long)base - kHalo + i;
      tw[i] = (p >= 0 && (u64)p < n) ? words[p] : 0ull;
    }
    __syncthreads();
    const int t0 = threadIdx.x * kTileItems;  // tile-relative
    const u64 pos0 = base + t0;
    const int nvalid = pos0 < n ? (int)umin64(n - pos0, (u64)kTileItems) : 0;
    u64 key[kTileItems];
#pragma unroll
    for (int k = 0; k < kTileItems; ++k) key[k] = tw[kHalo + t0 + k];
    const u64 prev = tw[kHalo + t0 - 1];
    // history of the first position: outcomes at pos0-h .. pos0-1, oldest high
    u64 hist = 0;
    for (u32 i = 0; i < h; ++i) hist = (hist << 1) | (tw[kHalo + t0 - (int)h + (int)i] & 1ull);
    u64 pat[kTileItems];
    u32 np = 0;
#pragma unroll
    for (int k = 0; k < kTileItems; ++k) {
      const u64 j = pos0 + k;
      bool ok = false;
      if (k < nvalid && j >= h) {
        const u64 older = tw[kHalo + t0 + k - (int)h];
        ok = (older >> a.gshift) == (key[k] >> a.gshift);
      }
      if (ok) {
        const u64 pw = (key[k] & 0xFFFFFFFF00000001ull) | ((hist & hmask) << 1);
        pat[np++] = pw;
        por |= pw;
        pand &= pw;
      }
      hist = (hist << 1) | (key[k] & 1ull);
    }
    npat += np;
    // compact this tile's pattern words behind one atomicAdd
    {
      const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
      u32 inc = np;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        u32 y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      if (lane == 31) scan_tot[w] = inc;
      __syncthreads();
      if (threadIdx.x == 0) {
        u32 s = 0;
        for (int q = 0; q < kTileThreads / 32; ++q) { u32 c = scan_tot[q]; scan_tot[q] = s; s += c; }
        s_base = atomicAdd(&st->n_patterns, (u64)s);
      }
      __syncthreads();
      u64 out = s_base + scan_tot[w] + inc - np;
      for (u32 k = 0; k < np; ++k) a.patterns[out + k] = pat[k];
    }
    // site heads and per-site event counts
    {
      u64 pw = prev;
#pragma unroll
      for (int k = 0; k < kTileItems; ++k) {
        if (k < nvalid) {
          if (pos0 + k == 0 || (key[k] >> 32) != (pw >> 32)) ++heads;
          pw = key[k];
        }
      }
    }
    tile_runs<kTileItems>(
        key, nvalid, pos0, prev, tile_n, [](u64 x) { return x >> 32; }, [](u64) { return 0ull; },
        [&](u64 len, u64) {
          if (len < (u64)kCocShared) atomicAdd(&site_coc[len], 1u);
          else if (len < (u64)kCocDense) atomicAdd(&a.arena->site_coc[len], 1ull);
          else overflow_append(a.over, a.over_cap, st, kTagSites, len);
          if (a.site_pred) emit_site_predicted(len, h, a.over, a.over_cap, a.arena);
        },
        &a.tiles[tile], sh, pre_slot);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kCocShared; i += kTileThreads)
    if (site_coc[i]) atomicAdd(&a.arena->site_coc[i], (u64)site_coc[i]);
  heads = block_reduce(heads, OpAdd(), 0ull, red64);
  por = block_reduce(por, OpOr(), 0ull, red64);
  pand = block_reduce(pand, OpAnd(), ~0ull, red64);
  npat = block_reduce(npat, OpAdd(), 0ull, red64);
  if (threadIdx.x == 0) {
    if (heads) atomicAdd(&st->branch_sites, heads);
    if (npat) {
      atomicOr(&st->pat_or, por);
      atomicAnd(&st->pat_and, pand);
    }
  }
}

__global__ void __launch_bounds__(kTileThreads) k_pattern_runs(PatternArgs a) {
  if (!gate_open(a.gate, a.gate_want)) return;
  __shared__ Seg sh[33];
  __shared__ u64 pre_slot[2];
  __shared__ u64 red64[32];
  __shared__ u32 pcoc[kPatSmem];
  DevState* st = &a.arena->st;
  for (int i = threadIdx.x; i < kPatSmem; i += kTileThreads) pcoc[i] = 0u;
  __syncthreads();
  const u64 n = *a.n;
  const u64* words = *a.cur ? a.b : a.a;
  const u32 ntiles = (u32)((n + kTile - 1) / kTile);
  u64 msum = 0, nsum = 0;
  for (u32 tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const u64 base = (u64)tile * kTile;
    const u64 pos0 = base + (u64)threadIdx.x * kTileItems;
    const int nvalid = pos0 < n ? (int)umin64(n - pos0, (u64)kTileItems) : 0;
    const u64 tile_n = umin64(n - base, (u64)kTile);
    u64 key[kTileItems];
#pragma unroll
    for (int k = 0; k < kTileItems; ++k) key[k] = k < nvalid ? words[pos0 + k] : 0ull;
    const u64 prev = (pos0 > 0 && nvalid > 0) ? words[pos0 - 1] : 0ull;
    tile_runs<kTileItems>(
        key, nvalid, pos0, prev, tile_n, [](u64 x) { return x >> 1; }, [](u64 x) { return x & 1ull; },
        [&](u64 len, u64 t) {
          msum += umin64(t, len - t);
          nsum += len;
          if (len < (u64)kPatSmem) atomicAdd(&pcoc[len], 1u);
          else emit_pattern_count(len, a.over, a.over_cap, a.arena);
        },
        &a.tiles[tile], sh, pre_slot);
    if (a.site_level)
      tile_runs<kTileItems>(
          key, nvalid, pos0, prev, tile_n, [](u64 x) { return x >> 32; }, [](u64) { return 0ull; },
          [&](u64 len, u64) { emit_site_pred_count(len, a.over, a.over_cap, a.arena); },
          &a.tiles[a.ntiles + tile], sh, pre_slot);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kPatSmem; i += kTileThreads)
    if (pcoc[i]) atomicAdd(&a.arena->pat_coc[i], (u64)pcoc[i]);
  msum = block_reduce(msum, OpAdd(), 0ull, red64);
  nsum = block_reduce(nsum, OpAdd(), 0ull, red64);
  if (threadIdx.x == 0) {
    if (msum) atomicAdd(&st->minsum, msum);
    if (nsum) atomicAdd(&st->npat, nsum);
  }
}

// Cross-tile fix-up: one block per level walks that level's tile summaries
// in chunks with a segmented scan and emits every run that crosses a tile
// boundary (and the final run), exactly once. KIND 0: memory levels; 1: site
// runs (h = 0: no per-site predicted counts); 2: level 0 pattern runs, level 1
// site runs of the pattern words.
template <int KIND>
__global__ void __launch_bounds__(1024) k_fixup(const TileSum* tiles, u32 ntiles_max, const u64* n_dev, u64 n_host,
                                                u64* over, u64 over_cap, Arena* arena, const u32* gate, u32 want,
                                                u32 h) {
  if (!gate_open(gate, want)) return;
  __shared__ Seg sh[33];
  __shared__ u64 red64[32];
  DevState* st = &arena->st;
  const int level = blockIdx.x;
  const u64 n = n_dev ? *n_dev : n_host;
  const u32 ntiles = (u32)((n + kTile - 1) / kTile);
  const TileSum* ts = tiles + (u64)level * ntiles_max;
  Seg carry = seg_identity();
  u64 msum = 0, nsum = 0;
  auto emit = [&](u64 len, u64 wsum) {
    if (KIND == 0) {
      if (len < (u64)kCocDense) atomicAdd(&arena->mem_coc[level][len], 1ull);
      else overflow_append(over, over_cap, st, level, len);
    } else if (KIND == 1) {
      if (len < (u64)kCocDense) atomicAdd(&arena->site_coc[len], 1ull);
      else overflow_append(over, over_cap, st, kTagSites, len);
      if (h) emit_site_predicted(len, h, over, over_cap, arena);
    } else if (level == 0) {
      msum += umin64(wsum, len - wsum);
      nsum += len;
      emit_pattern_count(len, over, over_cap, arena);
    } else {
      emit_site_pred_count(len, over, over_cap, arena);
    }
  };
  for (u32 c0 = 0; c0 < ntiles; c0 += blockDim.x) {
    const u32 t = c0 + threadIdx.x;
    Seg e = seg_identity();
    TileSum s;
    if (t < ntiles) {
      s = ts[t];
      e.b = s.has_b;
      e.v = s.has_b ? s.suf : s.tot;
      e.w = s.has_b ? s.suf_w : s.tot_w;
    }
    Seg agg;
    Seg ex = block_seg_scan(e, &agg, sh);
    ex = seg_op(carry, ex);
    if (t < ntiles && s.has_b && ex.b) emit(ex.v + s.pre, ex.w + s.pre_w);
    carry = seg_op(carry, agg);
  }
  if (threadIdx.x == 0 && carry.b) emit(carry.v, carry.w);
  if (KIND == 2) {
    msum = block_reduce(msum, OpAdd(), 0ull, red64);
    nsum = block_reduce(nsum, OpAdd(), 0ull, red64);
    if (threadIdx.x == 0) {
      if (msum) atomicAdd(&st->minsum, msum);
      if (nsum) atomicAdd(&st->npat, nsum);
    }
  }
}

}  // namespace

void launch_branch_ingest(const BranchIngestArgs& a, cudaStream_t s) {
  if (a.n == 0) return;
  const u64 per_block = (u64)kBrThreads * kBrItems;
  u64 blocks = (a.n + per_block - 1) / per_block;
  if (blocks > 152ull * 8) blocks = 152ull * 8;
  k_branch_ingest<<<(unsigned)blocks, kBrThreads, 0, s>>>(a);
  count_launches(1);
}

// Sized for the smaller tile, which has more of them.
size_t site_sort_count_words(u64 n) { return (size_t)(cs_tiles(n, 14) ? cs_tiles(n, 14) : 1) * kCsSites; }
size_t site_sort_chunk_words(u64 n) { return (size_t)(cs_chunks(n, 14) + 2) * kCsSites; }  // + totals, starts
u32 site_sort_tile_shift(u64 n, int sm_count) { return cs_tiles(n, kCsMaxShift) >= 2ull * (u64)sm_count ? 15u : 14u; }

void launch_site_sort_count(const SiteSortArgs& a, cudaStream_t s) {
  if (a.n == 0) return;
  const u64 ntiles = cs_tiles(a.n, a.tile_shift), nchunks = cs_chunks(a.n, a.tile_shift);
  k_cs_count<<<(unsigned)std::min<u64>(ntiles, (u64)a.sm_count * 8), kCsThreads, 0, s>>>(a);
  k_cs_scan_chunks<<<dim3((unsigned)nchunks, kCsSites / kCs2Sites), kCs2Threads, 0, s>>>(a);
  k_cs_scan_site_chunks<<<kCsSites / kCs2Threads, kCs2Threads, 0, s>>>(a);
  k_cs_scan_sites<<<1, kCsScanThreads, 0, s>>>(a);
  count_launches(4);
}

void launch_site_sort_scatter(const SiteSortArgs& a, cudaStream_t s) {
  if (a.n == 0) return;
  const unsigned g = (unsigned)std::min<u64>(cs_tiles(a.n, a.tile_shift), (u64)a.sm_count * 2);
  if (a.dst8) k_cs_scatter<true><<<g, kCsThreads, kCsScatterSmem, s>>>(a);
  else k_cs_scatter<false><<<g, kCsThreads, kCsScatterSmem, s>>>(a);
  count_launches(1);
}

void launch_site_heads(const SiteArgs& a, cudaStream_t s) {
  if (a.n == 0) return;
  u64 blocks = (a.n + 255) / 256;
  if (blocks > (u64)a.grid * 4) blocks = (u64)a.grid * 4;
  k_site_heads<<<(unsigned)blocks, 256, 0, s>>>(a);
  count_launches(1);
}

void launch_persite_decide(Arena* arena, u32 h, u64 sites_cap, u64 long_cap, int allow, cudaStream_t s) {
  k_persite_decide<<<1, 1, 0, s>>>(arena, h, sites_cap, long_cap, allow);
  count_launches(1);
}

static size_t site_patterns_smem() {
  return (size_t)(2 * kSpBitWords + (1 << kSpBinsLog)) * 4 + (size_t)(1 << kSpBinsLog) * 2;
}

void init_branch_attributes() {
  cudaFuncSetAttribute(k_site_patterns, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)site_patterns_smem());
  cudaFuncSetAttribute(k_site_chunks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)site_patterns_smem());
  cudaFuncSetAttribute(k_cs_scatter<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCsScatterSmem);
  cudaFuncSetAttribute(k_cs_scatter<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCsScatterSmem);
}

void launch_site_patterns(const SiteArgs& a, cudaStream_t s) {
  k_site_patterns<<<a.grid, kSpThreads, site_patterns_smem(), s>>>(a);
  count_launches(1);
}

void launch_site_long(const SiteArgs& a, cudaStream_t s) {
  k_long_prep<<<a.grid, 256, 0, s>>>(a);
  k_site_chunks<<<a.grid, kSpThreads, site_patterns_smem(), s>>>(a);
  k_long_walk<<<a.grid, kLwThreads, 0, s>>>(a);
  count_launches(3);
}

void launch_branch_windows(const WindowArgs& a, cudaStream_t s) {
  if (a.ntiles == 0) return;
  unsigned g = (unsigned)(a.grid < (int)a.ntiles ? a.grid : (int)a.ntiles);
  k_windows<<<g, kTileThreads, 0, s>>>(a);
  count_launches(1);
}

void launch_pattern_runs(const PatternArgs& a, cudaStream_t s) {
  if (a.ntiles == 0) return;
  unsigned g = (unsigned)(a.grid < (int)a.ntiles ? a.grid : (int)a.ntiles);
  k_pattern_runs<<<g, kTileThreads, 0, s>>>(a);
  count_launches(1);
}

void launch_runs_fixup(int kind, const TileSum* tiles, u32 ntiles_max, const u64* n_dev, u64 n_host, int levels,
                       u64* over, u64 over_cap, Arena* arena, cudaStream_t s, const u32* gate, u32 gate_want, u32 h) {
  if (ntiles_max == 0) return;
  if (kind == 0)
    k_fixup<0><<<levels, 1024, 0, s>>>(tiles, ntiles_max, n_dev, n_host, over, over_cap, arena, gate, gate_want, h);
  else if (kind == 1)
    k_fixup<1><<<levels, 1024, 0, s>>>(tiles, ntiles_max, n_dev, n_host, over, over_cap, arena, gate, gate_want, h);
  else
    k_fixup<2><<<levels, 1024, 0, s>>>(tiles, ntiles_max, n_dev, n_host, over, over_cap, arena, gate, gate_want, h);
  count_launches(1);
}

}  // namespace aiwc
