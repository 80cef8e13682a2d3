// Run lengths of equal groups in a sorted array, tile by tile.
//
// A run is a maximal stretch of consecutive sorted keys with the same group
// (for example key >> n). Each 4096-key tile is held in blocked arrangement
// (thread t owns positions base + 16t .. base + 16t + 15). Runs that start and
// end inside one thread are emitted by that thread; runs that cross threads
// are found with a block-wide segmented scan; runs that cross tiles are left
// to a fix-up pass over per-tile summaries (has a head, length before the
// first head, length from the last head, total), which is a segmented scan
// over tiles. Every run is emitted exactly once, with its length and the sum
// of a per-key weight over the run.
#pragma once

#include "aiwc_internal.cuh"

namespace aiwc {

struct Seg {
  u32 b;  // a head (group start) lies in the covered range
  u64 v;  // length of the run open at the end of the range
  u64 w;  // weight of that open run
};

__device__ __forceinline__ Seg seg_identity() { return Seg{0u, 0ull, 0ull}; }

// (x then y): a head in y restarts the open run.
__device__ __forceinline__ Seg seg_op(const Seg& x, const Seg& y) {
  Seg r;
  r.b = x.b | y.b;
  r.v = y.b ? y.v : x.v + y.v;
  r.w = y.b ? y.w : x.w + y.w;
  return r;
}

__device__ __forceinline__ Seg seg_shfl_up(const Seg& x, int o) {
  Seg r;
  r.b = __shfl_up_sync(0xffffffffu, x.b, o);
  r.v = __shfl_up_sync(0xffffffffu, x.v, o);
  r.w = __shfl_up_sync(0xffffffffu, x.w, o);
  return r;
}

// Block-wide exclusive segmented scan. sh must hold 33 entries.
__device__ __forceinline__ Seg block_seg_scan(const Seg& x, Seg* agg, Seg* sh) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  Seg inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    Seg y = seg_shfl_up(inc, o);
    if (lane >= o) inc = seg_op(y, inc);
  }
  Seg ex = seg_shfl_up(inc, 1);
  if (lane == 0) ex = seg_identity();
  if (lane == 31) sh[wp] = inc;
  __syncthreads();
  if (wp == 0) {
    Seg v = lane < nw ? sh[lane] : seg_identity();
    Seg vi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      Seg y = seg_shfl_up(vi, o);
      if (lane >= o) vi = seg_op(y, vi);
    }
    Seg vx = seg_shfl_up(vi, 1);
    if (lane == 0) vx = seg_identity();
    if (lane < nw) sh[lane] = vx;
    if (lane == nw - 1) sh[32] = vi;
  }
  __syncthreads();
  Seg r = seg_op(sh[wp], ex);
  *agg = sh[32];
  __syncthreads();
  return r;
}

// One tile. key[] holds this thread's ITEMS keys, the first `nvalid` valid;
// prev is the key before key[0] (ignored when pos0 == 0). grp maps a key to
// its group, wt to its weight; emit(len, wsum) receives completed runs.
// The tile summary is written to *sum by thread 0. sh: 33 Seg; pre_slot: 2 u64.
template <int ITEMS, typename Grp, typename Wt, typename Emit>
__device__ __forceinline__ void tile_runs(const u64 (&key)[ITEMS], int nvalid, u64 pos0, u64 prev, u64 tile_n,
                                          Grp grp, Wt wt, Emit emit, TileSum* sum, Seg* sh, u64* pre_slot) {
  int fh = -1, lh = -1;
  u64 w_lead = 0, w_run = 0;
  u64 g_prev = grp(prev);
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    if (k < nvalid) {
      u64 g = grp(key[k]);
      bool hd = (pos0 + k == 0) || (g != g_prev);
      if (hd) {
        if (lh >= 0) emit((u64)(k - lh), w_run);
        else fh = k;
        lh = k;
        w_run = 0;
      }
      u64 wk = wt(key[k]);
      if (lh < 0) w_lead += wk; else w_run += wk;
      g_prev = g;
    }
  }
  const bool has_b = fh >= 0;
  Seg e;
  e.b = has_b ? 1u : 0u;
  e.v = has_b ? (u64)(nvalid - lh) : (u64)nvalid;
  e.w = has_b ? w_run : w_lead;
  Seg agg;
  Seg ex = block_seg_scan(e, &agg, sh);
  if (has_b) {
    if (ex.b) {
      emit(ex.v + (u64)fh, ex.w + w_lead);
    } else {
      pre_slot[0] = ex.v + (u64)fh;
      pre_slot[1] = ex.w + w_lead;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    TileSum t;
    t.has_b = agg.b;
    t.pad = 0;
    t.pre = agg.b ? pre_slot[0] : agg.v;
    t.pre_w = agg.b ? pre_slot[1] : agg.w;
    t.suf = agg.b ? agg.v : 0ull;
    t.suf_w = agg.b ? agg.w : 0ull;
    t.tot = tile_n;
    t.tot_w = agg.b ? 0ull : agg.w;
    *sum = t;
  }
  __syncthreads();
}

}  // namespace aiwc
