// End-of-kernel statistics (Sec. V, kernelEnd): coverage counts, entropies,
// order statistics and ratios from the exact integer distributions.
//
// Every distribution is held as a dense count array for small values plus a
// tagged, sorted overflow list for large ones, so all integers are exact and
// every sum below runs in a fixed order (results do not depend on scheduling).
#include <math.h>

#include <algorithm>

#include "aiwc_internal.cuh"
#include "common.cuh"

namespace aiwc {
namespace {

constexpr int kFinThreads = 1024;

__global__ void k_wi_count(const u32* bitmap, Arena* arena) {
  __shared__ u64 red64[32];
  DevState* st = &arena->st;
  const u32 lo = st->wi_min, hi = st->wi_max;
  u64 c = 0;
  if (lo <= hi) {
    const u64 w0 = lo >> 5, w1 = hi >> 5;
    for (u64 w = w0 + (u64)blockIdx.x * blockDim.x + threadIdx.x; w <= w1; w += (u64)gridDim.x * blockDim.x)
      c += __popc(bitmap[w]);
  }
  c = block_reduce(c, OpAdd(), 0ull, red64);
  if (threadIdx.x == 0 && c) atomicAdd(&st->work_items, c);
}

__global__ void k_wi_clear(u32* bitmap, Arena* arena) {
  const DevState* st = &arena->st;
  const u32 lo = st->wi_min, hi = st->wi_max;
  if (lo > hi) return;
  const u64 w0 = lo >> 5, w1 = hi >> 5;
  for (u64 w = w0 + (u64)blockIdx.x * blockDim.x + threadIdx.x; w <= w1; w += (u64)gridDim.x * blockDim.x)
    bitmap[w] = 0u;
}

static_assert(sizeof(DevState) % 8 == 0 && sizeof(Arena) % 8 == 0, "the reset clears whole words");

// The end of an invocation's reductions in one launch: the first blocks take
// the opcode distribution (unique opcodes, their total and its count-of-counts), every block counts the
// work-item bitmap words in [wi_min, wi_max] and clears them behind it (the
// bitmap is read by nothing after the count).
__global__ void __launch_bounds__(256) k_tail_counts(const u64* hist, u32 n_opcodes, u32 op_blocks, u32* bitmap,
                                                     u64* over, u64 cap, Arena* arena) {
  __shared__ u64 red64[32];
  DevState* st = &arena->st;
  if (blockIdx.x < op_blocks) {
    u64 uniq = 0, tot = 0;
    for (u32 o = blockIdx.x * blockDim.x + threadIdx.x; o < n_opcodes; o += op_blocks * blockDim.x) {
      const u64 c = hist[o];
      if (c) {
        ++uniq;
        tot += c;
        if (c < (u64)kCocDense) atomicAdd(&arena->opc_coc[c], 1ull);
        else overflow_append(over, cap, st, kTagOpcodes, c);
      }
    }
    uniq = block_reduce(uniq, OpAdd(), 0ull, red64);
    tot = block_reduce(tot, OpAdd(), 0ull, red64);
    if (threadIdx.x == 0) {
      if (uniq) atomicAdd(&st->unique_opcodes, uniq);
      if (tot) atomicAdd(&st->total_instructions, tot);
    }
  }
  const u32 lo = st->wi_min, hi = st->wi_max;
  u64 c = 0;
  if (bitmap && lo <= hi) {
    const u64 w0 = lo >> 5, w1 = hi >> 5;
    for (u64 w = w0 + (u64)blockIdx.x * blockDim.x + threadIdx.x; w <= w1; w += (u64)gridDim.x * blockDim.x) {
      c += __popc(bitmap[w]);
      bitmap[w] = 0u;
    }
  }
  c = block_reduce(c, OpAdd(), 0ull, red64);
  if (threadIdx.x == 0 && c) atomicAdd(&st->work_items, c);
}

// A handle's device state back to the start of an invocation in one launch:
// the arena zeroed (block 0 takes the counters and then sets the AND
// accumulators and minima to their identities), the opcode histogram and the
// superblock table's keys and counters zeroed.
__global__ void __launch_bounds__(256) k_reset(Arena* arena, u64* hist, u32 n_opcodes, u64* sbt, u64 sbt_words) {
  if (blockIdx.x == 0) {
    u64* sw = reinterpret_cast<u64*>(&arena->st);
    for (u32 i = threadIdx.x; i < sizeof(DevState) / 8; i += blockDim.x) sw[i] = 0ull;
    __syncthreads();
    if (threadIdx.x == 0) {
      DevState* st = &arena->st;
      st->mem_and = ~0ull;
      st->br_and = ~0ull;
      st->pat_and = ~0ull;
      st->run_and = ~0ull;
      st->over_and = ~0ull;
      st->wi_min = 0xFFFFFFFFu;
      st->wi_max = 0u;
    }
    return;
  }
  const u64 tid = (u64)(blockIdx.x - 1) * blockDim.x + threadIdx.x, nt = (u64)(gridDim.x - 1) * blockDim.x;
  u64* rest = reinterpret_cast<u64*>(arena) + sizeof(DevState) / 8;
  const u64 rest_words = (sizeof(Arena) - sizeof(DevState)) / 8;
  for (u64 i = tid; i < rest_words; i += nt) rest[i] = 0ull;
  for (u64 i = tid; i < n_opcodes; i += nt) hist[i] = 0ull;
  for (u64 i = tid; i < sbt_words; i += nt) sbt[i] = 0ull;
}

__global__ void k_identities(Arena* arena) {
  DevState* st = &arena->st;
  st->mem_and = ~0ull;
  st->br_and = ~0ull;
  st->pat_and = ~0ull;
  st->run_and = ~0ull;
  st->over_and = ~0ull;
  st->wi_min = 0xFFFFFFFFu;
  st->wi_max = 0u;
}

// ---------------------------------------------------------------- finalize

struct Shared {
  u64 red[32];
  double redd[32];
  u64 scan[33];
  u64 scan2[33];
  u64 tag_begin[kNumTags + 1];
  u64 found;
  u64 found_k;
};

__device__ __forceinline__ u64 block_sum_u64(u64 x, Shared& s) { return block_reduce(x, OpAdd(), 0ull, s.red); }

__device__ __forceinline__ double block_sum_f64(double x, Shared& s) {
  // fixed-shape tree: deterministic for a fixed assignment of inputs to threads
  return block_reduce(x, OpAdd(), 0.0, s.redd);
}

// Inclusive block scan of two u64 sequences at once.
__device__ __forceinline__ void block_scan2(u64 x, u64 y, u64* ix, u64* iy, u64* tx, u64* ty, Shared& s) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  u64 a = x, b = y;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    u64 pa = __shfl_up_sync(0xffffffffu, a, o), pb = __shfl_up_sync(0xffffffffu, b, o);
    if (lane >= o) { a += pa; b += pb; }
  }
  __syncthreads();
  if (lane == 31) { s.scan[w] = a; s.scan2[w] = b; }
  __syncthreads();
  if (w == 0) {
    u64 va = lane < nw ? s.scan[lane] : 0ull, vb = lane < nw ? s.scan2[lane] : 0ull;
    u64 ia = va, ib = vb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      u64 pa = __shfl_up_sync(0xffffffffu, ia, o), pb = __shfl_up_sync(0xffffffffu, ib, o);
      if (lane >= o) { ia += pa; ib += pb; }
    }
    if (lane < nw) { s.scan[lane] = ia - va; s.scan2[lane] = ib - vb; }
    if (lane == nw - 1) { s.scan[32] = ia; s.scan2[32] = ib; }
  }
  __syncthreads();
  *ix = a + s.scan[w];
  *iy = b + s.scan2[w];
  *tx = s.scan[32];
  *ty = s.scan2[32];
  __syncthreads();
}

// Fewest groups whose sizes cover num/den of `total`: the smallest k with
// den * (sum of the k largest sizes) >= num * total. Sizes come as the
// overflow segment [ob, oe) (ascending) followed by dense[c] groups of size c.
__device__ u64 cover_walk(const u64* dense, int dense_n, const u64* over, u64 ob, u64 oe, u64 total, u32 num,
                          u32 den, Shared& s) {
  if (total == 0) return 0;
  typedef unsigned __int128 u128;
  const u128 target = (u128)num * total;
  u64 cum = 0, kcount = 0;
  // large sizes, descending
  for (u64 c0 = 0; c0 < oe - ob; c0 += blockDim.x) {
    const u64 idx = c0 + threadIdx.x;
    const bool v = idx < oe - ob;
    const u64 c = v ? (over[oe - 1 - idx] & kValueMask) : 0ull;
    u64 ic, im, tc, tm;
    block_scan2(c, v ? 1ull : 0ull, &ic, &im, &tc, &tm, s);
    if (threadIdx.x == 0) s.found = ~0ull;
    __syncthreads();
    if (v && (u128)den * (cum + ic) >= target) atomicMin(&s.found, idx - c0);
    __syncthreads();
    const u64 f = s.found;
    __syncthreads();
    if (f != ~0ull) return kcount + f + 1;
    cum += tc;
    kcount += tm;
  }
  // dense sizes, descending: thread t takes size dense_n-1-t (chunks of blockDim)
  for (int c0 = 0; c0 < dense_n; c0 += blockDim.x) {
    const int ci = dense_n - 1 - (c0 + (int)threadIdx.x);
    const bool v = ci >= 1;
    const u64 m = v ? dense[ci] : 0ull;
    const u64 mc = m * (u64)(v ? ci : 0);
    u64 imc, im, tmc, tm;
    block_scan2(mc, m, &imc, &im, &tmc, &tm, s);
    if (threadIdx.x == 0) { s.found = ~0ull; s.found_k = 0; }
    __syncthreads();
    const bool hit = v && m && (u128)den * (cum + imc) >= target;
    u64 k_here = 0;
    if (hit) {
      // the largest size reaching the target; within it, how many groups of size ci
      const u128 before = (u128)den * (cum + imc - mc);
      const u128 need = target > before ? target - before : 0;
      const u128 per = (u128)den * (u64)ci;
      const u64 r = (u64)((need + per - 1) / per);
      k_here = kcount + (im - m) + (r ? r : 1);
      atomicMin(&s.found, (u64)(c0 + threadIdx.x));
    }
    __syncthreads();
    if (hit && (u64)(c0 + threadIdx.x) == s.found) s.found_k = k_here;
    __syncthreads();
    const u64 found = s.found, found_k = s.found_k;
    __syncthreads();
    if (found != ~0ull) return found_k;
    cum += tmc;
    kcount += tm;
  }
  return kcount;
}

// Order statistics of a value distribution: dense[v] values v for v <
// kValDense, then the ascending overflow segment [ob, oe). Each thread owns
// kPer consecutive bins; one pass sums them (independent loads; bins from
// dense_n on are known to be empty and are not read), one block scan places
// every thread's slice, and the threads whose slices hold the wanted ranks
// find the values.
constexpr int kPer = kValDense / kFinThreads;
static_assert(kValDense % kFinThreads == 0, "bins must split evenly over the block");

__device__ void order_stats(const u64* dense, int dense_n, const u64* over, u64 ob, u64 oe, u64* cnt, u64* mn,
                            u64* mx, u64* lo, u64* hi, double* med, Shared& s) {
  const int b0 = threadIdx.x * kPer;
  const ulonglong2* d2 = reinterpret_cast<const ulonglong2*>(dense + b0);
  u64 mine = 0;
#pragma unroll 8
  for (int q = 0; q < kPer / 2; ++q) {
    if (b0 + 2 * q >= dense_n) break;
    const ulonglong2 v = d2[q];
    mine += v.x + v.y;
  }
  u64 inc, dummy, tot, dt;
  block_scan2(mine, 0ull, &inc, &dummy, &tot, &dt, s);
  const u64 c = tot + (oe - ob);
  *cnt = c;
  if (c == 0) { *mn = *mx = *lo = *hi = 0; *med = 0.0; return; }
  const u64 ranks[4] = {0, c - 1, (c - 1) / 2, c / 2};
  __shared__ u64 found[4];
  const u64 ex = inc - mine;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const u64 k = ranks[r];
    if (k < tot) {
      if (k >= ex && k < inc) {
        u64 acc = ex;
        for (int v = b0; v < b0 + kPer; ++v) {
          acc += dense[v];
          if (k < acc) { found[r] = (u64)v; break; }
        }
      }
    } else if (threadIdx.x == 0) {
      const u64 j = k - tot;
      found[r] = ob + j < oe ? (over[ob + j] & kValueMask) : 0ull;
    }
  }
  __syncthreads();
  *mn = found[0];
  *mx = found[1];
  *lo = found[2];
  *hi = found[3];
  *med = 0.5 * ((double)*lo + (double)*hi);
  __syncthreads();
}

// Index one past the run of value v that starts at i in the ascending
// overflow segment [i, oe).
__device__ __forceinline__ u64 run_end(const u64* over, u64 i, u64 oe, u64 v) {
  u64 lo = i + 1, hi = oe;
  while (lo < hi) {
    const u64 mid = (lo + hi) >> 1;
    if ((over[mid] & kValueMask) == v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Sum over groups of c*log2(c), given m_c for small c and the overflow list
// entries for large c. Equal sizes are adjacent in the sorted overflow
// segment, so each distinct size is evaluated once, times its multiplicity
// (the thread holding the first entry of a run owns it). FP64 path: each
// term in double. FP32 path: with c = f * 2^e (f in [1,2)), c*log2(c) =
// c*e + c*log2(f); the first part is an exact integer, the second is
// accumulated in float with Kahan compensation per thread; only the
// cross-thread reduction is in double.
__device__ double clog_sum(const u64* dense, int dense_n, const u64* over, u64 ob, u64 oe, u32 precision,
                           Shared& s, int c_lo = 0) {
  if (precision == 0) {
    double acc = 0.0;
    // bins c_lo .. dense_n-1, eight loads in flight per thread
    for (int c0 = c_lo + (int)threadIdx.x; c0 < dense_n; c0 += 8 * blockDim.x) {
      u64 m[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int c = c0 + q * (int)blockDim.x;
        m[q] = c < dense_n ? dense[c] : 0ull;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int c = c0 + q * (int)blockDim.x;
        if (m[q] && c > 1) acc += (double)m[q] * ((double)c * log2((double)c));
      }
    }
    for (u64 i = ob + threadIdx.x; i < oe; i += blockDim.x) {
      const u64 v = over[i] & kValueMask;
      if (i > ob && (over[i - 1] & kValueMask) == v) continue;
      const u64 m = run_end(over, i, oe, v) - i;
      const double c = (double)v;
      acc += (double)m * (c * log2(c));
    }
    return block_sum_f64(acc, s);
  }
  u64 exact = 0;
  float sum = 0.0f, comp = 0.0f;
  auto add = [&](u64 c, u64 m) {
    const int e = 63 - __clzll((long long)c);
    exact += m * c * (u64)e;
    const float f = (float)((double)c / (double)(1ull << e));
    const float term = (float)(m * c) * log2f(f);
    const float y = term - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
  };
  for (int c = c_lo + (int)threadIdx.x; c < dense_n; c += blockDim.x) {
    const u64 m = dense[c];
    if (m && c > 1) add((u64)c, m);
  }
  for (u64 i = ob + threadIdx.x; i < oe; i += blockDim.x) {
    const u64 v = over[i] & kValueMask;
    if (i > ob && (over[i - 1] & kValueMask) == v) continue;
    add(v, run_end(over, i, oe, v) - i);
  }
  const u64 ex = block_sum_u64(exact, s);
  const double fl = block_sum_f64((double)sum - (double)comp, s);
  return (double)ex + fl;
}

// One block per independent task: blocks 0..10 the entropy of each skip
// level, 11..13 the three coverage counts, 14..15 the ITB / IPT order
// statistics, 16 the scalar fields, 17..17+kYokParts-1 slices of the pattern
// term of the Yokota entropy and the next block its site term; the last of
// those to finish combines them in a fixed order. Each block writes disjoint
// fields.
constexpr int kYokParts = 8;
constexpr int kFinBlocks = 17 + kYokParts + 1;

__global__ void __launch_bounds__(kFinThreads) k_finalize(FinalizeArgs a) {
  __shared__ Shared s;
  Arena* ar = a.arena;
  const DevState& st = ar->st;
  const u64* over = *a.over_cur ? a.over_b : a.over_a;
  const u64 nover = umin64(st.n_over, a.over_cap);
  // segment of each tag in the sorted overflow list (lower bound of tag << 56)
  if (threadIdx.x <= kNumTags) {
    const u64 key = (u64)threadIdx.x << 56;
    u64 lo = 0, hi = nover;
    while (lo < hi) {
      const u64 mid = (lo + hi) >> 1;
      if (over[mid] < key) lo = mid + 1; else hi = mid;
    }
    s.tag_begin[threadIdx.x] = lo;
  }
  __syncthreads();
  aiwc_metrics* m = &a.result->m;
  const int task = blockIdx.x;
  const u64 N = st.total_reads + st.total_writes;
  // bins past these are empty: an ITB or IPT value counts at most every
  // instruction slot, a pattern or site at most every branch outcome
  const int val_n = (int)umin64(st.total_instructions + st.barriers + 1, (u64)kValDense);
  const int pat_n = (int)umin64(st.n_branch + 1, (u64)kValDense);
  if (task < kLevels) {
    const int l = task;
    const double S = clog_sum(ar->mem_coc[l], kCocDense, over, s.tag_begin[l], s.tag_begin[l + 1], a.precision, s);
    if (threadIdx.x == 0) {
      double H = 0.0;
      if (N) {
        if (a.precision) {
          // log2 N = e + log2(f) with the same split as the terms
          const int e = 63 - __clzll((long long)N);
          H = (double)e + (double)log2f((float)((double)N / (double)(1ull << e)));
        } else {
          H = log2((double)N);
        }
        H -= S / (double)N;
        if (H < 0.0) H = 0.0;
      }
      m->entropy[l] = H;
    }
  } else if (task == 11) {
    const u64 c = cover_walk(ar->mem_coc[0], kCocDense, over, s.tag_begin[0], s.tag_begin[1], N, a.cover_num,
                             a.cover_den, s);
    if (threadIdx.x == 0) m->footprint_cover = c;
  } else if (task == 12) {
    const u64 c = cover_walk(ar->site_coc, kCocDense, over, s.tag_begin[kTagSites], s.tag_begin[kTagSites + 1],
                             st.n_branch, a.cover_num, a.cover_den, s);
    if (threadIdx.x == 0) m->branch_cover = c;
  } else if (task == 13) {
    const u64 c = cover_walk(ar->opc_coc, kCocDense, over, s.tag_begin[kTagOpcodes], s.tag_begin[kTagOpcodes + 1],
                             st.total_instructions, a.cover_num, a.cover_den, s);
    if (threadIdx.x == 0) m->opcode_cover = c;
  } else if (task == 14 || task == 15) {
    const bool itb = task == 14;
    const int tag = itb ? kTagItb : kTagIpt;
    u64 c, mn, mx, lo, hi;
    double med;
    order_stats(itb ? ar->itb_dense : ar->ipt_dense, val_n, over, s.tag_begin[tag], s.tag_begin[tag + 1], &c, &mn,
                &mx, &lo, &hi, &med, s);
    if (threadIdx.x == 0) {
      if (itb) {
        m->itb_count = c; m->itb_min = mn; m->itb_max = mx; m->itb_median_lo = lo; m->itb_median_hi = hi;
        // 1 / mean ITB, mean ITB = total instructions / ITB count (Sec. VI)
        m->barriers_per_instruction = (double)c / (double)st.total_instructions;
        m->itb_median = med;
      } else {
        m->ipt_count = c; m->ipt_min = mn; m->ipt_max = mx; m->ipt_median_lo = lo; m->ipt_median_hi = hi;
        m->load_imbalance = (double)(mx - mn);  // Sec. VI
        m->ipt_median = med;
      }
    }
  } else if (task >= 17) {
    // H(history | site) = (1/N') [sum_s N'_s log2 N'_s - sum_P n_P log2 n_P], in units of h bits
    const int part = task - 17;
    double v;
    if (part < kYokParts) {
      constexpr int kSlice = kValDense / kYokParts;
      const u64 ob = part == 0 ? s.tag_begin[kTagPat] : 0, oe = part == 0 ? s.tag_begin[kTagPat + 1] : 0;
      v = clog_sum(ar->pat_coc, min((part + 1) * kSlice, pat_n), over, ob, oe, 0, s, part * kSlice);
    } else {
      v = clog_sum(ar->site_pat_coc, pat_n, over, s.tag_begin[kTagSitePat], s.tag_begin[kTagSitePat + 1], 0, s);
    }
    __shared__ bool last;
    if (threadIdx.x == 0) {
      ar->yok_part[part] = v;
      __threadfence();
      last = atomicAdd(&ar->yok_done, 1u) == (u32)kYokParts;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
      __threadfence();
      const volatile double* p = ar->yok_part;
      double sp = 0.0;
      for (int q = 0; q < kYokParts; ++q) sp += p[q];
      const double y = st.npat ? (p[kYokParts] - sp) / ((double)st.npat * (double)a.history_len) : 0.0;
      m->yokota = y < 0.0 ? 0.0 : y;
    }
  } else if (threadIdx.x == 0) {
    m->total_instructions = st.total_instructions;
    m->unique_opcodes = st.unique_opcodes;
    m->work_items = st.work_items;
    m->barriers = st.barriers;
    m->total_reads = st.total_reads;
    m->total_writes = st.total_writes;
    m->footprint = st.footprint;
    m->unique_reads = st.unique_reads;
    m->unique_writes = st.unique_writes;
    m->branch_events = st.n_branch;
    m->branch_sites = st.branch_sites;
    m->branch_patterns = st.npat;
    m->branch_minsum = st.minsum;
    // one FP64 division of two exact integers in both precision modes: there is
    // no sum to compensate, so FP32 would only lose accuracy
    m->albe = st.npat ? 2.0 * (double)st.minsum / (double)st.npat : 0.0;
    m->unique_rw_ratio = (double)st.unique_reads / (double)st.unique_writes;
    m->reread_ratio = (double)st.unique_reads / (double)st.total_reads;
    m->rewrite_ratio = (double)st.unique_writes / (double)st.total_writes;
    // SIMD widths (Table I): population variance from exact integer sums,
    // (count * sumsq - sum^2) / count^2
    m->simd_count = st.simd_count;
    m->simd_max = st.simd_max;
    m->simd_sum = st.simd_sum;
    m->simd_sumsq = st.simd_sumsq;
    if (st.simd_count) {
      typedef unsigned __int128 u128;
      const u128 num = (u128)st.simd_count * st.simd_sumsq - (u128)st.simd_sum * st.simd_sum;
      m->simd_mean = (double)st.simd_sum / (double)st.simd_count;
      m->simd_sd = sqrt((double)num / ((double)st.simd_count * (double)st.simd_count));
    } else {
      m->simd_mean = 0.0;
      m->simd_sd = 0.0;
    }
    // derived parallelism quantities of the Kiviat diagrams (Sec. VI)
    m->granularity = 1.0 / (double)st.work_items;
    m->instructions_per_operand = 1.0 / (double)st.simd_sum;
    m->opcode_hist = nullptr;
    a.result->err = st.err;
  }
}

// ---------------------------------------------------------------- partitioned invocations
// Every distribution a partition reduces to is exact and additive: dense
// count-of-counts and value bins add, overflow entries concatenate, counters
// add (maxima and minima combine). The total arena is touched only by these
// kernels, in stream order, so plain read-modify-writes suffice.

// Appends the partition's overflow entries behind the total's.
__global__ void k_merge_over(const Arena* part, const u64* part_over, u64 part_cap, Arena* total, u64* total_over,
                             u64 total_cap) {
  const u64 n = umin64(part->st.n_over, part_cap);
  const u64 base = total->st.n_over;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
    if (base + i < total_cap) total_over[base + i] = part_over[i];
}

__global__ void k_merge_arena(const Arena* part, Arena* total, u64 part_cap, u64 total_cap) {
  const u64 stride = (u64)gridDim.x * blockDim.x;
  const u64 i0 = (u64)blockIdx.x * blockDim.x + threadIdx.x;
  auto add = [&](u64* dst, const u64* src, u64 n) {
    for (u64 i = i0; i < n; i += stride)
      if (src[i]) dst[i] += src[i];
  };
  add(&total->mem_coc[0][0], &part->mem_coc[0][0], (u64)kLevels * kCocDense);
  add(total->site_coc, part->site_coc, kCocDense);
  add(total->itb_dense, part->itb_dense, kValDense);
  add(total->ipt_dense, part->ipt_dense, kValDense);
  add(total->pat_coc, part->pat_coc, kValDense);
  add(total->site_pat_coc, part->site_pat_coc, kValDense);
  if (i0 == 0) {
    const DevState& p = part->st;
    DevState& t = total->st;
    t.total_reads += p.total_reads;
    t.total_writes += p.total_writes;
    t.footprint += p.footprint;
    t.unique_reads += p.unique_reads;
    t.unique_writes += p.unique_writes;
    t.n_branch += p.n_branch;
    t.branch_sites += p.branch_sites;
    t.npat += p.npat;
    t.minsum += p.minsum;
    t.barriers += p.barriers;
    t.simd_count += p.simd_count;
    t.simd_sum += p.simd_sum;
    t.simd_sumsq += p.simd_sumsq;
    t.simd_max = p.simd_max > t.simd_max ? p.simd_max : t.simd_max;
    t.err |= p.err;
    if (p.wi_min < t.wi_min) t.wi_min = p.wi_min;
    if (p.wi_max > t.wi_max) t.wi_max = p.wi_max;
    const u64 n = umin64(p.n_over, part_cap);
    if (p.n_over > part_cap || t.n_over + n > total_cap) t.err |= kErrOverflow;
    t.n_over += n;
    t.over_or |= p.over_or;
    t.over_and &= p.over_and;
  }
}

}  // namespace

// Sharded invocations: a rank's opcode histogram is added to the merged one,
// and its work-item bitmap words are ORed into the merged bitmap.
__global__ void k_add_u64(u64* dst, const u64* src, u64 n) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
    if (src[i]) dst[i] += src[i];
}
__global__ void k_or_u32(u32* dst, const u32* src, u64 n) {
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
    if (src[i]) dst[i] |= src[i];
}

void launch_add_u64(u64* dst, const u64* src, u64 n, int sm_count, cudaStream_t s) {
  if (!n) return;
  const u64 g = std::min<u64>((n + 255) / 256, (u64)sm_count * 4);
  k_add_u64<<<(unsigned)g, 256, 0, s>>>(dst, src, n);
  count_launches(1);
}
void launch_or_u32(u32* dst, const u32* src, u64 n, int sm_count, cudaStream_t s) {
  if (!n) return;
  const u64 g = std::min<u64>((n + 255) / 256, (u64)sm_count * 4);
  k_or_u32<<<(unsigned)g, 256, 0, s>>>(dst, src, n);
  count_launches(1);
}

void launch_merge_partition(const Arena* part, const u64* part_over, u64 part_cap, Arena* total, u64* total_over,
                            u64 total_cap, cudaStream_t s) {
  k_merge_over<<<152 * 2, 256, 0, s>>>(part, part_over, part_cap, total, total_over, total_cap);
  k_merge_arena<<<152 * 2, 256, 0, s>>>(part, total, part_cap, total_cap);
  count_launches(2);
}

void launch_tail_counts(const u64* hist, u32 n_opcodes, u32* bitmap, u64* over, u64 over_cap, Arena* arena,
                        cudaStream_t s) {
  const u32 op_blocks = std::max<u32>(1u, std::min<u32>((n_opcodes + 255) / 256, 64u));
  k_tail_counts<<<152 * 2, 256, 0, s>>>(hist, n_opcodes, op_blocks, bitmap, over, over_cap, arena);
  count_launches(1);
}

void launch_reset(Arena* arena, u64* hist, u32 n_opcodes, u64* sbt, u64 sbt_words, cudaStream_t s) {
  k_reset<<<1 + 152 * 2, 256, 0, s>>>(arena, hist, n_opcodes, sbt, sbt_words);
  count_launches(1);
}

void launch_wi_count(const u32* bitmap, Arena* arena, cudaStream_t s) {
  k_wi_count<<<152 * 2, 256, 0, s>>>(bitmap, arena);
  count_launches(1);
}

void launch_wi_clear(u32* bitmap, Arena* arena, cudaStream_t s) {
  k_wi_clear<<<152 * 2, 256, 0, s>>>(bitmap, arena);
  count_launches(1);
}

void launch_reset_identities(Arena* arena, cudaStream_t s) {
  k_identities<<<1, 1, 0, s>>>(arena);
  count_launches(1);
}

void launch_finalize(const FinalizeArgs& a, cudaStream_t s) {
  k_finalize<<<kFinBlocks, kFinThreads, 0, s>>>(a);
  count_launches(1);
}

}  // namespace aiwc
