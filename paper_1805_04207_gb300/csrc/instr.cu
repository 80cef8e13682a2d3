// Instruction path (Table I compute and parallelism rows; Sec. III / Sec. V):
// opcode histogram, barrier count, instructions-to-barrier (ITB) segments and
// instructions per thread (IPT).
//
// One warp scans one run (a work-item's opcodes in program order) 512
// opcodes at a time, 16 per lane. Segments closed by two barriers inside the
// run are emitted directly; a warp-wide segmented scan carries the open tally
// across lanes and steps. What a run cannot finish alone -- the tally before
// its first barrier and after its last -- is left in a 4-word run summary;
// after the runs are sorted by (work-item, push order) one thread per
// work-item chains its summaries, emitting the cross-run segments, the final
// implicit-barrier segment and the work-item's IPT.
#include <algorithm>

#include "aiwc_internal.cuh"
#include "common.cuh"
#include "runs.cuh"

namespace aiwc {
namespace {

constexpr int kInThreads = 256;
constexpr int kInWarps = kInThreads / 32;
constexpr int kOpsPerLane = 32;  // opcodes each lane takes per step (16-byte loads of 8; at most 32)

// Value histograms (ITB / IPT): privatised in shared memory below kValSmem,
// global dense below kValDense, overflow list above.
__device__ __forceinline__ void emit_value(u32* smem_hist, u64* dense, u64* over, u64 cap, DevState* st, int tag,
                                           u64 v) {
  if (v < (u64)kValSmem) atomicAdd(&smem_hist[v], 1u);
  else if (v < (u64)kValDense) atomicAdd(&dense[v], 1ull);
  else overflow_append(over, cap, st, tag, v);
}

// In-step segmented scan over the lanes, packed in one word: bit 31 = a
// barrier lies in the covered lanes, bits 0..30 = instructions since the last
// one (at most 512 per step). Returns the exclusive prefix; *agg = the whole
// warp's value.
__device__ __forceinline__ u32 warp_seg_scan32(u32 x, u32* agg) {
  const int lane = threadIdx.x & 31;
  u32 inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u32 y = __shfl_up_sync(0xffffffffu, inc, o);
    // (y then inc): a barrier in inc restarts the count
    if (lane >= o) inc = (inc >> 31) ? inc : y + inc;
  }
  *agg = __shfl_sync(0xffffffffu, inc, 31);
  const u32 ex = __shfl_up_sync(0xffffffffu, inc, 1);
  return lane == 0 ? 0u : ex;
}

// HMODE: 0 = per-warp shared histograms, 1 = one shared histogram per
// block, 2 = global atomics. Every opcode slot adds to bin min(opcode,
// n_opcodes): the spare bin n_opcodes takes barriers, padding (written as
// barrier markers) and invalid opcodes, so invalid opcodes are found at the
// end as spare - barriers - padding. Opcodes are handled two per 32-bit word
// (a halfword compare finds the barrier markers, a halfword minimum clamps
// the bins).
template <int HMODE>
__global__ void __launch_bounds__(kInThreads, 4) k_instr_runs(RunBatchArgs a) {
  constexpr int hist_mode = HMODE;
  extern __shared__ u32 dyn[];
  __shared__ u32 itb_small[kValSmem];
  __shared__ u64 red64[32];
  __shared__ u32 red32[32];
  DevState* st = &a.arena->st;
  const u32 nop = a.n_opcodes;
  const u32 clampv = nop | (nop << 16);
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const u32 hstride = nop + 1;
  const u32 hwords = hist_mode == 0 ? hstride * kInWarps : (hist_mode == 1 ? hstride : 0u);
  for (u32 i = threadIdx.x; i < hwords; i += kInThreads) dyn[i] = 0u;
  for (int i = threadIdx.x; i < kValSmem; i += kInThreads) itb_small[i] = 0u;
  __syncthreads();
  u32* my_hist = hist_mode == 0 ? dyn + wp * hstride : dyn;
  u64 nbar = 0, npad = 0, nspare_g = 0, run_or = 0, run_and = ~0ull;
  u32 err = 0, wmin = 0xFFFFFFFFu, wmax = 0u;
  const u64 gwarp = (u64)blockIdx.x * kInWarps + wp;
  const u64 nwarps = (u64)gridDim.x * kInWarps;
  // the next run's descriptor is loaded while the current one is scanned
  u64 n_off = 0, n_len = 0;
  u32 n_wi = 0;
  if (gwarp < a.n_runs) { n_off = a.run_off[gwarp]; n_len = a.run_len[gwarp]; n_wi = a.run_wi[gwarp]; }
  for (u64 r = gwarp; r < a.n_runs; r += nwarps) {
    const u64 off = n_off;
    u64 len = n_len;
    const u32 wi = n_wi;
    if (r + nwarps < a.n_runs) {
      n_off = a.run_off[r + nwarps];
      n_len = a.run_len[r + nwarps];
      n_wi = a.run_wi[r + nwarps];
    }
    if (off > a.n_ops || len > a.n_ops - off) {
      err |= kErrRun;
      len = 0;
    }
    mark_work_items(a.wi_bitmap, a.max_wi, wi, lane == 0, &err);
    if ((u64)wi < a.max_wi) {
      wmin = min(wmin, wi);
      wmax = max(wmax, wi);
    }
    const uint16_t* p = a.ops + off;
    const bool aligned = ((reinterpret_cast<uintptr_t>(p) & 15u) == 0);
    bool carry_b = false;  // a barrier seen so far in this run
    u64 carry_v = 0;       // instructions since the last barrier (or the run start)
    u64 tot = 0, run_pre = 0;
    bool have_pre = false;
    for (u64 s0 = 0; s0 < len; s0 += 32 * kOpsPerLane) {
      const u64 my0 = s0 + (u64)lane * kOpsPerLane;
      const int nv = my0 < len ? (int)umin64(len - my0, (u64)kOpsPerLane) : 0;
      u32 pk[kOpsPerLane / 2];  // two opcodes per word, low half first; padding = barrier marker
      if (nv == kOpsPerLane && aligned) {
        const uint4* q = reinterpret_cast<const uint4*>(p + my0);
#pragma unroll
        for (int v = 0; v < kOpsPerLane / 8; ++v) {
          const uint4 x = __ldcs(q + v);
          pk[4 * v] = x.x;
          pk[4 * v + 1] = x.y;
          pk[4 * v + 2] = x.z;
          pk[4 * v + 3] = x.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < kOpsPerLane / 2; ++k) {
          const u32 lo = 2 * k < nv ? (u32)p[my0 + 2 * k] : (u32)AIWC_BARRIER;
          const u32 hi = 2 * k + 1 < nv ? (u32)p[my0 + 2 * k + 1] : (u32)AIWC_BARRIER;
          pk[k] = lo | (hi << 16);
        }
        npad += (u64)(kOpsPerLane - nv);
      }
      // bit k of bm: opcode k is a barrier marker. Per four opcodes: the
      // halfword compares give 0xFFFF per marker, one byte permute keeps a
      // byte of each, and a multiply gathers the four top bits into a nibble
      u32 bm = 0;
#pragma unroll
      for (int k = 0; k < kOpsPerLane / 2; k += 2) {
        const u32 bytes = __byte_perm(__vcmpeq2(pk[k], 0xFFFFFFFFu), __vcmpeq2(pk[k + 1], 0xFFFFFFFFu), 0x7531);
        bm |= (((bytes & 0x80808080u) * 0x00204081u) >> 28) << (2 * k);
      }
#pragma unroll
      for (int k = 0; k < kOpsPerLane / 2; ++k) {
        if (hist_mode == 2) {
          const u32 lo = pk[k] & 0xFFFFu, hi = pk[k] >> 16;
          if (lo < nop) atomicAdd(&a.opc_hist[lo], 1ull);
          else ++nspare_g;
          if (hi < nop) atomicAdd(&a.opc_hist[hi], 1ull);
          else ++nspare_g;
        } else {
          const u32 c = __vminu2(pk[k], clampv);  // both bins: min(opcode, n_opcodes)
          atomicAdd(&my_hist[c & 0xFFFFu], 1u);
          atomicAdd(&my_hist[c >> 16], 1u);
        }
      }
      const u32 vm = nv >= 32 ? 0xFFFFFFFFu : ((1u << nv) - 1u);
      bm &= vm;
      const u32 nbm = vm & ~bm;
      const u32 cnt = (u32)__popc(nbm);
      u32 lead, cur;
      if (bm) {
        const int fb = __ffs(bm) - 1, lb = 31 - __clz(bm);
        lead = (u32)__popc(nbm & ((1u << fb) - 1u));
        cur = (u32)__popc(nbm & ~((2u << lb) - 1u));
        nbar += (u64)__popc(bm);
        // segments closed by two barriers of this lane
        u32 rest = bm & (bm - 1u);
        int prevb = fb;
        while (rest) {
          const int nb = __ffs(rest) - 1;
          const u32 between = ((1u << nb) - 1u) & ~((2u << prevb) - 1u);
          emit_value(itb_small, a.arena->itb_dense, a.over, a.over_cap, st, kTagItb, (u64)__popc(nbm & between));
          prevb = nb;
          rest &= rest - 1u;
        }
      } else {
        lead = cnt;
        cur = 0;
      }
      u32 agg;
      const u32 ex = warp_seg_scan32(bm ? (0x80000000u | cur) : lead, &agg);
      if (bm) {
        // the segment this lane's first barrier closes: the open count before
        // the step (if no barrier came earlier in the step), then the lanes before
        const u64 seg = (ex >> 31 ? 0ull : carry_v) + (ex & 0x7FFFFFFFu) + lead;
        if (carry_b || (ex >> 31)) emit_value(itb_small, a.arena->itb_dense, a.over, a.over_cap, st, kTagItb, seg);
        else { run_pre = seg; have_pre = true; }
      }
      if (agg >> 31) {
        carry_b = true;
        carry_v = agg & 0x7FFFFFFFu;
      } else {
        carry_v += agg;
      }
      tot += __reduce_add_sync(0xffffffffu, cnt);
    }
    const u32 pre_owner = __ballot_sync(0xffffffffu, have_pre);
    if (pre_owner) run_pre = __shfl_sync(0xffffffffu, run_pre, __ffs(pre_owner) - 1);
    if (lane == 0) {
      const u64 seq = a.seq_base + r;
      const u64 key = ((u64)wi << 32) | (seq & 0xFFFFFFFFull);
      a.run_keys[seq] = key;
      u64* sm = a.run_sum + 4 * seq;
      sm[0] = carry_b ? 1ull : 0ull;
      sm[1] = carry_b ? run_pre : tot;
      sm[2] = carry_b ? carry_v : 0ull;
      sm[3] = tot;
      run_or |= key;
      run_and &= key;
    }
    have_pre = false;
  }
  __syncthreads();
  u64 spare = nspare_g;
  if (hist_mode == 0) {
    for (u32 o = threadIdx.x; o < nop; o += kInThreads) {
      u32 s = 0;
      for (int q = 0; q < kInWarps; ++q) s += dyn[q * hstride + o];
      if (s) atomicAdd(&a.opc_hist[o], (u64)s);
    }
    if (threadIdx.x < kInWarps) spare += dyn[threadIdx.x * hstride + nop];
  } else if (hist_mode == 1) {
    for (u32 o = threadIdx.x; o < nop; o += kInThreads)
      if (dyn[o]) atomicAdd(&a.opc_hist[o], (u64)dyn[o]);
    if (threadIdx.x == 0) spare += dyn[nop];
  }
  for (int i = threadIdx.x; i < kValSmem; i += kInThreads)
    if (itb_small[i]) atomicAdd(&a.arena->itb_dense[i], (u64)itb_small[i]);
  nbar = block_reduce(nbar, OpAdd(), 0ull, red64);
  npad = block_reduce(npad, OpAdd(), 0ull, red64);
  spare = block_reduce(spare, OpAdd(), 0ull, red64);
  run_or = block_reduce(run_or, OpOr(), 0ull, red64);
  run_and = block_reduce(run_and, OpAnd(), ~0ull, red64);
  err = block_reduce(err, OpOr(), 0u, red32);
  wmin = block_reduce(wmin, OpMin(), 0xFFFFFFFFu, red32);
  wmax = block_reduce(wmax, OpMax(), 0u, red32);
  if (threadIdx.x == 0) {
    if (spare != nbar + npad) err |= kErrOpcode;  // slots in the spare bin that are neither barriers nor padding
    if (nbar) atomicAdd(&st->barriers, nbar);
    if (wmin <= wmax) {
      atomicOr(&st->run_or, run_or);
      atomicAnd(&st->run_and, run_and);
      atomicMin(&st->wi_min, wmin);
      atomicMax(&st->wi_max, wmax);
    }
    if (err) atomicOr(&st->err, err);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&st->n_runs, a.n_runs);
}

// One thread per run position in (work-item, push order); the first run of
// each work-item chains that work-item's runs.
__global__ void __launch_bounds__(256) k_instr_combine(CombineArgs a) {
  __shared__ u32 itb_small[kValSmem];
  __shared__ u32 ipt_small[kValSmem];
  DevState* st = &a.arena->st;
  for (int i = threadIdx.x; i < kValSmem; i += blockDim.x) { itb_small[i] = 0u; ipt_small[i] = 0u; }
  __syncthreads();
  const u64* keys = *a.cur ? a.b : a.a;
  const u64 stride = (u64)gridDim.x * blockDim.x;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < a.n_runs; i += stride) {
    const u64 k = keys[i];
    const u64 wi = k >> 32;
    if (i > 0 && (keys[i - 1] >> 32) == wi) continue;
    u64 open = 0, ipt = 0;
    for (u64 j = i; j < a.n_runs; ++j) {
      const u64 kj = keys[j];
      if ((kj >> 32) != wi) break;
      const u64* sm = a.run_sum + 4 * (kj & 0xFFFFFFFFull);
      if (sm[0]) {
        emit_value(itb_small, a.arena->itb_dense, a.over, a.over_cap, st, kTagItb, open + sm[1]);
        open = sm[2];
      } else {
        open += sm[3];
      }
      ipt += sm[3];
    }
    emit_value(itb_small, a.arena->itb_dense, a.over, a.over_cap, st, kTagItb, open);
    emit_value(ipt_small, a.arena->ipt_dense, a.over, a.over_cap, st, kTagIpt, ipt);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kValSmem; i += blockDim.x) {
    if (itb_small[i]) atomicAdd(&a.arena->itb_dense[i], (u64)itb_small[i]);
    if (ipt_small[i]) atomicAdd(&a.arena->ipt_dense[i], (u64)ipt_small[i]);
  }
}

// SIMD metrics (Table I): count, sum, sum of squares and maximum of the
// result widths; eight widths per 16-byte load when the array is aligned.
__global__ void __launch_bounds__(256) k_simd_widths(const uint16_t* w, u64 n, Arena* arena) {
  __shared__ u64 red64[32];
  u64 sum = 0, sumsq = 0, mx = 0;
  const u64 stride = (u64)gridDim.x * blockDim.x;
  const bool aligned = ((reinterpret_cast<uintptr_t>(w) & 15u) == 0);
  const u64 nv = aligned ? n / 8 : 0;
  const uint4* w8 = reinterpret_cast<const uint4*>(w);
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
    const uint4 v = __ldcs(w8 + i);
    const u32 p[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const u32 lo = p[q] & 0xFFFFu, hi = p[q] >> 16;
      sum += lo + hi;
      sumsq += (u64)(lo * lo) + (u64)(hi * hi);
      mx = umax64(mx, max(lo, hi));
    }
  }
  for (u64 i = nv * 8 + (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const u32 x = w[i];
    sum += x;
    sumsq += (u64)x * x;
    mx = umax64(mx, x);
  }
  sum = block_reduce(sum, OpAdd(), 0ull, red64);
  sumsq = block_reduce(sumsq, OpAdd(), 0ull, red64);
  mx = block_reduce(mx, OpMax(), 0ull, red64);
  if (threadIdx.x == 0) {
    DevState* st = &arena->st;
    if (sum) atomicAdd(&st->simd_sum, sum);
    if (sumsq) atomicAdd(&st->simd_sumsq, sumsq);
    if (mx) atomicMax(&st->simd_max, mx);
    if (blockIdx.x == 0) atomicAdd(&st->simd_count, n);
  }
}

__global__ void __launch_bounds__(256) k_keys_sorted(const u64* keys, u64 n, u32* flag) {
  bool bad = false;
  for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x + 1; i < n; i += (u64)gridDim.x * blockDim.x)
    bad |= keys[i] < keys[i - 1];
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) *flag = 1u;
}

}  // namespace

void launch_simd_widths(const uint16_t* widths, u64 n, Arena* arena, cudaStream_t s) {
  if (n == 0) return;
  const u64 blocks = std::min<u64>((n + 8 * 256 - 1) / (8 * 256), 152ull * 8);
  k_simd_widths<<<(unsigned)blocks, 256, 0, s>>>(widths, n, arena);
  count_launches(1);
}

void launch_keys_sorted(const u64* keys, u64 n, u32* flag, cudaStream_t s) {
  if (n < 2) return;
  const u64 blocks = std::min<u64>((n + 255) / 256, 152ull * 8);
  k_keys_sorted<<<(unsigned)blocks, 256, 0, s>>>(keys, n, flag);
  count_launches(1);
}

void launch_instr_runs(const RunBatchArgs& a, cudaStream_t s) {
  if (a.n_runs == 0) return;
  int mode;
  size_t smem;
  const size_t bins = (size_t)a.n_opcodes + 1;
  if (bins * kInWarps * 4 <= 48 * 1024) { mode = 0; smem = bins * kInWarps * 4; }
  else if (bins * 4 <= 96 * 1024) { mode = 1; smem = bins * 4; }
  else { mode = 2; smem = 0; }
  u64 blocks = (a.n_runs + kInWarps - 1) / kInWarps;
  if (blocks > 152ull * 16) blocks = 152ull * 16;
  if (mode == 0) k_instr_runs<0><<<(unsigned)blocks, kInThreads, smem, s>>>(a);
  else if (mode == 1) k_instr_runs<1><<<(unsigned)blocks, kInThreads, smem, s>>>(a);
  else k_instr_runs<2><<<(unsigned)blocks, kInThreads, smem, s>>>(a);
  count_launches(1);
}

void init_instr_attributes() {
  cudaFuncSetAttribute(k_instr_runs<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  cudaFuncSetAttribute(k_instr_runs<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
}

void launch_instr_combine(const CombineArgs& a, cudaStream_t s) {
  if (a.n_runs == 0) return;
  u64 blocks = (a.n_runs + 255) / 256;
  if (blocks > 152ull * 4) blocks = 152ull * 4;
  k_instr_combine<<<(unsigned)blocks, 256, 0, s>>>(a);
  count_launches(1);
}

}  // namespace aiwc
