// Host side of the C ABI declared in include/aiwc.h: handle lifecycle,
// staging of host pushes, and the end-of-invocation pipeline.
//
// Pushes run their ingest kernels immediately on the handle's stream (the
// memory ingest counts each event's superblock and writes slot words, or sort
// words in the sort plan; the branch ingest writes branch words; the
// instruction kernel reduces each run at once), so host-to-device copies of
// one chunk overlap the ingest of the previous one. aiwc_compute then reads
// the ingest-time counters once to plan, reduces the memory events on the
// handle's stream and (hash plan) the branch events on a side stream at the
// same time, finalises and copies one fixed-size result back.
#include <algorithm>
#include <atomic>
#include <cstddef>
#include <functional>
#include <mutex>
#include <new>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "aiwc_internal.cuh"
#include "route.h"

using namespace aiwc;

namespace {

thread_local std::string g_last_error;
std::atomic<unsigned long long> g_epoch{0};
constexpr size_t kStageBytes = 64ull << 20;
constexpr size_t kPendingOps = 1ull << 24;
constexpr size_t kPendingRuns = 1ull << 16;

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int d) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != d) cudaSetDevice(d);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

inline u64 ntiles_of(u64 n) { return (n + kTile - 1) / kTile; }

enum Stage {
  kStMemIngest, kStBrIngest, kStInstrRuns, kStMemSort, kStMemScatter, kStMemLevels, kStBrSort, kStWindows,
  kStPatSort, kStPatRuns, kStRunSort, kStCombine, kStFinalize, kStMemExpand, kNumStages
};
const char* const kStageNames[kNumStages] = {"mem_ingest", "branch_ingest", "instr_runs", "mem_sort",
                                             "mem_scatter", "mem_levels", "branch_sort", "windows",
                                             "pattern_sort", "pattern_runs", "run_sort", "run_combine",
                                             "finalize", "mem_expand"};

}  // namespace

void aiwc::set_last_error(const std::string& msg) { g_last_error = msg; }

// Page-locked host memory for the partition buffers (host-to-device copies
// run at link speed from it); resize leaves new elements uninitialised.
template <typename T>
struct PinnedAlloc {
  using value_type = T;
  PinnedAlloc() = default;
  template <typename U>
  PinnedAlloc(const PinnedAlloc<U>&) {}
  T* allocate(size_t n) {
    void* p = nullptr;
    if (cudaMallocHost(&p, n * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      throw std::bad_alloc();
    }
    return static_cast<T*>(p);
  }
  void deallocate(T* p, size_t) { cudaFreeHost(p); }
  template <typename U>
  void construct(U* p) {
    ::new (static_cast<void*>(p)) U;
  }
  template <typename U, typename... A>
  void construct(U* p, A&&... a) {
    ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
  }
  bool operator==(const PinnedAlloc&) const { return true; }
  bool operator!=(const PinnedAlloc&) const { return false; }
};
template <typename T>
using pinned_vector = std::vector<T, PinnedAlloc<T>>;

struct aiwc_handle {
  aiwc_config cfg;
  cudaStream_t stream = nullptr;
  cudaStream_t copy_stream = nullptr;
  // the branch reduction runs beside the memory reduction (hash plan)
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr};
  cudaEvent_t ev_free[2] = {nullptr, nullptr};
  int stage_next = 0;
  int sm_count = 152;
  bool broken = false;
  std::string err;
  Arena* arena = nullptr;
  Result* d_result = nullptr;
  Result* h_result = nullptr;
  uint64_t* d_hist = nullptr;
  uint64_t* h_hist = nullptr;
  u32* wi_bitmap = nullptr;
  u64 max_wi = 0;
  size_t bytes = 0;
  DevBuf mem_a, mem_b, br_a, br_b, pat_a, pat_b, rk_a, rk_b, run_sum, over_a, over_b, counts, bsums, tiles;
  DevBuf br_c;                  // branch events as site << 1 | taken, two bytes each (the site counting sort reads these)
  DevBuf stage[2];
  DevBuf desc;
  // byte-granular addresses: the tile offsets and byte counts of a batch of chunks
  DevBuf exp_meta;
  u64* h_exp = nullptr;  // pinned copy of the batch's byte counts
  // superblock table of the hash plan (sized for the next invocation)
  DevBuf sbt, sbt_scan;
  u64 sbt_cap = 0;       // slots currently allocated
  u64 sbt_want = 1ull << 20;
  u64 sbt_floor = 0;     // slots an overflowing invocation asked for (the automatic size never goes below)
  int inv_plan = 0;      // plan 0: this invocation's memory plan, chosen by its first memory push (1 sort, 2 hash)
  DevState* h_state = nullptr;  // pinned copy of the device counters
  DevBuf sites;                 // the per-site path's list of long sites (the site list lives in pat_b)
  bool last_plan_hash = false;
  u64 n_mem = 0, n_br = 0, n_runs = 0;
  u32 br_pushes = 0;    // branch ingest launches in this invocation (orders the sortedness check)
  u64 epoch = 0;        // changes whenever a device buffer of the handle moves (keys cached graphs)
  // sizes fixed by prepare() for the current compute
  u64 c_over_cap = 0, c_sites_cap = 0;
  size_t c_site_off = 0;        // the site list's byte offset in pat_b (after the counting sort's chunk sums)
  size_t c_low_off = 0;
  u64 value_bound = 0;  // bound on ITB / IPT values >= kValDense (each uses kValDense instructions)
  // run tables of host run pushes, one per staging buffer (pinned, so that
  // their copies are asynchronous)
  pinned_vector<unsigned char> tab_pin[2];
  // pending single-run pushes (host data, or device pointers)
  std::vector<uint16_t> pend_ops;
  std::vector<uint32_t> pend_wi;
  std::vector<uint64_t> pend_off, pend_len;
  bool pend_device = false;
  // optional stage timing
  bool timing = false;
  std::vector<cudaEvent_t> event_pool;
  struct Interval { int stage; cudaEvent_t a, b; };
  std::vector<Interval> intervals;
  double stage_acc[kNumStages] = {0};
  double stage_last[kNumStages] = {0};
  // partitioned invocations: pushed events held on the host per partition
  struct PartBuf {
    pinned_vector<uint8_t> mem;    // 16-byte memory events
    pinned_vector<uint64_t> br;    // 8-byte branch events
    pinned_vector<uint16_t> ops;
    pinned_vector<uint32_t> run_wi;
    pinned_vector<uint64_t> run_off, run_len;
    pinned_vector<uint16_t> widths;
    void clear() {  // keeps the capacity for the next invocation
      mem.clear();
      br.clear();
      ops.clear();
      run_wi.clear();
      run_off.clear();
      run_len.clear();
      widths.clear();
    }
  };
  std::vector<PartBuf> parts;      // empty when not partitioned
  bool replaying = false;          // compute is pushing one partition to the device
  u32 part_err = 0;                // routing found an invalid run (reported by compute)
  Arena* total = nullptr;          // the partitions' merged distributions
  DevBuf over_total;
  // sharded invocations: this rank's exported distributions, held until the
  // caller takes them; staging for the blobs being merged
  std::vector<uint8_t> shard_blob;
  DevBuf shard_tmp;
  // defer_pushes: device pushes recorded in order, ingested at compute time
  struct Deferred {
    int kind;  // 0 memory events, 1 branch events, 2 instruction runs, 3 widths
    const void* p[4];
    size_t n, n_ops;
  };
  std::vector<Deferred> deferred;
  bool flushing = false;  // the recorded pushes are being ingested
};

namespace {

aiwc_status fail(aiwc_handle* h, aiwc_status st, const std::string& msg, bool breaks = true) {
  if (h) {
    h->err = msg;
    if (breaks && st != AIWC_EINVAL) h->broken = true;
  }
  g_last_error = msg;
  return st;
}

aiwc_status cuda_fail(aiwc_handle* h, const char* what, cudaError_t e) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
  return fail(h, e == cudaErrorMemoryAllocation ? AIWC_ENOMEM : AIWC_ECUDA, buf);
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(h, #call, e_);    \
  } while (0)

// Brackets one stage with CUDA events on the handle's stream when timing is on.
struct StageScope {
  aiwc_handle* h;
  int stage;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  bool range = false;  // an NVTX range named after the stage (seen by nsys / ncu --nvtx)
  cudaEvent_t take() {
    cudaEvent_t e = nullptr;
    if (!h->event_pool.empty()) {
      e = h->event_pool.back();
      h->event_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      e = nullptr;
    }
    return e;
  }
  // s: the stream the stage's kernels go to (the handle's stream by default)
  StageScope(aiwc_handle* hh, int st, cudaStream_t ss = nullptr) : h(hh), stage(st), s(ss ? ss : hh->stream) {
    nvtxRangePushA(kStageNames[st]);
    range = true;
    if (!h->timing) return;
    a = take();
    b = take();
    if (a) cudaEventRecord(a, s);
  }
  void end() {
    if (range) {
      nvtxRangePop();
      range = false;
    }
    if (!a || !b) return;
    cudaEventRecord(b, s);
    h->intervals.push_back({stage, a, b});
    a = b = nullptr;
  }
  ~StageScope() { end(); }
  StageScope(const StageScope&) = delete;  // one push and one pop per range
  StageScope& operator=(const StageScope&) = delete;
};

// After the stream is synchronised: fold the recorded intervals into stage times.
void collect_stage_times(aiwc_handle* h) {
  for (auto& iv : h->intervals) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, iv.a, iv.b) == cudaSuccess) h->stage_acc[iv.stage] += ms;
    else cudaGetLastError();
    h->event_pool.push_back(iv.a);
    h->event_pool.push_back(iv.b);
  }
  h->intervals.clear();
  for (int i = 0; i < kNumStages; ++i) {
    h->stage_last[i] = h->stage_acc[i];
    h->stage_acc[i] = 0.0;
  }
}

aiwc_status ensure(aiwc_handle* h, DevBuf& b, size_t bytes, bool preserve) {
  if (bytes <= b.cap) return AIWC_OK;
  size_t want = std::max(bytes, b.cap + b.cap / 2);
  want = (want + 255) & ~size_t(255);
  if (h->cfg.hbm_budget && h->bytes - b.cap + want > h->cfg.hbm_budget) {
    want = bytes;
    if (h->bytes - b.cap + want > h->cfg.hbm_budget)
      return fail(h, AIWC_ENOMEM, "device scratch would exceed hbm_budget", false);
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, AIWC_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e), false);
  }
  if (b.p) {
    if (preserve) CK(cudaMemcpyAsync(p, b.p, b.cap, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaFree(b.p));
  }
  h->bytes = h->bytes - b.cap + want;
  b.p = p;
  b.cap = want;
  h->epoch = ++g_epoch;
  return AIWC_OK;
}

#define ENSURE(buf, bytes, keep)                              \
  do {                                                        \
    aiwc_status s_ = ensure(h, buf, bytes, keep);             \
    if (s_ != AIWC_OK) return s_;                             \
  } while (0)

aiwc_status ensure_bitmap(aiwc_handle* h) {
  if (h->wi_bitmap) return AIWC_OK;
  const size_t words = (size_t)((h->max_wi + 31) / 32);
  if (h->cfg.hbm_budget && h->bytes + words * 4 > h->cfg.hbm_budget)
    return fail(h, AIWC_ENOMEM, "work-item bitmap would exceed hbm_budget", false);
  CK(cudaMalloc(&h->wi_bitmap, words * 4));
  CK(cudaMemsetAsync(h->wi_bitmap, 0, words * 4, h->stream));
  h->bytes += words * 4;
  return AIWC_OK;
}

template <typename Launch>
aiwc_status staged_copy(aiwc_handle* h, const void* src, size_t bytes, size_t unit, Launch launch) {
  // Double-buffered: the copy of chunk k+1 overlaps the ingest of chunk k.
  const size_t per = (kStageBytes / unit) * unit;
  for (int i = 0; i < 2; ++i) ENSURE(h->stage[i], kStageBytes, false);
  cudaEvent_t last = nullptr;
  for (size_t off = 0; off < bytes; off += per) {
    const size_t nb = std::min(per, bytes - off);
    const int k = h->stage_next;
    h->stage_next ^= 1;
    CK(cudaStreamWaitEvent(h->copy_stream, h->ev_free[k], 0));
    CK(cudaMemcpyAsync(h->stage[k].p, (const char*)src + off, nb, cudaMemcpyHostToDevice, h->copy_stream));
    CK(cudaEventRecord(h->ev_copied[k], h->copy_stream));
    CK(cudaStreamWaitEvent(h->stream, h->ev_copied[k], 0));
    launch(h->stage[k].p, off / unit, nb / unit);
    CK(cudaGetLastError());
    CK(cudaEventRecord(h->ev_free[k], h->stream));
    last = h->ev_copied[k];
  }
  if (last) CK(cudaEventSynchronize(last));  // the caller may reuse its buffer on return
  return AIWC_OK;
}

bool use_hash(const aiwc_handle* h) { return h->cfg.plan == 2 || (h->cfg.plan == 0 && h->inv_plan != 1); }

// Automatic planning (plan 0), per invocation, from its first memory push of
// n events: up to kAutoSortMax events take the sort plan (its fixed cost, a
// few radix passes over a small array, is below the hash plan's table clear
// and scan); larger ones the hash plan with a table of at least n slots
// (table_slots 0: a single push cannot overflow it), between 2^12 and 2^20
// and never below what an earlier overflow asked for. The table only grows
// between invocations.
constexpr u64 kAutoSortMax = 1ull << 15;
void auto_plan(aiwc_handle* h, u64 n) {
  if (h->cfg.plan != 0) return;
  h->inv_plan = n <= kAutoSortMax ? 1 : 2;
  if (h->inv_plan == 2 && !h->cfg.table_slots) {
    u64 want = 1ull << 12;
    while (want < n && want < kMaxHashSlots) want <<= 1;
    h->sbt_want = std::max<u64>(want, h->sbt_floor);
  }
}

SbTable table_view(aiwc_handle* h) {
  SbTable t;
  char* p = (char*)h->sbt.p;
  const u64 C = h->sbt_cap;
  t.keys = (u64*)p;
  t.cnt = (u32*)(p + 8 * C);
  t.off = (u32*)(p + kSbtClearBytes * C);
  t.mask = C - 1;
  return t;
}

// Allocates (or regrows, between invocations) the superblock table; cleared.
aiwc_status ensure_table(aiwc_handle* h) {
  if (h->sbt_cap >= h->sbt_want && h->sbt.p) return AIWC_OK;
  if (h->n_mem) return AIWC_OK;  // never resize in the middle of an invocation
  const u64 C = std::min<u64>(h->sbt_want, kMaxHashSlots);
  aiwc_status s = ensure(h, h->sbt, kSbtBytes * C, false);
  if (s != AIWC_OK) return s;
  s = ensure(h, h->sbt_scan, 4 * sbt_scan_words(C), false);
  if (s != AIWC_OK) return s;
  h->sbt_cap = C;
  CK(cudaMemsetAsync(h->sbt.p, 0, kSbtClearBytes * C, h->stream));
  return AIWC_OK;
}

aiwc_status check_usable(aiwc_handle* h) {
  if (!h) return fail(nullptr, AIWC_EINVAL, "null handle");
  if (h->broken) return AIWC_ESTATE;
  return AIWC_OK;
}

// Overflow entries an invocation can append: group sizes >= kCocDense per
// level, large site and pattern counts, opcode counts, large ITB / IPT values.
u64 over_bound_sizes(u32 n_opcodes, u64 n_mem, u64 n_br, u64 n_runs, u64 value_bound) {
  return (u64)kLevels * (n_mem / kCocDense + 2) + (n_br / kCocDense + 2) + 2 * (n_br / kValDense + 2) +
         (u64)n_opcodes + 2 * value_bound + 2 * (n_runs + 2) + 256;
}

u64 over_bound(const aiwc_handle* h, u64 n_mem, u64 n_br, u64 n_runs) {
  return over_bound_sizes(h->cfg.n_opcodes, n_mem, n_br, n_runs, h->value_bound);
}

aiwc_status runs_device(aiwc_handle* h, const u32* run_wi, const u64* run_off, const u64* run_len, size_t n_runs,
                        const uint16_t* ops, u64 n_ops, u64 ops_total) {
  if (h->n_runs + n_runs >= (1ull << 32))
    return fail(h, AIWC_EINVAL, "more than 2^32 - 1 instruction runs in one invocation", false);
  ENSURE(h->rk_a, (h->n_runs + n_runs) * 8, true);
  ENSURE(h->run_sum, (h->n_runs + n_runs) * 32, true);
  h->value_bound += ops_total / kValDense + 2;
  ENSURE(h->over_a, over_bound(h, h->n_mem, h->n_br, h->n_runs + n_runs) * 8, true);
  aiwc_status s = ensure_bitmap(h);
  if (s != AIWC_OK) return s;
  RunBatchArgs a;
  a.ops = ops;
  a.n_ops = n_ops;
  a.run_wi = run_wi;
  a.run_off = run_off;
  a.run_len = run_len;
  a.n_runs = n_runs;
  a.seq_base = h->n_runs;
  a.n_opcodes = h->cfg.n_opcodes;
  a.run_keys = (u64*)h->rk_a.p;
  a.run_sum = (u64*)h->run_sum.p;
  a.wi_bitmap = h->wi_bitmap;
  a.max_wi = h->max_wi;
  a.opc_hist = (u64*)h->d_hist;
  a.over = (u64*)h->over_a.p;
  a.over_cap = h->over_a.cap / 8;
  a.arena = h->arena;
  StageScope scope(h, kStInstrRuns);
  launch_instr_runs(a, h->stream);
  CK(cudaGetLastError());
  h->n_runs += n_runs;
  return AIWC_OK;
}

// Host run tables: copied in batches whose opcode span fits a stage buffer.
// Each batch's run table is built in the pinned table of its staging buffer
// while the previous batch is still being copied; the host waits only before
// it rewrites a table and, at the end, for the last copy (the caller may
// reuse its opcodes when the call returns).
aiwc_status runs_host(aiwc_handle* h, const uint32_t* run_wi, const uint64_t* run_off, const uint64_t* run_len,
                      size_t n_runs, const uint16_t* ops, size_t n_ops) {
  for (size_t r = 0; r < n_runs; ++r)
    if (run_off[r] > n_ops || run_len[r] > n_ops - run_off[r])
      return fail(h, AIWC_EINVAL, "instruction run reaches past its opcode array", false);
  size_t r0 = 0;
  int last = -1;
  while (r0 < n_runs) {
    u64 lo = run_off[r0], hi = run_off[r0] + run_len[r0];
    size_t r1 = r0 + 1;
    while (r1 < n_runs) {
      const u64 nlo = std::min<u64>(lo, run_off[r1]), nhi = std::max<u64>(hi, run_off[r1] + run_len[r1]);
      const size_t need = ((nhi - nlo) * 2 + 15) / 16 * 16 + (r1 + 1 - r0) * 24;
      if (need > kStageBytes) break;
      lo = nlo;
      hi = nhi;
      ++r1;
    }
    const size_t nb = r1 - r0;
    const size_t ops_bytes = ((hi - lo) * 2 + 15) / 16 * 16;
    const size_t need = ops_bytes + nb * 24;
    const int k = h->stage_next;
    h->stage_next ^= 1;
    ENSURE(h->stage[k], std::max(need, kStageBytes), false);
    CK(cudaEventSynchronize(h->ev_copied[k]));  // this table's previous copy is done
    auto& tab = h->tab_pin[k];
    if (tab.size() < nb * 24) tab.resize(nb * 24);
    u64* offs = (u64*)tab.data();
    u64* lens = offs + nb;
    u32* wis = (u32*)(lens + nb);
    for (size_t i = 0; i < nb; ++i) {
      offs[i] = run_off[r0 + i] - lo;
      lens[i] = run_len[r0 + i];
      wis[i] = run_wi[r0 + i];
    }
    char* base = (char*)h->stage[k].p;
    CK(cudaStreamWaitEvent(h->copy_stream, h->ev_free[k], 0));
    if (hi > lo) CK(cudaMemcpyAsync(base, ops + lo, (hi - lo) * 2, cudaMemcpyHostToDevice, h->copy_stream));
    CK(cudaMemcpyAsync(base + ops_bytes, tab.data(), nb * 24, cudaMemcpyHostToDevice, h->copy_stream));
    CK(cudaEventRecord(h->ev_copied[k], h->copy_stream));
    CK(cudaStreamWaitEvent(h->stream, h->ev_copied[k], 0));
    aiwc_status s = runs_device(h, (const u32*)(base + ops_bytes + nb * 16), (const u64*)(base + ops_bytes),
                                (const u64*)(base + ops_bytes + nb * 8), nb, (const uint16_t*)base, hi - lo, hi - lo);
    if (s != AIWC_OK) return s;
    CK(cudaEventRecord(h->ev_free[k], h->stream));
    last = k;
    r0 = r1;
  }
  if (last >= 0) CK(cudaEventSynchronize(h->ev_copied[last]));  // the caller may reuse ops
  return AIWC_OK;
}

aiwc_status flush_pending(aiwc_handle* h) {
  if (h->pend_wi.empty()) return AIWC_OK;
  aiwc_status s;
  if (!h->pend_device) {
    s = runs_host(h, h->pend_wi.data(), h->pend_off.data(), h->pend_len.data(), h->pend_wi.size(),
                  h->pend_ops.data(), h->pend_ops.size());
  } else {
    // descriptors of device runs: offsets are element addresses from 0
    const size_t nb = h->pend_wi.size();
    const int k = h->stage_next;
    h->stage_next ^= 1;
    ENSURE(h->stage[k], std::max(nb * 24, kStageBytes), false);
    std::vector<unsigned char> tab(nb * 24);
    memcpy(tab.data(), h->pend_off.data(), nb * 8);
    memcpy(tab.data() + nb * 8, h->pend_len.data(), nb * 8);
    memcpy(tab.data() + nb * 16, h->pend_wi.data(), nb * 4);
    char* base = (char*)h->stage[k].p;
    CK(cudaStreamWaitEvent(h->copy_stream, h->ev_free[k], 0));
    CK(cudaMemcpyAsync(base, tab.data(), nb * 24, cudaMemcpyHostToDevice, h->copy_stream));
    CK(cudaEventRecord(h->ev_copied[k], h->copy_stream));
    CK(cudaStreamWaitEvent(h->stream, h->ev_copied[k], 0));
    u64 total = 0;
    for (u64 l : h->pend_len) total += l;
    s = runs_device(h, (const u32*)(base + nb * 16), (const u64*)base, (const u64*)(base + nb * 8), nb,
                    (const uint16_t*)nullptr, ~0ull, total);
    if (s == AIWC_OK) {
      CK(cudaEventRecord(h->ev_free[k], h->stream));
      CK(cudaEventSynchronize(h->ev_copied[k]));
    }
  }
  h->pend_ops.clear();
  h->pend_wi.clear();
  h->pend_off.clear();
  h->pend_len.clear();
  return s;
}

void release(aiwc_handle* h, DevBuf& b) {
  if (b.p) cudaFree(b.p);
  h->bytes -= b.cap;
  b.p = nullptr;
  b.cap = 0;
}

// The device state back to the start of an invocation. clear_bitmap: the
// work-item bitmap may hold marks (a finalisation counts and clears it).
aiwc_status reset_device_state(aiwc_handle* h, cudaStream_t st, bool clear_bitmap) {
  if (clear_bitmap && h->wi_bitmap) launch_wi_clear(h->wi_bitmap, h->arena, st);
  launch_reset(h->arena, (u64*)h->d_hist, h->cfg.n_opcodes, h->sbt.p ? (u64*)h->sbt.p : nullptr,
               h->sbt.p ? kSbtClearBytes * h->sbt_cap / 8 : 0, st);
  CK(cudaGetLastError());
  return AIWC_OK;
}

// ---------------------------------------------------------------- partitioned invocations

bool routing(const aiwc_handle* h) { return !h->parts.empty() && !h->replaying; }

// Host copy of caller data (device pointers are read back first).
template <typename T>
aiwc_status host_view(aiwc_handle* h, const T* p, size_t n, int on_device, std::vector<T>* tmp, const T** out) {
  if (!on_device) {
    *out = p;
    return AIWC_OK;
  }
  tmp->resize(n);
  CK(cudaMemcpy(tmp->data(), p, n * sizeof(T), cudaMemcpyDeviceToHost));
  *out = tmp->data();
  return AIWC_OK;
}

// Memory events go with their superblock (space, address >> 11): every
// skip-level group lies inside one superblock, so a partition's groups are
// whole.
aiwc_status route_mem(aiwc_handle* h, const aiwc_mem_event* ev, size_t n, int on_device) {
  std::vector<aiwc_mem_event> tmp;
  const aiwc_mem_event* e = nullptr;
  aiwc_status s = host_view(h, ev, n, on_device, &tmp, &e);
  if (s != AIWC_OK) return s;
  std::vector<aiwc_mem_event> split;
  if (h->cfg.byte_addresses && split_at_superblocks(e, n, &split)) {
    e = split.data();
    n = split.size();
  }
  const u32 P = (u32)h->parts.size();
  stable_partition(
      n, P, [&](size_t i) { return part_of(mem_route_key(e[i]), P); },
      [](size_t) { return (uint64_t)1; },
      [&](u32 p, uint64_t len) {
        auto& m = h->parts[p].mem;
        if (len) m.resize(16 * len);
        return (uint64_t)(m.size() / 16);
      },
      [&](size_t i, u32 p, uint64_t at) { memcpy(h->parts[p].mem.data() + 16 * at, e + i, 16); });
  return AIWC_OK;
}

// Branch events go with their site (histories are per site).
aiwc_status route_branch(aiwc_handle* h, const aiwc_branch_event* ev, size_t n, int on_device) {
  std::vector<aiwc_branch_event> tmp;
  const aiwc_branch_event* e = nullptr;
  aiwc_status s = host_view(h, ev, n, on_device, &tmp, &e);
  if (s != AIWC_OK) return s;
  const u32 P = (u32)h->parts.size();
  stable_partition(
      n, P, [&](size_t i) { return part_of(e[i].site, P); }, [](size_t) { return (uint64_t)1; },
      [&](u32 p, uint64_t len) {
        auto& b = h->parts[p].br;
        if (len) b.resize(len);
        return (uint64_t)b.size();
      },
      [&](size_t i, u32 p, uint64_t at) { memcpy(h->parts[p].br.data() + at, e + i, 8); });
  return AIWC_OK;
}

// Instruction runs go with their work-item (ITB chains per work-item).
aiwc_status route_runs(aiwc_handle* h, const uint32_t* run_wi, const uint64_t* run_off, const uint64_t* run_len,
                       size_t n_runs, const uint16_t* ops, size_t n_ops, int on_device) {
  std::vector<uint32_t> twi;
  std::vector<uint64_t> toff, tlen;
  std::vector<uint16_t> tops;
  const uint32_t* wi = nullptr;
  const uint64_t *off = nullptr, *len = nullptr;
  const uint16_t* op = nullptr;
  aiwc_status s;
  if ((s = host_view(h, run_wi, n_runs, on_device, &twi, &wi)) != AIWC_OK ||
      (s = host_view(h, run_off, n_runs, on_device, &toff, &off)) != AIWC_OK ||
      (s = host_view(h, run_len, n_runs, on_device, &tlen, &len)) != AIWC_OK ||
      (s = host_view(h, ops, n_ops, on_device, &tops, &op)) != AIWC_OK)
    return s;
  for (size_t r = 0; r < n_runs; ++r)
    if (off[r] > n_ops || len[r] > n_ops - off[r]) {
      h->part_err |= kErrRun;
      return AIWC_OK;  // reported by compute, like the unpartitioned path
    }
  const u32 P = (u32)h->parts.size();
  // runs first (one unit each), then their opcodes (len units each), both stable
  std::vector<uint64_t> run_at(n_runs);
  stable_partition(
      n_runs, P, [&](size_t r) { return part_of(wi[r], P); }, [](size_t) { return (uint64_t)1; },
      [&](u32 p, uint64_t n) {
        auto& pb = h->parts[p];
        if (n) {
          pb.run_wi.resize(n);
          pb.run_off.resize(n);
          pb.run_len.resize(n);
        }
        return (uint64_t)pb.run_wi.size();
      },
      [&](size_t r, u32 p, uint64_t at) {
        h->parts[p].run_wi[at] = wi[r];
        h->parts[p].run_len[at] = len[r];
        run_at[r] = at;
      });
  stable_partition(
      n_runs, P, [&](size_t r) { return part_of(wi[r], P); }, [&](size_t r) { return len[r]; },
      [&](u32 p, uint64_t n) {
        auto& o = h->parts[p].ops;
        if (n) o.resize(n);
        return (uint64_t)o.size();
      },
      [&](size_t r, u32 p, uint64_t at) {
        h->parts[p].run_off[run_at[r]] = at;
        memcpy(h->parts[p].ops.data() + at, op + off[r], len[r] * 2);
      });
  return AIWC_OK;
}

aiwc_status route_widths(aiwc_handle* h, const uint16_t* w, size_t n, int on_device) {
  std::vector<uint16_t> tmp;
  const uint16_t* p = nullptr;
  aiwc_status s = host_view(h, w, n, on_device, &tmp, &p);
  if (s != AIWC_OK) return s;
  auto& v = h->parts[0].widths;  // the SIMD statistics add over any split
  v.insert(v.end(), p, p + n);
  return AIWC_OK;
}

aiwc_status compute_partitioned(aiwc_handle* h, aiwc_metrics* out);
aiwc_status finalize_merged(aiwc_handle* h, u64 total_cap, aiwc_metrics* out, uint64_t* user_hist);

// Runs a routing step; page-locked host memory running out is AIWC_ENOMEM.
template <typename F>
aiwc_status routed(aiwc_handle* h, F&& f) {
  try {
    return f();
  } catch (const std::bad_alloc&) {
    return fail(h, AIWC_ENOMEM, "page-locked host memory for the partitions is exhausted", false);
  }
}

}  // namespace

namespace {

// defer_pushes: does this device push wait for the compute?
bool defers(const aiwc_handle* h, int on_device) {
  return h->cfg.defer_pushes && on_device && !h->flushing && h->parts.empty();
}

aiwc_status record(aiwc_handle* h, int kind, const void* p0, const void* p1, const void* p2, const void* p3,
                   size_t n, size_t n_ops) {
  aiwc_handle::Deferred d;
  d.kind = kind;
  d.p[0] = p0;
  d.p[1] = p1;
  d.p[2] = p2;
  d.p[3] = p3;
  d.n = n;
  d.n_ops = n_ops;
  h->deferred.push_back(d);
  return AIWC_OK;
}

}  // namespace

// Ingests the recorded device pushes in their order on h->stream.
aiwc_status flush_deferred(aiwc_handle* h) {
  if (h->deferred.empty() || h->flushing) return AIWC_OK;
  h->flushing = true;
  std::vector<aiwc_handle::Deferred> list;
  list.swap(h->deferred);
  aiwc_status s = AIWC_OK;
  for (const auto& d : list) {
    switch (d.kind) {
      case 0: s = aiwc_push_mem(h, static_cast<const aiwc_mem_event*>(d.p[0]), d.n, 1); break;
      case 1: s = aiwc_push_branch(h, static_cast<const aiwc_branch_event*>(d.p[0]), d.n, 1); break;
      case 2:
        s = aiwc_push_instr_runs(h, static_cast<const uint32_t*>(d.p[0]), static_cast<const uint64_t*>(d.p[1]),
                                 static_cast<const uint64_t*>(d.p[2]), d.n, static_cast<const uint16_t*>(d.p[3]),
                                 d.n_ops, 1);
        break;
      default: s = aiwc_push_widths(h, static_cast<const uint16_t*>(d.p[0]), d.n, 1); break;
    }
    if (s != AIWC_OK) break;
  }
  h->flushing = false;
  return s;
}

extern "C" {

void aiwc_config_default(aiwc_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->device = 0;
  c->cuda_stream = nullptr;
  c->history_len = 16;
  c->cover_num = 9;
  c->cover_den = 10;
  c->n_opcodes = 65535;
  c->space_mask = 0xF;
  c->precision = 0;
  c->plan = 0;
  c->max_work_items = 0;
  c->hbm_budget = 0;
  c->table_slots = 0;
}

aiwc_status aiwc_create(const aiwc_config* cfg, aiwc_handle** out) {
  if (!cfg || !out) return fail(nullptr, AIWC_EINVAL, "null config or output pointer");
  *out = nullptr;
  if (cfg->history_len < 1 || cfg->history_len > 31) return fail(nullptr, AIWC_EINVAL, "history_len must be 1..31");
  if (cfg->cover_den == 0 || cfg->cover_num == 0 || cfg->cover_num > cfg->cover_den)
    return fail(nullptr, AIWC_EINVAL, "coverage fraction must be in (0, 1]");
  if (cfg->n_opcodes == 0 || cfg->n_opcodes > 65535) return fail(nullptr, AIWC_EINVAL, "n_opcodes must be 1..65535");
  if (cfg->precision > 1 || cfg->plan > 2) return fail(nullptr, AIWC_EINVAL, "unknown precision or plan");
  if (cfg->max_work_items > (1ull << 32)) return fail(nullptr, AIWC_EINVAL, "max_work_items must be <= 2^32");
  if (cfg->table_slots && ((cfg->table_slots & (cfg->table_slots - 1)) || cfg->table_slots < 64 ||
                           cfg->table_slots > (1ull << 30)))
    return fail(nullptr, AIWC_EINVAL, "table_slots must be a power of two in [64, 2^30]");
  if (cfg->partitions > 256 || (cfg->partitions & (cfg->partitions - 1)))
    return fail(nullptr, AIWC_EINVAL, "partitions must be 0 or a power of two <= 256");
  if (cfg->byte_addresses > 1 || cfg->history_scope > 1)
    return fail(nullptr, AIWC_EINVAL, "byte_addresses and history_scope must be 0 or 1");
  if (cfg->defer_pushes > 1 || (cfg->defer_pushes && cfg->partitions > 1))
    return fail(nullptr, AIWC_EINVAL, "defer_pushes must be 0 or 1, and 0 with partitions");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
    cudaGetLastError();
    return fail(nullptr, AIWC_ECUDA, "no such CUDA device");
  }
  DeviceGuard g(cfg->device);
  aiwc_handle* h = new aiwc_handle();
  h->cfg = *cfg;
  h->cfg.space_mask &= 0xF;
  h->stream = (cudaStream_t)cfg->cuda_stream;
  h->max_wi = cfg->max_work_items ? cfg->max_work_items : (1ull << 32);
  h->sbt_want = cfg->table_slots ? cfg->table_slots : (1ull << 20);
  if (cfg->partitions > 1) h->parts.resize(cfg->partitions);
  auto bail = [&](aiwc_status s) {
    aiwc_destroy(h);
    return s;
  };
  cudaError_t e;
  if ((e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, cfg->device)) != cudaSuccess)
    return bail(cuda_fail(nullptr, "cudaDeviceGetAttribute", e));
  if ((e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(cuda_fail(nullptr, "cudaStreamCreate", e));
  if ((e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming)) != cudaSuccess)
    return bail(cuda_fail(nullptr, "cudaEventCreate", e));
  for (int i = 0; i < 2; ++i) {
    if ((e = cudaEventCreateWithFlags(&h->ev_copied[i], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->ev_free[i], cudaEventDisableTiming)) != cudaSuccess)
      return bail(cuda_fail(nullptr, "cudaEventCreate", e));
  }
  // the opcode histogram follows the result, on the device and on the host
  if ((e = cudaMalloc(&h->arena, sizeof(Arena))) != cudaSuccess ||
      (e = cudaMalloc(&h->d_result, result_bytes(cfg->n_opcodes))) != cudaSuccess ||
      (e = cudaMallocHost(&h->h_result, result_bytes(cfg->n_opcodes))) != cudaSuccess ||
      (e = cudaMallocHost(&h->h_state, sizeof(DevState))) != cudaSuccess)
    return bail(cuda_fail(nullptr, "allocation", e));
  h->d_hist = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(h->d_result) + kHistOffset);
  h->h_hist = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(h->h_result) + kHistOffset);
  h->bytes = sizeof(Arena) + result_bytes(cfg->n_opcodes);
  init_branch_attributes();
  init_instr_attributes();
  if (reset_device_state(h, h->stream, true) != AIWC_OK) return bail(fail(nullptr, AIWC_ECUDA, h->err));
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return bail(cuda_fail(nullptr, "initial reset", e));
  *out = h;
  return AIWC_OK;
}

}  // extern "C"

namespace {

// Buffers and common arguments of an ingest that adds n accesses to the
// current invocation.
aiwc_status ingest_args(aiwc_handle* h, size_t n, MemIngestArgs* a) {
  aiwc_status s;
  if (h->n_mem == 0) auto_plan(h, n);
  ENSURE(h->mem_a, (h->n_mem + n) * 8, true);
  if ((s = ensure_bitmap(h)) != AIWC_OK) return s;
  if (use_hash(h) && (s = ensure_table(h)) != AIWC_OK) return s;
  a->use_tab = use_hash(h) && h->sbt_cap ? 1 : 0;
  if (a->use_tab) {
    ENSURE(h->mem_b, (h->n_mem + n) * 8, true);  // slot words and ranks
    a->tab = table_view(h);
    a->slotw = (u64*)h->mem_b.p;
    a->spill = (u64*)h->mem_a.p;
  }
  a->space_mask = h->cfg.space_mask;
  a->words = (u64*)h->mem_a.p;
  a->wi_bitmap = h->wi_bitmap;
  a->max_wi = h->max_wi;
  a->arena = h->arena;
  a->word_base = h->n_mem;
  return AIWC_OK;
}

// The ingest of n memory events (device or host) into the current invocation.
aiwc_status push_mem_events(aiwc_handle* h, const aiwc_mem_event* ev, size_t n, int on_device) {
  MemIngestArgs a;
  aiwc_status s = ingest_args(h, n, &a);
  if (s != AIWC_OK) return s;
  const u64 base = h->n_mem;
  StageScope scope(h, kStMemIngest);
  if (on_device) {
    a.ev = ev;
    a.n = n;
    launch_mem_ingest(a, h->stream);
    CK(cudaGetLastError());
  } else {
    s = staged_copy(h, ev, n * 16, 16, [&](void* p, size_t first, size_t cnt) {
      MemIngestArgs b = a;
      b.ev = p;
      b.n = cnt;
      b.word_base = base + first;
      launch_mem_ingest(b, h->stream);
    });
    if (s != AIWC_OK) return s;
  }
  h->n_mem += n;
  return AIWC_OK;
}

// Byte-granular addresses: every byte an access touches becomes an access of
// its own. The host reads the byte counts of up to kExpandBatch chunks back
// at once, sizes the ingest, and each chunk's one-byte accesses are formed and
// ingested in one kernel at their tiles' offsets.
constexpr size_t kExpandBatch = 16;

aiwc_status expand_events(aiwc_handle* h, const void* dev_ev, size_t n) {
  aiwc_status s;
  const size_t nt = (size_t)(kExpandChunk / kExpandTile);
  const size_t per_chunk = expand_meta_bytes();  // tile offsets, then tile sums
  for (size_t b0 = 0; b0 < n; b0 += kExpandBatch * kExpandChunk) {
    const size_t nb = std::min<size_t>(kExpandBatch, (n - b0 + kExpandChunk - 1) / kExpandChunk);
    ENSURE(h->exp_meta, kExpandBatch * (per_chunk + 8), false);
    if ((s = ensure_bitmap(h)) != AIWC_OK) return s;
    if (!h->h_exp) CK(cudaMallocHost(&h->h_exp, kExpandBatch * sizeof(u64)));
    u64* totals = (u64*)h->exp_meta.p;
    ExpandArgs x[kExpandBatch];
    for (size_t j = 0; j < nb; ++j) {
      const size_t c0 = b0 + j * kExpandChunk;
      x[j].ev = (const char*)dev_ev + 16 * c0;
      x[j].n = std::min<size_t>((size_t)kExpandChunk, n - c0);
      x[j].tile_off = (u64*)((char*)h->exp_meta.p + kExpandBatch * 8 + j * per_chunk);
      x[j].tile_sum = (u32*)(x[j].tile_off + nt);
      x[j].total = totals + j;
      x[j].space_mask = h->cfg.space_mask;
      x[j].wi_bitmap = h->wi_bitmap;
      x[j].max_wi = h->max_wi;
      x[j].arena = h->arena;
      x[j].sm_count = h->sm_count;
    }
    {
      StageScope scope(h, kStMemExpand);
      for (size_t j = 0; j < nb; ++j) launch_expand_count(x[j], h->stream);
    }
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h->h_exp, totals, nb * sizeof(u64), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    u64 m = 0;
    for (size_t j = 0; j < nb; ++j) m += h->h_exp[j];
    if (m == 0) continue;
    MemIngestArgs a;
    if ((s = ingest_args(h, m, &a)) != AIWC_OK) return s;
    {
      StageScope scope(h, kStMemIngest);
      u64 at = h->n_mem;
      for (size_t j = 0; j < nb; ++j) {
        MemIngestArgs b = a;
        b.ev = x[j].ev;
        b.n = x[j].n;
        b.word_base = at;
        launch_mem_ingest_bytes(b, x[j].tile_off, h->stream);
        at += h->h_exp[j];
      }
    }
    CK(cudaGetLastError());
    h->n_mem += m;
  }
  return AIWC_OK;
}

}  // namespace

extern "C" {

aiwc_status aiwc_push_mem(aiwc_handle* h, const aiwc_mem_event* ev, size_t n, int on_device) {
  aiwc_status s = check_usable(h);
  if (s != AIWC_OK) return s;
  if (n == 0) return AIWC_OK;
  if (!ev) return fail(h, AIWC_EINVAL, "null event pointer", false);
  DeviceGuard g(h->cfg.device);
  if (on_device && ((uintptr_t)ev & 15u))
    return fail(h, AIWC_EINVAL, "device memory events must be 16-byte aligned", false);
  if (defers(h, on_device) && !h->cfg.byte_addresses) return record(h, 0, ev, nullptr, nullptr, nullptr, n, 0);
  if ((s = flush_deferred(h)) != AIWC_OK) return s;
  if (routing(h)) return routed(h, [&] { return route_mem(h, ev, n, on_device); });
  if (!h->cfg.byte_addresses) return push_mem_events(h, ev, n, on_device);
  if (on_device) return expand_events(h, ev, n);
  aiwc_status es = AIWC_OK;
  s = staged_copy(h, ev, n * 16, 16, [&](void* p, size_t, size_t cnt) {
    if (es == AIWC_OK) es = expand_events(h, p, cnt);
  });
  return s != AIWC_OK ? s : es;
}

aiwc_status aiwc_push_branch(aiwc_handle* h, const aiwc_branch_event* ev, size_t n, int on_device) {
  aiwc_status s = check_usable(h);
  if (s != AIWC_OK) return s;
  if (n == 0) return AIWC_OK;
  if (!ev) return fail(h, AIWC_EINVAL, "null event pointer", false);
  DeviceGuard g(h->cfg.device);
  if (on_device && ((uintptr_t)ev & 7u))
    return fail(h, AIWC_EINVAL, "device branch events must be 8-byte aligned", false);
  if (defers(h, on_device)) return record(h, 1, ev, nullptr, nullptr, nullptr, n, 0);
  if ((s = flush_deferred(h)) != AIWC_OK) return s;
  if (routing(h)) return routed(h, [&] { return route_branch(h, ev, n, on_device); });
  ENSURE(h->br_a, (h->n_br + n) * 8, true);
  ENSURE(h->br_c, (h->n_br + n) * 2, true);
  if ((s = ensure_bitmap(h)) != AIWC_OK) return s;
  BranchIngestArgs a;
  a.push_index = h->br_pushes;
  a.words = (u64*)h->br_a.p;
  a.compact = (uint16_t*)h->br_c.p;
  a.wi_bitmap = h->wi_bitmap;
  a.max_wi = h->max_wi;
  a.arena = h->arena;
  const u64 base = h->n_br;
  StageScope scope(h, kStBrIngest);
  if (on_device) {
    a.ev = ev;
    a.n = n;
    a.word_base = base;
    launch_branch_ingest(a, h->stream);
    CK(cudaGetLastError());
    h->br_pushes++;
    h->n_br += n;
    return AIWC_OK;
  } else {
    s = staged_copy(h, ev, n * 8, 8, [&](void* p, size_t first, size_t cnt) {
      BranchIngestArgs b = a;
      b.push_index = h->br_pushes++;
      b.ev = p;
      b.n = cnt;
      b.word_base = base + first;
      launch_branch_ingest(b, h->stream);
    });
    if (s != AIWC_OK) return s;
  }
  h->n_br += n;
  return AIWC_OK;
}

aiwc_status aiwc_push_widths(aiwc_handle* h, const uint16_t* widths, size_t n, int on_device) {
  aiwc_status s = check_usable(h);
  if (s != AIWC_OK) return s;
  if (n == 0) return AIWC_OK;
  if (!widths) return fail(h, AIWC_EINVAL, "null width pointer", false);
  DeviceGuard g(h->cfg.device);
  if (defers(h, on_device)) return record(h, 3, widths, nullptr, nullptr, nullptr, n, 0);
  if ((s = flush_deferred(h)) != AIWC_OK) return s;
  if (routing(h)) return routed(h, [&] { return route_widths(h, widths, n, on_device); });
  StageScope scope(h, kStInstrRuns);
  if (on_device) {
    launch_simd_widths(widths, n, h->arena, h->stream);
    CK(cudaGetLastError());
    return AIWC_OK;
  }
  return staged_copy(h, widths, n * 2, 2, [&](void* p, size_t, size_t cnt) {
    launch_simd_widths((const uint16_t*)p, cnt, h->arena, h->stream);
  });
}

aiwc_status aiwc_push_instr(aiwc_handle* h, uint32_t work_item, const uint16_t* ops, size_t n, int on_device) {
  aiwc_status s = check_usable(h);
  if (s != AIWC_OK) return s;
  if (n && !ops) return fail(h, AIWC_EINVAL, "null opcode pointer", false);
  DeviceGuard g(h->cfg.device);
  const bool dev = on_device != 0;
  if (dev && ((uintptr_t)ops & 1u)) return fail(h, AIWC_EINVAL, "device opcodes must be 2-byte aligned", false);
  if ((s = flush_deferred(h)) != AIWC_OK) return s;
  if (routing(h)) {
    const uint64_t off = 0, len = n;
    std::vector<uint16_t> one;
    const uint16_t* p = ops;
    if ((s = host_view(h, ops, n, on_device, &one, &p)) != AIWC_OK) return s;
    return routed(h, [&] { return route_runs(h, &work_item, &off, &len, 1, p, n, 0); });
  }
  if (!h->pend_wi.empty() && h->pend_device != dev) {
    if ((s = flush_pending(h)) != AIWC_OK) return s;
  }
  h->pend_device = dev;
  h->pend_wi.push_back(work_item);
  h->pend_len.push_back(n);
  if (dev) {
    h->pend_off.push_back((u64)(uintptr_t)ops / 2);
  } else {
    h->pend_off.push_back(h->pend_ops.size());
    h->pend_ops.insert(h->pend_ops.end(), ops, ops + n);
  }
  if (h->pend_ops.size() >= kPendingOps || h->pend_wi.size() >= kPendingRuns) return flush_pending(h);
  return AIWC_OK;
}

aiwc_status aiwc_push_instr_runs(aiwc_handle* h, const uint32_t* run_wi, const uint64_t* run_off,
                                 const uint64_t* run_len, size_t n_runs, const uint16_t* ops, size_t n_ops,
                                 int on_device) {
  aiwc_status s = check_usable(h);
  if (s != AIWC_OK) return s;
  if (n_runs == 0) return AIWC_OK;
  if (!run_wi || !run_off || !run_len || (n_ops && !ops)) return fail(h, AIWC_EINVAL, "null run table", false);
  DeviceGuard g(h->cfg.device);
  if (on_device && (((uintptr_t)ops & 1u) || ((uintptr_t)run_wi & 3u) || ((uintptr_t)run_off & 7u) ||
                    ((uintptr_t)run_len & 7u)))
    return fail(h, AIWC_EINVAL, "device run tables / opcodes are misaligned", false);
  if (defers(h, on_device) && h->pend_wi.empty()) return record(h, 2, run_wi, run_off, run_len, ops, n_runs, n_ops);
  if ((s = flush_deferred(h)) != AIWC_OK) return s;
  if ((s = flush_pending(h)) != AIWC_OK) return s;
  if (routing(h)) return routed(h, [&] { return route_runs(h, run_wi, run_off, run_len, n_runs, ops, n_ops, on_device); });
  if (on_device)
    return runs_device(h, run_wi, (const u64*)run_off, (const u64*)run_len, n_runs, ops, n_ops, n_ops);
  return runs_host(h, run_wi, run_off, run_len, n_runs, ops, n_ops);
}

}  // extern "C"

namespace {

// One captured CUDA graph per device for aiwc_compute_batch: every handle's
// stages on forked streams (parallel branches), replayed while the batch
// signature (handles, sizes, plans, buffer epochs) repeats.
struct BatchGraph {
  std::mutex mu;
  std::vector<u64> sig;
  cudaGraphExec_t exec = nullptr;
  u64 kernels = 0;  // kernels captured in exec (each replay launches them all)
  cudaStream_t cs = nullptr;
  std::vector<cudaStream_t> forks;
  cudaEvent_t ev_user = nullptr, ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_join;

  aiwc_status init() {
    if (cs) return AIWC_OK;
    constexpr int kForks = 16;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_user, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming);
    for (int i = 0; i < kForks && e == cudaSuccess; ++i) {
      cudaStream_t f;
      cudaEvent_t j;
      e = cudaStreamCreateWithFlags(&f, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
      if (e == cudaSuccess) {
        forks.push_back(f);
        ev_join.push_back(j);
      }
    }
    if (e != cudaSuccess) return cuda_fail(nullptr, "batch graph streams", e);
    return AIWC_OK;
  }

  aiwc_status run(const std::vector<u64>& s, cudaStream_t user,
                  const std::function<aiwc_status(cudaStream_t, std::vector<cudaStream_t>&)>& enqueue) {
    std::lock_guard<std::mutex> lk(mu);
    aiwc_status st = init();
    if (st != AIWC_OK) return st;
    cudaError_t e;
    if (!exec || s != sig) {
      if (exec) {
        cudaGraphExecDestroy(exec);
        exec = nullptr;
      }
      sig.clear();
      if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
        return cuda_fail(nullptr, "cudaStreamBeginCapture", e);
      const u64 before = launches_so_far();
      cudaEventRecord(ev_fork, cs);
      for (cudaStream_t f : forks) cudaStreamWaitEvent(f, ev_fork, 0);
      st = enqueue(cs, forks);
      kernels = launches_so_far() - before;
      for (size_t k = 0; k < forks.size(); ++k) {
        cudaEventRecord(ev_join[k], forks[k]);
        cudaStreamWaitEvent(cs, ev_join[k], 0);
      }
      cudaGraph_t graph = nullptr;
      e = cudaStreamEndCapture(cs, &graph);
      if (st != AIWC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (e != cudaSuccess) return cuda_fail(nullptr, "cudaStreamEndCapture", e);
      e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        exec = nullptr;
        return cuda_fail(nullptr, "cudaGraphInstantiate", e);
      }
      sig = s;
    } else {
      count_launches(kernels);  // a replay launches every captured kernel again
    }
    if ((e = cudaEventRecord(ev_user, user)) != cudaSuccess || (e = cudaStreamWaitEvent(cs, ev_user, 0)) != cudaSuccess ||
        (e = cudaGraphLaunch(exec, cs)) != cudaSuccess || (e = cudaStreamSynchronize(cs)) != cudaSuccess)
      return cuda_fail(nullptr, "batch graph launch", e);
    return AIWC_OK;
  }
};

BatchGraph& batch_graph(int device) {
  static BatchGraph graphs[64];
  return graphs[device & 63];
}

// Streams on which aiwc_compute_batch ingests the handles' deferred pushes in
// parallel (one set per device, created on first use).
struct PushForks {
  std::mutex mu;
  std::vector<cudaStream_t> s;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  aiwc_status init() {
    if (fork) return AIWC_OK;
    constexpr int kStreams = 16;
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int i = 0; i < kStreams && e == cudaSuccess; ++i) {
      cudaStream_t st;
      cudaEvent_t j;
      e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j, cudaEventDisableTiming);
      if (e == cudaSuccess) {
        s.push_back(st);
        join.push_back(j);
      }
    }
    if (e != cudaSuccess) return cuda_fail(nullptr, "push streams", e);
    return AIWC_OK;
  }
};
PushForks& push_forks(int device) {
  static PushForks forks[64];
  return forks[device & 63];
}

}  // namespace

namespace {

// What a compute launches. Host decisions come from the ingest-time device
// counters; `gated` leaves the branch-path choice to a device flag so that a
// captured graph holds both alternatives.
struct Plan {
  bool gated = false;
  bool hash_ok = false;   // memory: hash plan (else the sort plan, rebuilding words if the table was used)
  bool per_site = false;  // branch: per-site patterns (when !gated)
  u32 br_passes = 0xFFu, run_passes = 0xFFu;
  int seg_shift = 0;      // memory, hash plan: low address bits that are zero in every kept event (0..3)
  bool site_sort = false; // branch: stable counting sort by site (in order work-item ids, site ids < kCsSites)
  bool long_sites = false;  // branch, per-site path: sites longer than kSiteMaxLen may exist
  bool defer_finalize = false;  // partitioned invocation: reduce only, the partitions are merged first
};

u32 active_passes(u64 kor, u64 kand, u64 mask) {
  const u64 varying = (kor ^ kand) & mask;
  u32 m = 0;
  for (int p = 0; p < 8; ++p)
    if ((varying >> (8 * p)) & 0xFFull) m |= 1u << p;
  return m;
}

// Host part of a compute: pending runs, and every buffer the stages need.
aiwc_status prepare(aiwc_handle* h) {
  aiwc_status s = flush_deferred(h);
  if (s != AIWC_OK) return s;
  if ((s = flush_pending(h)) != AIWC_OK) return s;
  const u64 n_mem = h->n_mem, n_br = h->n_br, n_runs = h->n_runs;
  ENSURE(h->over_a, over_bound(h, n_mem, n_br, n_runs) * 8, true);
  h->c_over_cap = h->over_a.cap / 8;
  const u64 nmax = std::max(std::max(n_mem, n_br), std::max(n_runs, h->c_over_cap));
  ENSURE(h->mem_a, std::max<u64>(n_mem, 1) * 8, true);
  ENSURE(h->mem_b, std::max<u64>(n_mem, 1) * 8, true);  // holds the slot words of the hash plan
  h->c_low_off = ((size_t)n_mem * 8 + 255) & ~size_t(255);
  ENSURE(h->mem_b, h->c_low_off + (size_t)n_mem * 2, true);
  ENSURE(h->br_a, std::max<u64>(n_br, 1) * 8, true);
  ENSURE(h->br_b, std::max<u64>(n_br, 1) * 8, false);
  ENSURE(h->pat_a, std::max<u64>(n_br, 1) * 8, false);
  // the site list (one word per site, n_br at most) follows the counting
  // sort's chunk sums in the second pattern buffer
  h->c_site_off = (site_sort_chunk_words(n_br) * 4 + 255) & ~size_t(255);
  ENSURE(h->pat_b, std::max<size_t>(h->c_site_off + n_br * 8, std::max<u64>(n_br, 1) * 8), false);
  ENSURE(h->rk_a, std::max<u64>(n_runs, 1) * 8, true);
  ENSURE(h->rk_b, std::max<u64>(n_runs, 1) * 8, false);
  ENSURE(h->run_sum, std::max<u64>(n_runs, 1) * 32, true);
  ENSURE(h->over_b, h->c_over_cap * 8, false);
  ENSURE(h->counts, sort_counts_words(nmax) * 4, false);
  ENSURE(h->bsums, sort_block_sums_words(nmax) * 4, false);
  // memory levels, or the branch site runs, or two levels of pattern runs
  ENSURE(h->tiles, std::max<u64>((u64)kLevels * ntiles_of(n_mem), 2 * ntiles_of(n_br) + 1) * sizeof(TileSum), false);
  // site starts and lengths are 32-bit fields: no list (the global path) from 2^32 events
  h->c_sites_cap = n_br < (1ull << 32) ? n_br : 0;
  // the long-site list: every long site has more than kSiteMaxLen events
  ENSURE(h->sites, (n_br / (kSiteMaxLen + 1) + 1) * 24, false);
  // runs pushed in (work-item, push) order need no sort: checked before the
  // counters are read back
  launch_keys_sorted((const u64*)h->rk_a.p, n_runs, &h->arena->st.run_unsorted, h->stream);
  return ensure_bitmap(h);
}

SortDesc sort_desc(aiwc_handle* h, DevBuf& a, DevBuf& b, int slot, const u64* n_dev, const u64* kor,
                   const u64* kand, u64 mask, u64 n_host) {
  SortDesc d;
  d.a = (u64*)a.p;
  d.b = (u64*)b.p;
  d.cur = &h->arena->st.sort_cur[slot];
  d.n = n_dev;
  d.n_cap = std::min<u64>(a.cap, b.cap) / 8;
  d.key_or = kor;
  d.key_and = kand;
  d.mask = mask;
  d.lo_bit = 0;
  d.counts = (u32*)h->counts.p;
  d.block_sums = (u32*)h->bsums.p;
  d.ntiles = sort_tiles(n_host);
  d.err = &h->arena->st.err;
  return d;
}

SortDesc branch_sort_desc(aiwc_handle* h) {
  DevState* dst = &h->arena->st;
  SortDesc d = sort_desc(h, h->br_a, h->br_b, kSortBranch, &dst->n_branch, &dst->br_or, &dst->br_and, ~1ull, h->n_br);
  d.unsorted = &dst->br_unsorted;
  return d;
}

// Long sites the per-site path can take: their tables live in the first
// pattern buffer (free on that path once the site sort has run), their list
// in `sites`.
u64 long_cap_of(const aiwc_handle* h) { return long_sites_cap(h->pat_a.cap, h->sites.cap, h->cfg.history_len); }

SiteArgs site_args(aiwc_handle* h, const SortDesc& bsort) {
  SiteArgs sa;
  sa.a = bsort.a;
  sa.b = bsort.b;
  sa.cur = bsort.cur;
  sa.n = h->n_br;
  sa.h = h->cfg.history_len;
  sa.sites = (u64*)((char*)h->pat_b.p + h->c_site_off);
  sa.sites_cap = h->c_sites_cap;
  sa.over = (u64*)h->over_a.p;
  sa.over_cap = h->c_over_cap;
  sa.arena = h->arena;
  sa.grid = h->sm_count;
  sa.long_tab = (u64*)h->pat_a.p;
  sa.long_list = (u64*)h->sites.p;
  sa.long_cap = long_cap_of(h);
  return sa;
}

SiteSortArgs site_sort_args(aiwc_handle* h) {
  SiteSortArgs ss;
  ss.src = (const u64*)h->br_a.p;
  ss.src16 = (const uint16_t*)h->br_c.p;
  ss.dst = (u64*)h->br_b.p;
  ss.sort_cur = &h->arena->st.sort_cur[kSortBranch];
  ss.n = h->n_br;
  ss.counts = (u32*)h->pat_a.p;
  ss.chunks = (u32*)h->pat_b.p;
  ss.sites = (u64*)((char*)h->pat_b.p + h->c_site_off);
  ss.sites_cap = h->c_sites_cap;
  ss.arena = h->arena;
  ss.sm_count = h->sm_count;
  ss.tile_shift = site_sort_tile_shift(h->n_br, h->sm_count);
  return ss;
}

// Stages that must run before the branch-path choice: the branch sort and the site list.
void enqueue_part1(aiwc_handle* h, cudaStream_t st, const Plan& p) {
  if (!h->n_br) return;
  if (p.site_sort) {
    // the site list, n_sites and the longest site; the sorted output follows
    // once the branch path is chosen
    StageScope sc(h, kStBrSort, st);
    launch_site_sort_count(site_sort_args(h), st);
    return;
  }
  SortDesc bsort = branch_sort_desc(h);
  {
    StageScope sc(h, kStBrSort, st);
    sort_keys(bsort, st, p.br_passes);
  }
  StageScope sc(h, kStWindows, st);
  launch_site_heads(site_args(h, bsort), st);
  if (p.gated)
    launch_persite_decide(h->arena, h->cfg.history_len, h->c_sites_cap, long_cap_of(h), h->cfg.plan != 1, st);
}

aiwc_status enqueue_finalize(aiwc_handle* h, cudaStream_t st);

// Everything after the branch-path choice, the result copies and the reset.
// The memory reduction after the ingest: segment scatter and walks (hash
// plan) or the sort and run lengths (sort plan).
void enqueue_mem_path(aiwc_handle* h, cudaStream_t st, const Plan& p) {
  const u64 n_mem = h->n_mem;
  DevState* dst = &h->arena->st;
  u64* over = (u64*)h->over_a.p;
  const u64 over_cap = h->c_over_cap;
  const int grid = h->sm_count * 3;
  const bool ran_hash = n_mem && use_hash(h) && h->sbt_cap;
  if (ran_hash && !p.hash_ok) {
    // the table overflowed: rebuild 64-bit words behind the spilled ones, then sort
    launch_rebuild_words((const u64*)h->mem_b.p, table_view(h), (u64*)h->mem_a.p, h->arena, grid * 2, st);
  }
  if (n_mem && p.hash_ok) {
    HashArgs ha;
    ha.slotw = (const u64*)h->mem_b.p;
    ha.n_cap = std::min<u64>(n_mem, (h->mem_b.cap - h->c_low_off) / 2);
    ha.low = (uint16_t*)((char*)h->mem_b.p + h->c_low_off);
    ha.tab = table_view(h);
    ha.scan_tmp = (u32*)h->sbt_scan.p;
    ha.n_used = dst->sb_used;
    ha.used_list = (u32*)((char*)h->sbt.p + (kSbtClearBytes + 4) * h->sbt_cap);
    ha.over = over;
    ha.over_cap = over_cap;
    ha.arena = h->arena;
    // up to eight blocks per SM, none without events (2048 events per block and step)
    ha.grid_scatter = (int)std::min<u64>((u64)h->sm_count * 8, std::max<u64>((n_mem + 2047) / 2048, 1));
    ha.sm_count = h->sm_count;
    ha.seg_shift = p.seg_shift;
    // the 64-bit word buffer is free in the hash plan: wide-segment histograms
    ha.big_hist = (u32*)h->mem_a.p;
    ha.big_cap = mem_hash_big_segments(n_mem, h->mem_a.cap, p.seg_shift);
    {
      StageScope sc(h, kStMemScatter, st);
      launch_mem_hash_scatter(ha, st);
    }
    StageScope sc(h, kStMemLevels, st);
    launch_mem_hash_segments(ha, st);
  } else if (n_mem) {
    SortDesc d = sort_desc(h, h->mem_a, h->mem_b, kSortMem, &dst->n_words, &dst->mem_or, &dst->mem_and, ~0ull, n_mem);
    {
      StageScope sc(h, kStMemSort, st);
      sort_keys(d, st, active_passes(h->h_state->mem_or, h->h_state->mem_and, ~0ull));
    }
    StageScope sc(h, kStMemLevels, st);
    LevelArgs la;
    la.a = d.a;
    la.b = d.b;
    la.cur = d.cur;
    la.n = &dst->n_words;
    la.tiles = (TileSum*)h->tiles.p;
    la.ntiles = (u32)ntiles_of(n_mem);
    la.over = over;
    la.over_cap = over_cap;
    la.arena = h->arena;
    la.grid = grid;
    launch_mem_levels(la, st);
    launch_runs_fixup(0, la.tiles, la.ntiles, &dst->n_words, 0, kLevels, over, over_cap, h->arena, st);
  }
}

// The branch reduction after the branch sort: per-site patterns or the global
// path (windows, pattern sort, pattern runs).
void enqueue_branch_path(aiwc_handle* h, cudaStream_t st, const Plan& p) {
  const u64 n_br = h->n_br;
  DevState* dst = &h->arena->st;
  u64* over = (u64*)h->over_a.p;
  const u64 over_cap = h->c_over_cap;
  const int grid = h->sm_count * 3;
  if (n_br) {
    // per-site patterns in shared memory, or the global path (windows,
    // pattern sort, pattern runs); with `gated` both are launched and a
    // device flag lets exactly one of them work
    const u32* gate = p.gated ? &dst->br_persite : nullptr;
    SortDesc bsort = branch_sort_desc(h);
    if (p.site_sort) {
      // the per-site path needs only the outcome bits: one byte per event
      StageScope sc(h, kStBrSort, st);
      SiteSortArgs ss = site_sort_args(h);
      if (p.per_site && !h->cfg.history_scope) ss.dst8 = (uint8_t*)h->br_b.p;
      launch_site_sort_scatter(ss, st);
    }
    if (p.gated || p.per_site) {
      StageScope sc(h, kStPatRuns, st);
      SiteArgs sa = site_args(h, bsort);
      sa.gate = gate;
      sa.gate_want = 1;
      if (p.site_sort && !h->cfg.history_scope) sa.outcomes = (const uint8_t*)h->br_b.p;
      sa.per_wi = h->cfg.history_scope != 0;
      launch_site_patterns(sa, st);
      if (p.long_sites) launch_site_long(sa, st);
    }
    if (p.gated || !p.per_site) {
      WindowArgs wa;
      wa.gate = gate;
      wa.gate_want = 0;
      wa.a = bsort.a;
      wa.b = bsort.b;
      wa.cur = bsort.cur;
      wa.n = n_br;
      wa.h = h->cfg.history_len;
      wa.gshift = h->cfg.history_scope ? 1u : 32u;
      wa.site_pred = h->cfg.history_scope == 0;
      wa.patterns = (u64*)h->pat_a.p;
      wa.tiles = (TileSum*)h->tiles.p;
      wa.ntiles = (u32)ntiles_of(n_br);
      wa.over = over;
      wa.over_cap = over_cap;
      wa.arena = h->arena;
      wa.grid = grid;
      {
        StageScope sc(h, kStWindows, st);
        launch_branch_windows(wa, st);
        launch_runs_fixup(1, wa.tiles, wa.ntiles, nullptr, n_br, 1, over, over_cap, h->arena, st, gate, 0,
                          h->cfg.history_scope ? 0u : h->cfg.history_len);
      }
      SortDesc ps = sort_desc(h, h->pat_a, h->pat_b, kSortPattern, &dst->n_patterns, &dst->pat_or, &dst->pat_and,
                              ~0ull, n_br);
      ps.gate = gate;
      ps.gate_want = 0;
      {
        StageScope sc(h, kStPatSort, st);
        sort_keys(ps, st);
      }
      StageScope sc(h, kStPatRuns, st);
      PatternArgs pa;
      pa.gate = gate;
      pa.gate_want = 0;
      pa.a = ps.a;
      pa.b = ps.b;
      pa.cur = ps.cur;
      pa.n = &dst->n_patterns;
      pa.tiles = (TileSum*)h->tiles.p;
      pa.ntiles = (u32)ntiles_of(n_br);
      pa.over = over;
      pa.over_cap = over_cap;
      pa.arena = h->arena;
      pa.grid = grid;
      pa.site_level = h->cfg.history_scope != 0;
      launch_pattern_runs(pa, st);
      launch_runs_fixup(2, pa.tiles, pa.ntiles, &dst->n_patterns, 0, pa.site_level ? 2 : 1, over, over_cap, h->arena,
                        st, gate, 0);
    }
  }
}

// Instruction runs chained per work-item, then (unless deferred) the finalisation.
aiwc_status enqueue_tail(aiwc_handle* h, cudaStream_t st, const Plan& p) {
  const u64 n_runs = h->n_runs;
  DevState* dst = &h->arena->st;
  u64* over = (u64*)h->over_a.p;
  const u64 over_cap = h->c_over_cap;
  if (n_runs) {
    SortDesc d = sort_desc(h, h->rk_a, h->rk_b, kSortRuns, &dst->n_runs, &dst->run_or, &dst->run_and, ~0ull, n_runs);
    {
      StageScope sc(h, kStRunSort, st);
      sort_keys(d, st, p.run_passes);
    }
    StageScope sc(h, kStCombine, st);
    CombineArgs ca;
    ca.a = d.a;
    ca.b = d.b;
    ca.cur = d.cur;
    ca.n_runs = n_runs;
    ca.run_sum = (const u64*)h->run_sum.p;
    ca.over = over;
    ca.over_cap = over_cap;
    ca.arena = h->arena;
    launch_instr_combine(ca, st);
  }
  if (p.defer_finalize) return AIWC_OK;
  return enqueue_finalize(h, st);
}

// Every stage after the branch-path choice, in one stream.
aiwc_status enqueue_part2(aiwc_handle* h, cudaStream_t st, const Plan& p) {
  enqueue_mem_path(h, st, p);
  enqueue_branch_path(h, st, p);
  return enqueue_tail(h, st, p);
}

// The end of an invocation: opcode distribution, work-item count, overflow
// sort, the finalize kernel, the result copies and the reset.
aiwc_status enqueue_finalize(aiwc_handle* h, cudaStream_t st) {
  DevState* dst = &h->arena->st;
  u64* over = (u64*)h->over_a.p;
  const u64 over_cap = h->c_over_cap;
  {
    StageScope fin_scope(h, kStFinalize, st);
    launch_tail_counts((const u64*)h->d_hist, h->cfg.n_opcodes, h->wi_bitmap, over, over_cap, h->arena, st);
    // Outside a graph capture the overflow list is complete here: one
    // synchronisation sizes its sort by the entries it holds (a few thousand
    // where the bound is millions) and runs only the passes whose digits vary.
    u64 n_sort = over_cap;
    u32 passes = 0xFFu;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone) {
      CK(cudaMemcpyAsync(h->h_state, dst, sizeof(DevState), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      n_sort = std::min<u64>(h->h_state->n_over, over_cap);
      passes = active_passes(h->h_state->over_or, h->h_state->over_and, ~0ull);
    } else {
      cudaGetLastError();
    }
    SortDesc d = sort_desc(h, h->over_a, h->over_b, kSortOver, &dst->n_over, &dst->over_or, &dst->over_and, ~0ull,
                           n_sort);
    sort_keys(d, st, passes);
    FinalizeArgs fa;
    fa.over_a = d.a;
    fa.over_b = d.b;
    fa.over_cur = d.cur;
    fa.over_cap = over_cap;
    fa.arena = h->arena;
    fa.result = h->d_result;
    fa.cover_num = h->cfg.cover_num;
    fa.cover_den = h->cfg.cover_den;
    fa.precision = h->cfg.precision;
    fa.history_len = h->cfg.history_len;
    launch_finalize(fa, st);
  }
  CK(cudaGetLastError());
  // the result and the opcode histogram after it: one copy
  CK(cudaMemcpyAsync(h->h_result, h->d_result, result_bytes(h->cfg.n_opcodes), cudaMemcpyDeviceToHost, st));
  return reset_device_state(h, st, false);
}

void reset_host(aiwc_handle* h) {
  h->n_mem = h->n_br = h->n_runs = 0;
  h->inv_plan = 0;
  h->br_pushes = 0;
  h->value_bound = 0;
  h->pend_ops.clear();
  h->pend_wi.clear();
  h->pend_off.clear();
  h->pend_len.clear();
}

// After the stream has been synchronised: results out, host state reset.
aiwc_status finish(aiwc_handle* h, aiwc_metrics* out, uint64_t* user_hist) {
  h->last_plan_hash = h->n_mem && use_hash(h) && h->sbt_cap;
  reset_host(h);
  *out = h->h_result->m;
  out->opcode_hist = user_hist;
  if (user_hist) memcpy(user_hist, h->h_hist, (size_t)h->cfg.n_opcodes * 8);
  const u32 err = h->h_result->err;
  if (err & kErrOverflow) return fail(h, AIWC_ECUDA, "internal overflow list exceeded its bound", false);
  if (err & kErrAddr) return fail(h, AIWC_EINVAL, "memory address outside the 61-bit domain", false);
  if (err & kErrOpcode) return fail(h, AIWC_EINVAL, "opcode >= n_opcodes that is not a barrier", false);
  if (err & kErrWorkItem) return fail(h, AIWC_EINVAL, "work-item id >= max_work_items", false);
  if (err & kErrRun) return fail(h, AIWC_EINVAL, "instruction run reaches past its opcode array", false);
  if (err & kErrSort) return fail(h, AIWC_ETIMEOUT, "a radix sort pass waited too long for an earlier tile", false);
  return AIWC_OK;
}

// Recovers a broken handle: drops the invocation.
aiwc_status recover(aiwc_handle* h) {
  reset_host(h);
  h->deferred.clear();
  h->flushing = false;
  h->replaying = false;
  h->part_err = 0;
  for (auto& pb : h->parts) pb.clear();
  cudaStreamSynchronize(h->side_stream);
  cudaGetLastError();
  if (reset_device_state(h, h->stream, true) == AIWC_OK && cudaStreamSynchronize(h->stream) == cudaSuccess)
    h->broken = false;
  return AIWC_ESTATE;
}

// The stable counting sort by site applies: work-item ids arrived in order
// and site ids are below kCsSites (h->h_state must be current).
bool site_sort_ok(const aiwc_handle* h) {
  const DevState& hs = *h->h_state;
  return h->n_br >= (1ull << 16) && h->n_br < (1ull << 32) && !hs.br_unsorted && (hs.br_or >> 32) < kCsSites &&
         h->cfg.plan != 1;
}

// The per-site branch path applies whatever the sites turn out to be: no
// more sites than the list holds (n_br of them at most, or kCsSites with the
// counting sort), and a table for every long site (each has more than
// kSiteMaxLen of the n_br events).
bool per_site_certain(const aiwc_handle* h, bool site_sort) {
  if (h->cfg.history_len > kSiteMaxHist || h->cfg.plan == 1) return false;
  if (h->n_br <= kSiteMaxLen) return true;
  const bool sites_fit = site_sort || h->n_br <= h->c_sites_cap;
  return sites_fit && h->n_br < (1ull << 32) && long_cap_of(h) >= h->n_br / (kSiteMaxLen + 1);
}

// Host decisions from the ingest-time counters (h->h_state must be current).
void plan_from_ingest(aiwc_handle* h, Plan* p) {
  const DevState& hs = *h->h_state;
  const bool hashed = h->n_mem && use_hash(h) && h->sbt_cap;
  // segment offsets are 32-bit: 2^32 kept events or more go to the sort plan
  p->hash_ok = hashed && hs.sbt_overflow == 0 && hs.n_words < (1ull << 32);
  if (hashed && hs.sbt_overflow) h->sbt_want = h->sbt_floor = std::min<u64>(h->sbt_cap * 4, kMaxHashSlots);
  p->br_passes = active_passes(hs.br_or, hs.br_and, hs.br_unsorted ? ~1ull : 0xFFFFFFFF00000000ull);
  p->run_passes = hs.run_unsorted ? active_passes(hs.run_or, hs.run_and, ~0ull) : 0u;
  // address bits sit above the store bit of the word
  const u64 addr_or = (hs.mem_or >> 1) & ((1ull << 61) - 1);
  p->seg_shift = addr_or ? std::min(__builtin_ctzll(addr_or), 3) : 3;
  // the counting sort's per-tile counts (n_br / 8 words or less) live in the
  // pattern buffers, which hold 2 n_br words each
  p->site_sort = !p->gated && site_sort_ok(h);
}

// Everything a compute enqueues for what is pushed now: the plan from the
// ingest-time counters, the stages, and (unless deferred) the finalisation.
aiwc_status reduce_current(aiwc_handle* h, bool defer_finalize) {
  cudaStream_t st = h->stream;
  aiwc_status s = prepare(h);
  if (s != AIWC_OK) return s;
  // read the ingest-time counters: memory plan, active sort passes
  CK(cudaMemcpyAsync(h->h_state, &h->arena->st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  Plan p;
  plan_from_ingest(h, &p);
  p.defer_finalize = defer_finalize;
  // In the hash plan the memory and branch reductions share no scratch
  // buffer (both only add to their own distributions and append to the
  // overflow list atomically): the branch reduction runs on the side stream,
  // forked after the ingest and joined before the tail.
  const bool split = p.hash_ok && h->n_br != 0;
  cudaStream_t sb = split ? h->side_stream : st;
  if (split) {
    CK(cudaEventRecord(h->ev_fork, st));
    CK(cudaStreamWaitEvent(sb, h->ev_fork, 0));
    enqueue_mem_path(h, st, p);
  }
  enqueue_part1(h, sb, p);
  if (h->n_br) {
    // the branch path depends on the longest site (only the branch fields of
    // the copy are read: the memory reduction may be running meanwhile)
    CK(cudaMemcpyAsync(h->h_state, &h->arena->st, sizeof(DevState), cudaMemcpyDeviceToHost, sb));
    CK(cudaStreamSynchronize(sb));
    const DevState& hs = *h->h_state;
    const bool longs_fit = hs.br_site_max <= kSiteMaxLen ||
                           (hs.n_long <= long_cap_of(h) && hs.br_site_max < (1ull << 32));
    p.per_site = h->cfg.history_len <= kSiteMaxHist && longs_fit && hs.n_sites <= h->c_sites_cap &&
                 h->cfg.plan != 1;
    p.long_sites = hs.n_long != 0;
  }
  if (!split) return enqueue_part2(h, st, p);
  enqueue_branch_path(h, sb, p);
  CK(cudaGetLastError());
  CK(cudaEventRecord(h->ev_join, sb));
  CK(cudaStreamWaitEvent(st, h->ev_join, 0));
  return enqueue_tail(h, st, p);
}

// Partitioned invocation: each partition is pushed to the device and reduced
// with the finalisation deferred, its distributions are added to the total,
// and the total is finalised once.
aiwc_status compute_partitioned(aiwc_handle* h, aiwc_metrics* out) {
  uint64_t* user_hist = out->opcode_hist;
  cudaStream_t st = h->stream;
  auto& parts = h->parts;
  const u32 perr = h->part_err;
  h->part_err = 0;
  if (perr & kErrRun) {
    for (auto& pb : parts) pb.clear();
    return fail(h, AIWC_EINVAL, "instruction run reaches past its opcode array", false);
  }
  u64 total_cap = 0;  // the merged entries fit the sum of the partitions' bounds
  for (auto& pb : parts)
    total_cap += over_bound_sizes(h->cfg.n_opcodes, pb.mem.size() / 16, pb.br.size(), pb.run_wi.size(),
                                  pb.ops.size() / kValDense + 2);
  if (!h->total) {
    CK(cudaMalloc(&h->total, sizeof(Arena)));
    h->bytes += sizeof(Arena);
  }
  ENSURE(h->over_total, total_cap * 8, false);
  CK(cudaMemsetAsync(h->total, 0, sizeof(Arena), st));
  launch_reset_identities(h->total, st);
  h->replaying = true;
  aiwc_status s = AIWC_OK;
  for (auto& pb : parts) {
    if (pb.mem.empty() && pb.br.empty() && pb.run_wi.empty() && pb.widths.empty()) continue;
    if (!pb.mem.empty())
      s = aiwc_push_mem(h, reinterpret_cast<const aiwc_mem_event*>(pb.mem.data()), pb.mem.size() / 16, 0);
    if (s == AIWC_OK && !pb.br.empty())
      s = aiwc_push_branch(h, reinterpret_cast<const aiwc_branch_event*>(pb.br.data()), pb.br.size(), 0);
    if (s == AIWC_OK && !pb.run_wi.empty())
      s = aiwc_push_instr_runs(h, pb.run_wi.data(), pb.run_off.data(), pb.run_len.data(), pb.run_wi.size(),
                               pb.ops.data(), pb.ops.size(), 0);
    if (s == AIWC_OK && !pb.widths.empty()) s = aiwc_push_widths(h, pb.widths.data(), pb.widths.size(), 0);
    if (s == AIWC_OK) s = reduce_current(h, true);
    pb.clear();
    if (s != AIWC_OK) {
      h->replaying = false;
      for (auto& q : parts) q.clear();
      return s;
    }
    launch_merge_partition(h->arena, (const u64*)h->over_a.p, h->c_over_cap, h->total, (u64*)h->over_total.p,
                           total_cap, st);
    // the partition's state goes; the opcode histogram and the work-item bitmap keep adding up
    CK(cudaMemsetAsync(h->arena, 0, sizeof(Arena), st));
    if (h->sbt.p) CK(cudaMemsetAsync(h->sbt.p, 0, kSbtClearBytes * h->sbt_cap, st));
    launch_reset_identities(h->arena, st);
    reset_host(h);
  }
  h->replaying = false;
  return finalize_merged(h, total_cap, out, user_hist);
}

// The end of a partitioned or sharded invocation: the merged distributions
// (h->total and total_cap entries of h->over_total; the opcode histogram and
// the work-item bitmap already merged in place) are finalised in the handle's
// own arena and overflow list.
aiwc_status finalize_merged(aiwc_handle* h, u64 total_cap, aiwc_metrics* out, uint64_t* user_hist) {
  cudaStream_t st = h->stream;
  aiwc_status s;
  const u64 cap = std::max<u64>(total_cap, 1);
  ENSURE(h->over_a, cap * 8, false);
  ENSURE(h->over_b, cap * 8, false);
  ENSURE(h->counts, sort_counts_words(cap) * 4, false);
  ENSURE(h->bsums, sort_block_sums_words(cap) * 4, false);
  h->c_over_cap = total_cap;
  CK(cudaMemcpyAsync(h->arena, h->total, sizeof(Arena), cudaMemcpyDeviceToDevice, st));
  if (total_cap) CK(cudaMemcpyAsync(h->over_a.p, h->over_total.p, total_cap * 8, cudaMemcpyDeviceToDevice, st));
  if ((s = enqueue_finalize(h, st)) != AIWC_OK) return s;
  CK(cudaStreamSynchronize(st));
  collect_stage_times(h);
  return finish(h, out, user_hist);
}


}  // namespace

extern "C" {

aiwc_status aiwc_compute(aiwc_handle* h, aiwc_metrics* out) {
  if (!h || !out) return fail(h, AIWC_EINVAL, "null handle or output pointer", false);
  DeviceGuard g(h->cfg.device);
  uint64_t* user_hist = out->opcode_hist;
  if (h->broken) return recover(h);
  if (!h->parts.empty()) return compute_partitioned(h, out);
  aiwc_status s = reduce_current(h, false);
  if (s != AIWC_OK) return s;
  CK(cudaStreamSynchronize(h->stream));
  collect_stage_times(h);
  return finish(h, out, user_hist);
}

aiwc_status aiwc_compute_batch(aiwc_handle* const* hs, size_t n, aiwc_metrics* outs) {
  if (n && (!hs || !outs)) return fail(nullptr, AIWC_EINVAL, "null batch arrays");
  if (n == 0) return AIWC_OK;
  for (size_t i = 0; i < n; ++i) {
    if (!hs[i]) return fail(nullptr, AIWC_EINVAL, "null handle in batch");
    if (hs[i]->cfg.device != hs[0]->cfg.device || hs[i]->stream != hs[0]->stream)
      return fail(nullptr, AIWC_EINVAL, "batched handles must share one device and one stream");
    if (!hs[i]->parts.empty()) return fail(nullptr, AIWC_EINVAL, "partitioned handles cannot be batched");
    for (size_t j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return fail(nullptr, AIWC_EINVAL, "a handle appears twice in the batch");
  }
  DeviceGuard g(hs[0]->cfg.device);
  cudaStream_t user = hs[0]->stream;
  std::vector<uint64_t*> hists(n);
  aiwc_status worst = AIWC_OK;
  std::vector<char> live(n, 1);
  // deferred device pushes: every handle's on one of the push streams, so
  // that small invocations ingest side by side; the user stream waits for all
  std::vector<aiwc_status> pushed(n, AIWC_OK);
  bool any_deferred = false;
  for (size_t i = 0; i < n; ++i) any_deferred |= !hs[i]->broken && !hs[i]->deferred.empty();
  if (any_deferred) {
    PushForks& pf = push_forks(hs[0]->cfg.device);
    std::lock_guard<std::mutex> lk(pf.mu);
    aiwc_status e = pf.init();
    if (e != AIWC_OK) return e;
    if (cudaEventRecord(pf.fork, user) != cudaSuccess) return cuda_fail(nullptr, "push fork", cudaGetLastError());
    const size_t S = pf.s.size();
    std::vector<char> used(S, 0);
    size_t k = 0;
    for (size_t i = 0; i < n; ++i) {
      aiwc_handle* h = hs[i];
      if (h->broken || h->deferred.empty()) continue;
      const size_t j = k++ % S;
      if (!used[j]) {
        if (cudaStreamWaitEvent(pf.s[j], pf.fork, 0) != cudaSuccess)
          return cuda_fail(nullptr, "push fork", cudaGetLastError());
        used[j] = 1;
      }
      cudaStream_t own = h->stream;
      h->stream = pf.s[j];
      pushed[i] = flush_deferred(h);
      h->stream = own;
    }
    for (size_t j = 0; j < S; ++j)
      if (used[j] && (cudaEventRecord(pf.join[j], pf.s[j]) != cudaSuccess ||
                      cudaStreamWaitEvent(user, pf.join[j], 0) != cudaSuccess))
        return cuda_fail(nullptr, "push join", cudaGetLastError());
  }
  for (size_t i = 0; i < n; ++i) {
    hists[i] = outs[i].opcode_hist;
    aiwc_handle* h = hs[i];
    aiwc_status s = pushed[i] != AIWC_OK ? pushed[i] : (h->broken ? recover(h) : prepare(h));
    if (s != AIWC_OK) {
      live[i] = 0;
      memset(&outs[i], 0, sizeof(aiwc_metrics));
      outs[i].opcode_hist = hists[i];
      if (worst == AIWC_OK) worst = s;
    }
  }
  // one synchronisation for every handle's ingest-time counters
  for (size_t i = 0; i < n; ++i)
    if (live[i])
      if (cudaMemcpyAsync(hs[i]->h_state, &hs[i]->arena->st, sizeof(DevState), cudaMemcpyDeviceToHost, user) !=
          cudaSuccess)
        return cuda_fail(nullptr, "batch state copy", cudaGetLastError());
  if (cudaStreamSynchronize(user) != cudaSuccess) return cuda_fail(nullptr, "batch sync", cudaGetLastError());
  std::vector<Plan> plans(n);
  BatchGraph& bg = batch_graph(hs[0]->cfg.device);
  std::vector<u64> sig;
  for (size_t i = 0; i < n; ++i) {
    if (!live[i]) continue;
    plans[i].gated = true;
    plan_from_ingest(hs[i], &plans[i]);
    const aiwc_handle* h = hs[i];
    // the branch-path choice needs the number of sites and of long sites,
    // known only on the device; where the per-site path is certain anyway the
    // graph holds it alone (gated, both paths are launched and a device flag
    // picks one)
    const bool cs = site_sort_ok(h);
    plans[i].long_sites = h->n_br > kSiteMaxLen;
    if (per_site_certain(h, cs)) {
      plans[i].gated = false;
      plans[i].per_site = true;
      plans[i].site_sort = cs;
    }
    sig.insert(sig.end(), {(u64)(uintptr_t)h, h->n_mem, h->n_br, h->n_runs, h->epoch, (u64)plans[i].hash_ok,
                           (u64)plans[i].gated | ((u64)plans[i].site_sort << 1) | ((u64)plans[i].long_sites << 2),
                           plans[i].br_passes, plans[i].run_passes, h->sbt_cap, (u64)plans[i].seg_shift,
                           active_passes(h->h_state->mem_or, h->h_state->mem_and, ~0ull)});
  }
  aiwc_status s = bg.run(sig, user, [&](cudaStream_t base, std::vector<cudaStream_t>& forks) -> aiwc_status {
    size_t k = 0;
    for (size_t i = 0; i < n; ++i) {
      if (!live[i]) continue;
      aiwc_handle* h = hs[i];
      cudaStream_t st = forks[k++ % forks.size()];
      const bool timing = h->timing;
      h->timing = false;  // stage events are not part of the graph
      enqueue_part1(h, st, plans[i]);
      aiwc_status e = enqueue_part2(h, st, plans[i]);
      h->timing = timing;
      if (e != AIWC_OK) return e;
    }
    (void)base;
    return AIWC_OK;
  });
  if (s != AIWC_OK) {
    for (size_t i = 0; i < n; ++i) hs[i]->broken = true;
    return s;
  }
  for (size_t i = 0; i < n; ++i) {
    if (!live[i]) continue;
    aiwc_status e = finish(hs[i], &outs[i], hists[i]);
    if (e != AIWC_OK && worst == AIWC_OK) worst = e;
  }
  return worst;
}

aiwc_status aiwc_aggregate(const aiwc_metrics* runs, size_t n, int mode, aiwc_metrics* out) {
  if (!out || (n && !runs)) return fail(nullptr, AIWC_EINVAL, "null aggregate argument");
  if (mode != AIWC_AGG_SUM && mode != AIWC_AGG_MEDIAN) return fail(nullptr, AIWC_EINVAL, "unknown aggregate mode");
  // every numeric field of aiwc_metrics, by offset
  static const size_t kU64[] = {
      offsetof(aiwc_metrics, total_instructions), offsetof(aiwc_metrics, unique_opcodes),
      offsetof(aiwc_metrics, opcode_cover), offsetof(aiwc_metrics, work_items), offsetof(aiwc_metrics, barriers),
      offsetof(aiwc_metrics, itb_count), offsetof(aiwc_metrics, itb_min), offsetof(aiwc_metrics, itb_max),
      offsetof(aiwc_metrics, itb_median_lo), offsetof(aiwc_metrics, itb_median_hi),
      offsetof(aiwc_metrics, ipt_count), offsetof(aiwc_metrics, ipt_min), offsetof(aiwc_metrics, ipt_max),
      offsetof(aiwc_metrics, ipt_median_lo), offsetof(aiwc_metrics, ipt_median_hi),
      offsetof(aiwc_metrics, total_reads), offsetof(aiwc_metrics, total_writes), offsetof(aiwc_metrics, footprint),
      offsetof(aiwc_metrics, footprint_cover), offsetof(aiwc_metrics, unique_reads),
      offsetof(aiwc_metrics, unique_writes), offsetof(aiwc_metrics, branch_events),
      offsetof(aiwc_metrics, branch_sites), offsetof(aiwc_metrics, branch_cover),
      offsetof(aiwc_metrics, branch_patterns), offsetof(aiwc_metrics, branch_minsum),
      offsetof(aiwc_metrics, simd_count), offsetof(aiwc_metrics, simd_max), offsetof(aiwc_metrics, simd_sum),
      offsetof(aiwc_metrics, simd_sumsq)};
  std::vector<size_t> f64 = {
      offsetof(aiwc_metrics, itb_median), offsetof(aiwc_metrics, ipt_median), offsetof(aiwc_metrics, albe),
      offsetof(aiwc_metrics, yokota),
      offsetof(aiwc_metrics, unique_rw_ratio), offsetof(aiwc_metrics, reread_ratio),
      offsetof(aiwc_metrics, rewrite_ratio), offsetof(aiwc_metrics, simd_mean), offsetof(aiwc_metrics, simd_sd),
      offsetof(aiwc_metrics, granularity), offsetof(aiwc_metrics, barriers_per_instruction),
      offsetof(aiwc_metrics, instructions_per_operand), offsetof(aiwc_metrics, load_imbalance)};
  for (int l = 0; l <= AIWC_MAX_SKIP; ++l) f64.push_back(offsetof(aiwc_metrics, entropy) + l * sizeof(double));
  uint64_t* keep_hist = out->opcode_hist;
  aiwc_metrics r;
  memset(&r, 0, sizeof(r));
  auto u64_at = [](const aiwc_metrics& m, size_t off) {
    uint64_t v;
    memcpy(&v, reinterpret_cast<const char*>(&m) + off, 8);
    return v;
  };
  auto f64_at = [](const aiwc_metrics& m, size_t off) {
    double v;
    memcpy(&v, reinterpret_cast<const char*>(&m) + off, 8);
    return v;
  };
  for (size_t off : kU64) {
    uint64_t v = 0;
    if (mode == AIWC_AGG_SUM) {
      for (size_t i = 0; i < n; ++i) v += u64_at(runs[i], off);
    } else if (n) {
      std::vector<uint64_t> xs(n);
      for (size_t i = 0; i < n; ++i) xs[i] = u64_at(runs[i], off);
      std::sort(xs.begin(), xs.end());
      v = xs[(n - 1) / 2];
    }
    memcpy(reinterpret_cast<char*>(&r) + off, &v, 8);
  }
  for (size_t off : f64) {
    double v = 0.0;
    if (mode == AIWC_AGG_SUM) {
      for (size_t i = 0; i < n; ++i) v += f64_at(runs[i], off);
    } else if (n) {
      std::vector<double> xs(n);
      for (size_t i = 0; i < n; ++i) xs[i] = f64_at(runs[i], off);
      std::sort(xs.begin(), xs.end());
      v = 0.5 * (xs[(n - 1) / 2] + xs[n / 2]);
    }
    memcpy(reinterpret_cast<char*>(&r) + off, &v, 8);
  }
  r.opcode_hist = keep_hist;
  *out = r;
  return AIWC_OK;
}

aiwc_status aiwc_destroy(aiwc_handle* h) {
  if (!h) return AIWC_OK;
  DeviceGuard g(h->cfg.device);
  if (h->stream || h->copy_stream) cudaStreamSynchronize(h->stream);
  if (h->side_stream) cudaStreamSynchronize(h->side_stream);
  DevBuf* bufs[] = {&h->mem_a, &h->mem_b, &h->br_a, &h->br_b, &h->br_c, &h->pat_a, &h->pat_b, &h->rk_a, &h->rk_b,
                    &h->run_sum, &h->over_a, &h->over_b, &h->counts, &h->bsums, &h->tiles, &h->stage[0],
                    &h->stage[1], &h->desc, &h->sbt, &h->sbt_scan, &h->sites, &h->over_total,
                    &h->exp_meta, &h->shard_tmp};
  for (DevBuf* b : bufs) release(h, *b);
  if (h->total) cudaFree(h->total);
  if (h->wi_bitmap) cudaFree(h->wi_bitmap);
  if (h->arena) cudaFree(h->arena);
  if (h->d_result) cudaFree(h->d_result);  // the histograms live in the same allocations
  if (h->h_result) cudaFreeHost(h->h_result);
  if (h->h_state) cudaFreeHost(h->h_state);
  if (h->h_exp) cudaFreeHost(h->h_exp);
  for (int i = 0; i < 2; ++i) {
    if (h->ev_copied[i]) cudaEventDestroy(h->ev_copied[i]);
    if (h->ev_free[i]) cudaEventDestroy(h->ev_free[i]);
  }
  for (auto& iv : h->intervals) {
    cudaEventDestroy(iv.a);
    cudaEventDestroy(iv.b);
  }
  for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side_stream) cudaStreamDestroy(h->side_stream);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  delete h;
  return AIWC_OK;
}

}  // extern "C"

namespace {

// Host blob of one rank's exact distributions (aiwc_shard_export): this
// header, the arena (every dense distribution and counter), the overflow
// entries, the opcode histogram and the words of the work-item bitmap that
// hold the rank's work-items. Valid between builds of the same library only:
// the arena's layout is internal, its size is checked.
struct ShardHeader {
  uint64_t magic;
  uint32_t version, arena_bytes;
  uint32_t n_opcodes, history_len, space_mask, byte_addresses, history_scope, pad;
  uint64_t max_wi;
  uint64_t n_over;
  uint64_t wi_word0, wi_words;
};
constexpr uint64_t kShardMagic = 0x3144524853435741ull;  // "AWCSHRD1" in little-endian bytes
constexpr uint32_t kShardVersion = 1;

size_t shard_blob_bytes(const ShardHeader& hd) {
  return sizeof(ShardHeader) + hd.arena_bytes + 8 * hd.n_over + 8ull * hd.n_opcodes + 4 * hd.wi_words;
}

// Reduces what the handle holds with the finalisation deferred, copies the
// distributions into h->shard_blob and resets the handle.
aiwc_status shard_capture(aiwc_handle* h) {
  cudaStream_t st = h->stream;
  aiwc_status s = reduce_current(h, true);
  if (s != AIWC_OK) return s;
  CK(cudaStreamSynchronize(st));
  CK(cudaMemcpy(h->h_state, &h->arena->st, sizeof(DevState), cudaMemcpyDeviceToHost));
  const DevState& ds = *h->h_state;
  ShardHeader hd{};
  hd.magic = kShardMagic;
  hd.version = kShardVersion;
  hd.arena_bytes = (uint32_t)sizeof(Arena);
  hd.n_opcodes = h->cfg.n_opcodes;
  hd.history_len = h->cfg.history_len;
  hd.space_mask = h->cfg.space_mask;
  hd.byte_addresses = h->cfg.byte_addresses;
  hd.history_scope = h->cfg.history_scope;
  hd.max_wi = h->max_wi;
  hd.n_over = std::min<u64>(ds.n_over, h->c_over_cap);  // an overflow is flagged in the arena's error bits
  if (ds.wi_min <= ds.wi_max && h->wi_bitmap) {
    hd.wi_word0 = ds.wi_min >> 5;
    hd.wi_words = (ds.wi_max >> 5) - hd.wi_word0 + 1;
  }
  h->shard_blob.resize(shard_blob_bytes(hd));
  uint8_t* b = h->shard_blob.data();
  memcpy(b, &hd, sizeof(hd));
  b += sizeof(hd);
  CK(cudaMemcpy(b, h->arena, sizeof(Arena), cudaMemcpyDeviceToHost));
  b += sizeof(Arena);
  if (hd.n_over) CK(cudaMemcpy(b, h->over_a.p, 8 * hd.n_over, cudaMemcpyDeviceToHost));
  b += 8 * hd.n_over;
  CK(cudaMemcpy(b, h->d_hist, 8ull * hd.n_opcodes, cudaMemcpyDeviceToHost));
  b += 8ull * hd.n_opcodes;
  if (hd.wi_words) CK(cudaMemcpy(b, h->wi_bitmap + hd.wi_word0, 4 * hd.wi_words, cudaMemcpyDeviceToHost));
  if ((s = reset_device_state(h, st, true)) != AIWC_OK) return s;
  CK(cudaStreamSynchronize(st));
  collect_stage_times(h);
  reset_host(h);
  return AIWC_OK;
}

}  // namespace

extern "C" {

aiwc_status aiwc_shard_export(aiwc_handle* h, void* blob, size_t cap, size_t* size) {
  if (!h || !size) return fail(h, AIWC_EINVAL, "null handle or size pointer", false);
  DeviceGuard g(h->cfg.device);
  if (h->broken) return recover(h);
  if (!h->parts.empty())
    return fail(h, AIWC_EINVAL, "aiwc_shard_export: a partitioned handle cannot export a shard", false);
  if (h->shard_blob.empty()) {
    aiwc_status s = shard_capture(h);
    if (s != AIWC_OK) {
      h->shard_blob.clear();
      return s;
    }
  }
  *size = h->shard_blob.size();
  if (!blob) return AIWC_OK;
  if (cap < h->shard_blob.size())
    return fail(h, AIWC_EINVAL, "aiwc_shard_export: the blob buffer is smaller than *size", false);
  memcpy(blob, h->shard_blob.data(), h->shard_blob.size());
  h->shard_blob.clear();
  return AIWC_OK;
}

aiwc_status aiwc_shard_merge(aiwc_handle* h, const void* const* blobs, const size_t* sizes, size_t n,
                             aiwc_metrics* out) {
  if (!h || !out || (n && (!blobs || !sizes))) return fail(h, AIWC_EINVAL, "null argument", false);
  DeviceGuard g(h->cfg.device);
  uint64_t* user_hist = out->opcode_hist;
  if (h->broken) return recover(h);
  if (!h->parts.empty())
    return fail(h, AIWC_EINVAL, "aiwc_shard_merge: a partitioned handle cannot merge shards", false);
  if (h->n_mem || h->n_br || h->n_runs || !h->pend_wi.empty() || !h->deferred.empty())
    return fail(h, AIWC_ESTATE, "aiwc_shard_merge: the handle holds pushed events of another invocation", false);
  // check every blob before anything is merged
  std::vector<ShardHeader> hds(n);
  u64 total_cap = 0, max_over = 0, max_words = 0;
  const u64 bitmap_words = (h->max_wi + 31) / 32;
  for (size_t i = 0; i < n; ++i) {
    if (!blobs[i] || sizes[i] < sizeof(ShardHeader)) return fail(h, AIWC_EINVAL, "shard blob too short", false);
    ShardHeader& hd = hds[i];
    memcpy(&hd, blobs[i], sizeof(hd));
    if (hd.magic != kShardMagic || hd.version != kShardVersion || hd.arena_bytes != sizeof(Arena))
      return fail(h, AIWC_EINVAL, "not a shard blob of this library build", false);
    if (hd.n_opcodes != h->cfg.n_opcodes || hd.history_len != h->cfg.history_len ||
        hd.space_mask != h->cfg.space_mask || hd.byte_addresses != h->cfg.byte_addresses ||
        hd.history_scope != h->cfg.history_scope || hd.max_wi != h->max_wi)
      return fail(h, AIWC_EINVAL, "shard blob reduced under another metric configuration", false);
    if (hd.wi_words > bitmap_words || hd.wi_word0 > bitmap_words - hd.wi_words || hd.n_over > (1ull << 40) ||
        sizes[i] != shard_blob_bytes(hd))
      return fail(h, AIWC_EINVAL, "shard blob size or work-item range is inconsistent", false);
    total_cap += hd.n_over;
    max_over = std::max<u64>(max_over, hd.n_over);
    max_words = std::max<u64>(max_words, hd.wi_words);
  }
  cudaStream_t st = h->stream;
  aiwc_status s;
  if (!h->total) {
    CK(cudaMalloc(&h->total, sizeof(Arena)));
    h->bytes += sizeof(Arena);
  }
  ENSURE(h->over_total, std::max<u64>(total_cap, 1) * 8, false);
  ENSURE(h->over_a, std::max<u64>(max_over, 1) * 8, false);
  ENSURE(h->shard_tmp, std::max<u64>(8ull * h->cfg.n_opcodes, 4 * max_words), false);
  if ((s = ensure_bitmap(h)) != AIWC_OK) return s;
  CK(cudaMemsetAsync(h->total, 0, sizeof(Arena), st));
  launch_reset_identities(h->total, st);
  for (size_t i = 0; i < n; ++i) {
    const ShardHeader& hd = hds[i];
    const uint8_t* b = static_cast<const uint8_t*>(blobs[i]) + sizeof(ShardHeader);
    // the handle's own arena and overflow list stage this rank's distributions
    CK(cudaMemcpyAsync(h->arena, b, sizeof(Arena), cudaMemcpyHostToDevice, st));
    b += sizeof(Arena);
    if (hd.n_over) CK(cudaMemcpyAsync(h->over_a.p, b, 8 * hd.n_over, cudaMemcpyHostToDevice, st));
    b += 8 * hd.n_over;
    launch_merge_partition(h->arena, (const u64*)h->over_a.p, hd.n_over, h->total, (u64*)h->over_total.p,
                           total_cap, st);
    CK(cudaMemcpyAsync(h->shard_tmp.p, b, 8ull * hd.n_opcodes, cudaMemcpyHostToDevice, st));
    launch_add_u64((u64*)h->d_hist, (const u64*)h->shard_tmp.p, hd.n_opcodes, h->sm_count, st);
    b += 8ull * hd.n_opcodes;
    if (hd.wi_words) {
      CK(cudaMemcpyAsync(h->shard_tmp.p, b, 4 * hd.wi_words, cudaMemcpyHostToDevice, st));
      launch_or_u32(h->wi_bitmap + hd.wi_word0, (const u32*)h->shard_tmp.p, hd.wi_words, h->sm_count, st);
    }
  }
  CK(cudaGetLastError());
  return finalize_merged(h, total_cap, out, user_hist);
}

const char* aiwc_last_error(const aiwc_handle* h) { return h ? h->err.c_str() : g_last_error.c_str(); }

uint64_t aiwc_device_bytes(const aiwc_handle* h) { return h ? (uint64_t)h->bytes : 0; }

uint64_t aiwc_kernel_launches(void) { return launches_so_far(); }

}  // extern "C"

bool aiwc::handle_config_matches(const aiwc_handle* h, const aiwc_config* c) {
  const aiwc_config& a = h->cfg;
  return a.history_len == c->history_len && a.cover_num == c->cover_num && a.cover_den == c->cover_den &&
         a.n_opcodes == c->n_opcodes && a.space_mask == (c->space_mask & 0xFu) && a.precision == c->precision &&
         a.plan == c->plan && a.max_work_items == c->max_work_items && a.table_slots == c->table_slots &&
         a.byte_addresses == c->byte_addresses && a.history_scope == c->history_scope &&
         a.defer_pushes == c->defer_pushes;
}

void aiwc::handle_set_budget(aiwc_handle* h, uint64_t bytes) { h->cfg.hbm_budget = bytes; }

extern "C" {

aiwc_status aiwc_set_stage_timing(aiwc_handle* h, int on) {
  if (!h) return fail(nullptr, AIWC_EINVAL, "null handle");
  h->timing = on != 0;
  return AIWC_OK;
}

int aiwc_stage_times(const aiwc_handle* h, double* ms, const char** names, int n) {
  if (!h || n <= 0) return 0;
  const int k = n < kNumStages ? n : kNumStages;
  for (int i = 0; i < k; ++i) {
    if (ms) ms[i] = h->stage_last[i];
    if (names) names[i] = kStageNames[i];
  }
  return k;
}

}  // extern "C"
