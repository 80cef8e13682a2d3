// Memory metrics of one small invocation using no device allocation at all.
//
// Some callers may not call cudaMalloc / cudaFree: code whose device memory is
// owned by another allocator (a framework's caching allocator, a fixed pool)
// and code that must not trigger the device-wide synchronisation that
// cudaFree implies. For them this entry point runs the memory path of the
// reduction (ingest with the superblock table, segment histograms, overflow
// sort, finalize) with every scratch buffer carved out of one file-scope
// device array, sized for at most kNoAllocMaxEvents events. The array is
// part of the library's image: every device that loads the library holds it
// until the process exits.
#include <mutex>
#include <string>

#include "aiwc_internal.cuh"

namespace aiwc {
namespace {

constexpr u64 kNoAllocMaxEvents = 1ull << 18;  // memory events per call
constexpr u64 kNoAllocSlots = 1ull << 19;      // superblock table: load factor <= 1/2
constexpr u64 kNoAllocMaxWi = 1ull << 20;      // work-item ids per call
constexpr u64 kNoAllocOverCap = (u64)kLevels * (kNoAllocMaxEvents / kCocDense + 2) + 256;

constexpr size_t a256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr u64 tiles_of(u64 n) { return (n + kTile - 1) / kTile; }

constexpr size_t kOffArena = 0;
constexpr size_t kOffResult = kOffArena + a256(sizeof(Arena));
constexpr size_t kOffWords = kOffResult + a256(sizeof(Result));
constexpr size_t kOffSlot = kOffWords + a256(8 * kNoAllocMaxEvents);
constexpr size_t kOffLow = kOffSlot + a256(8 * kNoAllocMaxEvents);
constexpr size_t kOffTable = kOffLow + a256(2 * kNoAllocMaxEvents);
constexpr size_t kOffScan = kOffTable + a256(kSbtBytes * kNoAllocSlots);
constexpr size_t kOffOverA = kOffScan + a256(4 * (kNoAllocSlots / 4096 + 1));
constexpr size_t kOffOverB = kOffOverA + a256(8 * kNoAllocOverCap);
// the radix sort's scratch for this capacity (tiles of 2048 keys): look-back
// words or digit counts, then digit totals and tile tickets
constexpr size_t kCountsWords = 512 * ((kNoAllocOverCap + 2047) / 2048);
constexpr size_t kOffCounts = kOffOverB + a256(8 * kNoAllocOverCap);
constexpr size_t kOffBsums = kOffCounts + a256(4 * kCountsWords);
constexpr size_t kOffBitmap = kOffBsums + a256(4 * (8 * 256 + 16));
constexpr size_t kOffBig = kOffBitmap + a256(kNoAllocMaxWi / 8);
constexpr size_t kNoAllocBigBytes = (kNoAllocMaxEvents / 16384) * 2 * 2048 * 4;  // wide-segment histograms
constexpr size_t kNoAllocBytes = kOffBig + a256(kNoAllocBigBytes);

static_assert(kNoAllocBytes <= (32ull << 20), "the no-allocation scratch must stay modest");

// The scratch every call of aiwc_mem_metrics_noalloc shares (one per device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device addresses of g_noalloc_scratch and SM counts, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// Makes device d current for the call and restores the caller's device.
struct Guard {
  int prev = -1;
  bool ok = true;
  explicit Guard(int d) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      prev = -1;
    }
    if (prev != d && cudaSetDevice(d) != cudaSuccess) {
      cudaGetLastError();
      ok = false;
    }
  }
  ~Guard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

aiwc_status fail(aiwc_status s, const std::string& msg) {
  set_last_error(msg);
  return s;
}

}  // namespace
}  // namespace aiwc

using namespace aiwc;

extern "C" aiwc_status aiwc_mem_metrics_noalloc(int device, void* cuda_stream, const aiwc_mem_event* events,
                                                size_t n, uint32_t space_mask, aiwc_metrics* out) {
  if (!out) return fail(AIWC_EINVAL, "null output");
  uint64_t* user_hist = out->opcode_hist;
  // on any error every field reads zero (the caller's histogram pointer kept)
  *out = aiwc_metrics{};
  out->opcode_hist = user_hist;
  if (n && !events) return fail(AIWC_EINVAL, "null events");
  if (n > kNoAllocMaxEvents)
    return fail(AIWC_EINVAL, "aiwc_mem_metrics_noalloc takes at most 262144 (2^18) memory events per call");
  if ((uintptr_t)events & 15u) return fail(AIWC_EINVAL, "device memory events must be 16-byte aligned");
  int n_dev = 0;
  cudaError_t e = cudaGetDeviceCount(&n_dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(AIWC_ECUDA, std::string("cudaGetDeviceCount: ") + cudaGetErrorString(e));
  }
  if (device < 0 || device >= n_dev || device >= kMaxDevices)
    return fail(AIWC_EINVAL, "aiwc_mem_metrics_noalloc: no CUDA device " + std::to_string(device));
  Guard g(device);
  if (!g.ok) return fail(AIWC_EINVAL, "aiwc_mem_metrics_noalloc: cannot make device " + std::to_string(device) +
                                          " current");
  if (n) {
    // the events must be memory this device can read: device memory of another
    // device, or plain pageable host memory, would be a fault, not an error
    cudaPointerAttributes pa{};
    e = cudaPointerGetAttributes(&pa, events);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(AIWC_EINVAL, std::string("aiwc_mem_metrics_noalloc: events pointer: ") + cudaGetErrorString(e));
    }
    if (pa.type == cudaMemoryTypeUnregistered)
      return fail(AIWC_EINVAL, "aiwc_mem_metrics_noalloc: events must be device memory");
    if (pa.type == cudaMemoryTypeDevice && pa.device != device)
      return fail(AIWC_EINVAL, "aiwc_mem_metrics_noalloc: events live on device " + std::to_string(pa.device) +
                                   ", not on device " + std::to_string(device));
  }
  void* base = nullptr;
  int sms = 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[device]) {
      // set-up on the first call on this device, with the device current
      void* addr = nullptr;
      e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(AIWC_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
      int count = 0;
      e = cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, device);
      if (e != cudaSuccess || count < 1) {
        cudaGetLastError();
        return fail(AIWC_ECUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
      }
      g_sms[device] = count;
      g_addr[device] = addr;
    }
    base = g_addr[device];
    sms = g_sms[device];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  char* p = (char*)base;
  Arena* arena = (Arena*)(p + kOffArena);
  Result* result = (Result*)(p + kOffResult);
  SbTable tab;
  tab.keys = (u64*)(p + kOffTable);
  tab.cnt = (u32*)(p + kOffTable + 8 * kNoAllocSlots);
  tab.off = (u32*)(p + kOffTable + kSbtClearBytes * kNoAllocSlots);
  tab.mask = kNoAllocSlots - 1;
  u32* used_list = (u32*)(p + kOffTable + (kSbtClearBytes + 4) * kNoAllocSlots);
  u32* bitmap = (u32*)(p + kOffBitmap);
  // the previous call's contents remain: clear what has to start at zero
  if ((e = cudaMemsetAsync(arena, 0, sizeof(Arena), s)) != cudaSuccess ||
      (e = cudaMemsetAsync(tab.keys, 0, kSbtClearBytes * kNoAllocSlots, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(bitmap, 0, kNoAllocMaxWi / 8, s)) != cudaSuccess)
    return fail(AIWC_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  launch_reset_identities(arena, s);
  MemIngestArgs ia;
  ia.tab = tab;
  ia.use_tab = 1;
  ia.slotw = (u64*)(p + kOffSlot);
  ia.spill = (u64*)(p + kOffWords);
  ia.ev = events;
  ia.n = n;
  ia.space_mask = space_mask & 0xFu;
  ia.words = (u64*)(p + kOffWords);
  ia.word_base = 0;
  ia.wi_bitmap = bitmap;
  ia.max_wi = kNoAllocMaxWi;
  ia.arena = arena;
  launch_mem_ingest(ia, s);
  u64* over_a = (u64*)(p + kOffOverA);
  u64* over_b = (u64*)(p + kOffOverB);
  HashArgs ha;
  ha.slotw = ia.slotw;
  ha.n_cap = kNoAllocMaxEvents;
  ha.low = (uint16_t*)(p + kOffLow);
  ha.tab = tab;
  ha.scan_tmp = (u32*)(p + kOffScan);
  ha.n_used = arena->st.sb_used;
  ha.used_list = used_list;
  ha.over = over_a;
  ha.over_cap = kNoAllocOverCap;
  ha.arena = arena;
  ha.grid_scatter = sms * 8;  // the launch shapes of the handle path
  ha.sm_count = sms;
  ha.seg_shift = 0;  // the event alignment is not read back: the general layout
  ha.big_hist = (u32*)(p + kOffBig);
  ha.big_cap = mem_hash_big_segments(n, kNoAllocBigBytes, 0);
  launch_mem_hash(ha, s);
  launch_wi_count(bitmap, arena, s);
  SortDesc d;
  d.a = over_a;
  d.b = over_b;
  d.cur = &arena->st.sort_cur[kSortOver];
  d.n = &arena->st.n_over;
  d.n_cap = kNoAllocOverCap;
  d.key_or = &arena->st.over_or;
  d.key_and = &arena->st.over_and;
  d.mask = ~0ull;
  d.dmask = nullptr;
  d.lo_bit = 0;
  d.counts = (u32*)(p + kOffCounts);
  d.block_sums = (u32*)(p + kOffBsums);
  d.ntiles = sort_tiles(kNoAllocOverCap);
  sort_keys(d, s);
  FinalizeArgs fa;
  fa.over_a = over_a;
  fa.over_b = over_b;
  fa.over_cur = d.cur;
  fa.over_cap = kNoAllocOverCap;
  fa.arena = arena;
  fa.result = result;
  fa.cover_num = 9;
  fa.cover_den = 10;
  fa.precision = 0;
  fa.history_len = 16;  // no branch events: the Yokota entropy is 0
  launch_finalize(fa, s);
  Result r;
  u32 table_overflow = 0;
  if ((e = cudaGetLastError()) != cudaSuccess ||
      (e = cudaMemcpyAsync(&r, result, sizeof(Result), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&table_overflow, &arena->st.sbt_overflow, 4, cudaMemcpyDeviceToHost, s)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return fail(AIWC_ECUDA, std::string("aiwc_mem_metrics_noalloc: ") + cudaGetErrorString(e));
  if (table_overflow) return fail(AIWC_ENOMEM, "superblock table of the no-allocation scratch overflowed");
  if (r.err & kErrOverflow) return fail(AIWC_ENOMEM, "overflow list of the no-allocation scratch overflowed");
  if (r.err & kErrAddr) return fail(AIWC_EINVAL, "memory address outside the 61-bit domain");
  if (r.err & kErrWorkItem) return fail(AIWC_EINVAL, "work-item id >= 2^20 in aiwc_mem_metrics_noalloc");
  *out = r.m;
  out->opcode_hist = user_hist;
  return AIWC_OK;
}
