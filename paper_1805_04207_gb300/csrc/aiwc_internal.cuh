// Internal declarations shared by the AIWC CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include <cstddef>

#include "aiwc.h"

namespace aiwc {

typedef unsigned long long u64;
typedef unsigned int u32;

// ------------------------------------------------------------------ sizes
constexpr int kLevels = AIWC_MAX_SKIP + 1;  // skip 0 (global) .. 10 (local)
constexpr int kCocDense = 4096;             // group sizes below this are binned densely
constexpr int kCocShared = 1024;            // ... and below this first in a block's shared bins
constexpr int kValDense = 65536;            // ITB / IPT values below this are binned densely
constexpr int kValSmem = 2048;              // ... of which the smallest are privatised in shared memory
constexpr int kTile = 4096;                 // elements per tile in the sort and run kernels
constexpr int kTileThreads = 256;
constexpr int kTileItems = kTile / kTileThreads;

// Tags of the shared overflow list: entry = tag << 56 | value.
constexpr int kTagSites = 16;
constexpr int kTagOpcodes = 17;
constexpr int kTagItb = 18;
constexpr int kTagIpt = 19;
constexpr int kTagPat = 20;      // predicted outcomes per (site, history) pattern >= kValDense
constexpr int kTagSitePat = 21;  // predicted outcomes per site >= kValDense
constexpr int kNumTags = 22;
constexpr u64 kValueMask = (1ull << 56) - 1;

// Error flags raised on the device (DevState::err).
constexpr u32 kErrAddr = 1u;        // memory address >= 2^61
constexpr u32 kErrOpcode = 2u;      // opcode >= n_opcodes and not a barrier
constexpr u32 kErrWorkItem = 4u;    // work-item id >= max_work_items
constexpr u32 kErrOverflow = 8u;    // an internal list exceeded its capacity
constexpr u32 kErrRun = 16u;        // a run reaches past its opcode array
constexpr u32 kErrSort = 32u;       // a sort's bounded wait for an earlier tile gave up

// Device-resident counters of one invocation. Zeroed by a memset, then the
// AND accumulators and minima are set to their identities.
struct DevState {
  u64 n_words;           // memory words after the space filter
  u64 total_reads, total_writes;
  u64 mem_or, mem_and;   // OR / AND over memory words: varying bits = or ^ and
  u64 footprint, unique_reads, unique_writes;
  u64 br_or, br_and;
  u64 n_patterns;        // outcomes with a full history
  u64 pat_or, pat_and;
  u64 branch_sites;
  u64 minsum, npat;
  u64 barriers;
  u64 run_or, run_and;
  u64 work_items;
  u64 n_over;            // entries in the overflow list
  u64 over_or, over_and;
  u64 unique_opcodes, total_instructions;
  u64 n_branch;          // branch events pushed
  u64 n_runs;            // instruction runs pushed
  u32 wi_min, wi_max;
  u32 err;
  u32 sbt_overflow;      // the superblock table could not place a key
  u32 pad2;
  u64 sb_used[2];        // occupied superblock slots: below / at or above the wide-block threshold
  u64 n_spill;           // hash plan: events whose superblock the table could not place
  u64 br_site_max;       // longest per-site outcome sequence
  u64 n_sites;           // entries of the site list
  u64 n_long;            // sites longer than kSiteMaxLen (counted in chunks by the per-site path)
  u64 long_next;         // entries of the long-site list
  u32 br_unsorted;       // some work-item id arrived below its predecessor
  u32 br_persite;        // the per-site branch path applies (set on the device)
  u32 br_last_wi[2];     // last work-item id of the previous / current push (by push parity)
  u32 run_unsorted;      // some run key is below its predecessor (the run sort is needed)
  u64 simd_count, simd_sum, simd_sumsq, simd_max;  // result widths of executed instructions
  u32 sort_cur[8];       // which ping-pong buffer holds each sort's data
  u32 pad;
};

// Open-addressing table of memory superblocks (key >> 11), kept in L2.
// keys[s] = superblock + 1 (0 = empty); cnt[s] = its events; off/cur =
// segment offset and scatter cursor. Capacity mask + 1 is a power of two.
constexpr u32 kNoSlot = 0xFFFFFFFFu;
constexpr int kMaxProbe = 256;
// Superblock table, C = mask + 1 slots: keys u64[C] | cnt u32[kSbtStripes][C]
// | off u32[C] | used u32[C]. The ingest counts an event in the counter stripe
// of its warp (global warp index mod kSbtStripes), so a hot superblock's
// counting atomics spread over kSbtStripes addresses; its rank is counted
// within that stripe. The offset scan leaves each slot's total in stripe 0
// and, in stripe s > 0, the offset where stripe s starts in the slot's
// segment (off[] holds stripe 0's).
constexpr int kStripeBits = 2;
constexpr int kSbtStripes = 1 << kStripeBits;
constexpr u64 kSbtClearBytes = 8 + 4 * kSbtStripes;  // per slot: keys and counters start at zero
constexpr u64 kSbtBytes = kSbtClearBytes + 8;        // per slot, with the offset and the used list
struct SbTable {
  u64* keys{};
  u32* cnt{};   // stripe s of slot i: cnt[s * (mask + 1) + i]
  u32* off{};
  u64 mask{};
};
// Slot word of the hash plan: rank << kRankShift | stripe << 32 | slot << 12
// | the word's low 12 bits; a rank >= kRankLimit sends the invocation to the
// sort plan (as a full table does).
constexpr int kRankShift = 32 + kStripeBits;
constexpr u32 kRankLimit = 1u << (32 - kStripeBits);

// Sort slots (index into DevState::sort_cur).
enum SortSlot { kSortMem = 0, kSortBranch = 1, kSortPattern = 2, kSortRuns = 3, kSortOver = 4 };

// Per-tile run summary for the cross-tile fix-up (see runs.cuh).
struct TileSum {
  u32 has_b;
  u32 pad;
  u64 pre, suf, tot;     // lengths: before the first head, from the last head, all
  u64 pre_w, suf_w, tot_w;  // the same, summing a per-element weight
};

// Dense distributions and the result live in one arena (one memset resets it).
struct Arena {
  DevState st;
  u64 mem_coc[kLevels][kCocDense];   // m_c for group sizes c < kCocDense, per skip level
  u64 site_coc[kCocDense];
  u64 opc_coc[kCocDense];
  alignas(16) u64 itb_dense[kValDense];
  alignas(16) u64 ipt_dense[kValDense];
  u64 pat_coc[kValDense];            // m_c of the predicted-outcome counts of history patterns (c < kValDense)
  double yok_part[16];               // finalize: partial sums of the Yokota entropy, combined by the last block
  u32 yok_done;
  u64 site_pat_coc[kValDense];       // m_c of the predicted-outcome counts of sites
  u64 tag_begin[kNumTags + 1];       // segment of each tag in the sorted overflow list
};
// the order statistics read the value bins 16 bytes at a time
static_assert(offsetof(Arena, itb_dense) % 16 == 0 && offsetof(Arena, ipt_dense) % 16 == 0,
              "value bins must be 16-byte aligned");

struct Result {
  aiwc_metrics m;  // opcode_hist pointer unused on the device
  u32 err;         // DevState::err at finalisation
  u32 pad;
};
// A handle keeps its opcode histogram right after its result (device and
// host alike), so that one copy brings both back.
constexpr size_t kHistOffset = (sizeof(Result) + 255) & ~size_t(255);
inline size_t result_bytes(u32 n_opcodes) { return kHistOffset + (size_t)n_opcodes * 8; }

// A radix sort over 64-bit keys held in a ping-pong pair (a, b); the live
// buffer is b when *cur is 1. Only bits in `mask` that vary between keys are
// sorted, in 8-bit windows starting at `lo_bit`.
struct SortDesc {
  const u32* gate{};   // run only when !gate || *gate == gate_want (device-side plan choice)
  u32 gate_want{};
  u64* a{};
  u64* b{};
  u32* cur{};
  const u64* n{};     // device count of keys (clamped to n_cap)
  u64 n_cap{};          // capacity of a and b, in keys
  const u64* key_or{};  // device OR over keys
  const u64* key_and{}; // device AND over keys
  u64 mask{};
  const u64* dmask{}; // optional device mask, ANDed with mask (NULL = none)
  const u32* unsorted{};  // branch words: the site bits alone when *unsorted == 0, else every bit but the outcome
  int lo_bit{};
  u32* counts{};      // sort_counts_words(n_cap) words: digit counts, or the one-sweep look-back words
  u32* block_sums{};  // sort_block_sums_words(n_cap) words: scan sums, or digit totals and tile tickets
  u32 ntiles{};
  u32* err{};         // DevState::err: kErrSort when a bounded wait gave up (NULL: not reported)
};

// Text returned by aiwc_last_error(NULL) on this thread.
void set_last_error(const std::string& msg);
// For the server: does h reduce with the same metric configuration as cfg
// (everything but device, stream and budget)? And set h's scratch budget.
bool handle_config_matches(const aiwc_handle* h, const aiwc_config* cfg);
void handle_set_budget(aiwc_handle* h, uint64_t bytes);

// Kernels launched by this library (process-wide, all handles).
void count_launches(u64 n);
u64 launches_so_far();

// ------------------------------------------------------------- launchers
// Launches the passes whose bit is set in host_passes (bit p: 8-bit window p);
// passes whose window holds no varying bit return at once on the device.
void sort_keys(const SortDesc& d, cudaStream_t s, u32 host_passes = 0xFFu);
size_t sort_counts_words(u64 n_max);  // u32 words needed for counts
u32 sort_tiles(u64 n);                // tiles of the sort for n keys (SortDesc::ntiles)
size_t sort_block_sums_words(u64 n_max);

constexpr u32 kSlotWordNone = 0xFFFFFFFFu;  // slot word of an event the table could not place
constexpr u64 kMaxHashSlots = 1ull << 20;   // slot words hold 20 slot bits

struct MemIngestArgs {
  SbTable tab{};       // used when use_tab (hash plan)
  int use_tab{};
  u64* slotw{};          // hash plan: out, slot word (low 32 bits) | counter stripe << 32 | rank << kRankShift
  u64* spill{};          // hash plan: out, full words of events the table could not place
  const void* ev{};      // 16-byte events
  u64 n{};
  u32 space_mask{};
  u64* words{};          // sort plan: out, 64-bit sort words
  u64 word_base{};       // offset for the unfiltered fast path
  u32* wi_bitmap{};
  u64 max_wi{};
  Arena* arena{};
};
void launch_mem_ingest(const MemIngestArgs& a, cudaStream_t s);

// Byte-granular addresses: the one-byte accesses of a chunk of memory events
// (addr + b for b < size, with the event's kind and space), for the events
// whose space is kept.
constexpr u64 kExpandTile = 1024;         // events per tile
constexpr u64 kExpandChunk = 1ull << 22;  // events per chunk (tile offsets for one chunk)
struct ExpandArgs {
  const void* ev{};   // 16-byte memory events (device, 16-byte aligned)
  u64 n{};            // events in the chunk, <= kExpandChunk
  u64* tile_off{};    // [ntiles] exclusive offsets of the tiles' one-byte events
  u64* total{};       // bytes the chunk touches
  u32* tile_sum{};    // [ntiles] bytes each tile touches
  u32 space_mask{};
  u32* wi_bitmap{};
  u64 max_wi{};
  Arena* arena{};
  int sm_count{};
};
size_t expand_meta_bytes();  // tile offsets and tile sums of one chunk (8 B and 4 B per tile)
// Counts the kept bytes of each tile, checks the start addresses and marks
// every event's work-item (the words carry none), then scans the tile counts
// into offsets and the chunk's total.
void launch_expand_count(const ExpandArgs& a, cudaStream_t s);
// Ingests a chunk's one-byte accesses (a.ev: its events, a.n of them) at
// a.word_base + the tile offsets from launch_expand_count; a byte at or above
// 2^61 raises the address error.
void launch_mem_ingest_bytes(const MemIngestArgs& a, const u64* tile_off, cudaStream_t s);

struct LevelArgs {
  const u32* gate{};   // run only when !gate || *gate == gate_want (device-side plan choice)
  u32 gate_want{};
  const u64* a{};
  const u64* b{};
  const u32* cur{};
  const u64* n{};
  TileSum* tiles{};      // kLevels * ntiles
  u32 ntiles{};
  u64* over{};
  u64 over_cap{};
  Arena* arena{};
  int grid{};
};
void launch_mem_levels(const LevelArgs& a, cudaStream_t s);

struct HashArgs {
  const u32* gate{};   // run only when !gate || *gate == gate_want (device-side plan choice)
  u32 gate_want{};
  const u64* slotw{};    // slot words | stripes << 32 | ranks << kRankShift from the ingest
  u64 n_cap{};           // capacity of slotw / low, in elements
  uint16_t* low{};       // out: low 12 bits grouped by superblock
  SbTable tab{};
  u32* scan_tmp{};     // sbt_scan_words(capacity) words
  u64* n_used{};         // out: occupied slots [0] below the wide-block threshold, [1] at or above it
  u32* used_list{};    // out: their indices (capacity = table slots)
  u64* over{};
  u64 over_cap{};
  Arena* arena{};
  u32* big_hist{};       // zeroed scratch: 2 * (2048 >> seg_shift) words per wide segment
  u64 big_cap{};         // wide segments big_hist holds (at least n_words / 16384)
  int grid_scatter{};
  int sm_count{};
  int seg_shift{};       // low address bits known to be zero in every event (0..3)
};
size_t sbt_scan_words(u64 cap);
void launch_mem_hash(const HashArgs& a, cudaStream_t s);           // both steps below
void launch_mem_hash_scatter(const HashArgs& a, cudaStream_t s);   // segment offsets, low bits into segments
void launch_mem_hash_segments(const HashArgs& a, cudaStream_t s);  // per-segment histograms and levels
// Wide segments (16384 events or more) a big_hist of `bytes` holds for n_words events.
u64 mem_hash_big_segments(u64 n_words, size_t bytes, int seg_shift);
// Fallback after a table overflow: rebuild the 64-bit sort words from the
// slot words and the table, after the n_spill spilled words already in words[].
void launch_rebuild_words(const u64* slotw, SbTable tab, u64* words, Arena* arena, int grid, cudaStream_t s,
                          const u32* gate = nullptr, u32 gate_want = 0);

struct BranchIngestArgs {
  u32 push_index{};    // pushes so far in this invocation (0 = first)
  const void* ev{};
  u64 n{};
  u64* words{};
  uint16_t* compact{};   // out: site << 1 | taken per event (sites below kCsSites; 0xFFFF otherwise)
  u64 word_base{};
  u32* wi_bitmap{};
  u64 max_wi{};
  Arena* arena{};
};
void launch_branch_ingest(const BranchIngestArgs& a, cudaStream_t s);

struct WindowArgs {
  const u32* gate{};   // run only when !gate || *gate == gate_want (device-side plan choice)
  u32 gate_want{};
  const u64* a{};      // sorted branch words (ping-pong)
  const u64* b{};
  const u32* cur{};
  u64 n{};               // branch events
  u32 h{};               // history length
  u32 gshift{32};        // one history per (word >> gshift): 32 = site, 1 = (site, work-item)
  bool site_pred{true};  // per-site predicted counts from the site runs (one history per site)
  u64* patterns{};     // out: compacted pattern words
  TileSum* tiles{};      // site-level tile summaries
  u32 ntiles{};
  u64* over{};
  u64 over_cap{};
  Arena* arena{};
  int grid{};
};
void launch_branch_windows(const WindowArgs& a, cudaStream_t s);

struct PatternArgs {
  const u32* gate{};   // run only when !gate || *gate == gate_want (device-side plan choice)
  u32 gate_want{};
  const u64* a{};
  const u64* b{};
  const u32* cur{};
  const u64* n{};      // valid pattern words (device)
  TileSum* tiles{};
  u32 ntiles{};
  u64* over{};           // pattern counts >= kValDense
  u64 over_cap{};
  Arena* arena{};
  int grid{};
  bool site_level{};     // also the site runs of the pattern words (tile summaries at tiles + ntiles):
                         // each site's predicted outcomes when histories are per (site, work-item)
};
void launch_pattern_runs(const PatternArgs& a, cudaStream_t s);

// Per-site path: list the site segments of the sorted branch words, then
// count (site, history) patterns of each site in shared memory.
struct SiteArgs {
  const u32* gate{};   // run only when !gate || *gate == gate_want (device-side plan choice)
  u32 gate_want{};
  const u64* a{};
  const u64* b{};
  const u32* cur{};
  u64 n{};               // branch events
  u32 h{};             // history length (<= kSiteMaxHist)
  u64* sites{};        // site list: one word per site, start << 32 | length
  u64 sites_cap{};
  u64* over{};
  u64 over_cap{};
  Arena* arena{};
  int grid{};
  const uint8_t* outcomes{};  // per-site path: outcome bytes sorted by site instead of the words
  bool per_wi{};       // one history per (site, work-item): needs the words (outcomes == nullptr)
  // sites longer than kSiteMaxLen: a dense table of 2^h (taken << 32 | total)
  // pattern counters per site, and per site (start, length, predicted outcomes)
  u64* long_tab{};
  u64* long_list{};
  u64 long_cap{};      // long sites the table and the list hold
};
// Stable counting sort of the branch words by site, for site ids below
// kCsSites when work-item ids arrived in non-decreasing order (the site alone
// then orders each site's history). Writes the same sorted words as the radix
// sort on the site bits, the site list and n_sites / br_site_max.
constexpr u32 kCsSites = 4096;
struct SiteSortArgs {
  const u64* src{};      // branch words in push order
  const uint16_t* src16{};  // the same events as site << 1 | taken (read when only sites and outcomes are needed)
  u64* dst{};            // out: words sorted by site (stable), or
  uint8_t* dst8{};       // out: just their outcome bits, one byte each (the per-site path reads no more)
  u32* sort_cur{};       // set to 1: dst is the live buffer
  u64 n{};
  u32* counts{};         // scratch: site_sort_count_words(n) words
  u32* chunks{};         // scratch: site_sort_chunk_words(n) words
  u64* sites{};          // out: start << 32 | length per site with events
  u64 sites_cap{};
  Arena* arena{};
  int sm_count{};
  u32 tile_shift{14};    // tiles of 2^tile_shift events (14 or 15): site_sort_tile_shift
};
size_t site_sort_count_words(u64 n);
size_t site_sort_chunk_words(u64 n);
u32 site_sort_tile_shift(u64 n, int sm_count);
void launch_site_sort_count(const SiteSortArgs& a, cudaStream_t s);    // counts, scan, site list
void launch_site_sort_scatter(const SiteSortArgs& a, cudaStream_t s);  // the sorted output

constexpr u32 kSiteMaxHist = 17;       // dense pattern bins: 2^15 per pass, at most 4 passes
constexpr u64 kSiteMaxLen = 65535;     // packed 16-bit taken / total counters
// Long sites: at most n / (kSiteMaxLen + 1) of n branch events; their tables
// take 8 << h bytes and their list entries 24 bytes each.
inline u64 long_sites_cap(size_t tab_bytes, size_t list_bytes, u32 h) {
  const u64 a = (u64)tab_bytes / (8ull << h), b = (u64)list_bytes / 24;
  return a < b ? a : b;
}
void launch_site_heads(const SiteArgs& a, cudaStream_t s);
// Device-side choice of the branch path: br_persite = the per-site path applies.
void launch_persite_decide(Arena* arena, u32 h, u64 sites_cap, u64 long_cap, int allow, cudaStream_t s);
void launch_site_patterns(const SiteArgs& a, cudaStream_t s);
// The long sites of the per-site path: list and clear, count chunks, walk the tables.
void launch_site_long(const SiteArgs& a, cudaStream_t s);

// Cross-tile fix-up of run lengths. kind: 0 = memory levels, 1 = sites, 2 = patterns.
// h: history length (kind 1, the site runs: each site predicts len - h outcomes).
void launch_runs_fixup(int kind, const TileSum* tiles, u32 ntiles_max, const u64* n_dev, u64 n_host,
                       int levels, u64* over, u64 over_cap, Arena* arena, cudaStream_t s,
                       const u32* gate = nullptr, u32 gate_want = 0, u32 h = 0);
// Set the attributes kernels with large dynamic shared memory need (current device).
void init_branch_attributes();
void init_instr_attributes();

struct RunBatchArgs {
  const uint16_t* ops{};
  u64 n_ops{};
  const u32* run_wi{};
  const u64* run_off{};
  const u64* run_len{};
  u64 n_runs{};
  u64 seq_base{};        // global index of the first run of this batch
  u32 n_opcodes{};
  u64* run_keys{};     // out: (wi << 32 | seq)
  u64* run_sum{};        // out: 4 words per run: has_b, pre, suf, tot
  u32* wi_bitmap{};
  u64 max_wi{};
  u64* opc_hist{};       // n_opcodes counts
  u64* over{};
  u64 over_cap{};
  Arena* arena{};
};
void launch_instr_runs(const RunBatchArgs& a, cudaStream_t s);
// Adds the count, sum, sum of squares and maximum of u16 widths to the arena.
void launch_simd_widths(const uint16_t* widths, u64 n, Arena* arena, cudaStream_t s);
// Sets *flag when keys[0..n) are not in non-decreasing order.
void launch_keys_sorted(const u64* keys, u64 n, u32* flag, cudaStream_t s);

struct CombineArgs {
  const u64* a{};
  const u64* b{};
  const u32* cur{};
  u64 n_runs{};
  const u64* run_sum{};
  u64* over{};
  u64 over_cap{};
  Arena* arena{};
};
void launch_instr_combine(const CombineArgs& a, cudaStream_t s);

void launch_wi_count(const u32* bitmap, Arena* arena, cudaStream_t s);
void launch_wi_clear(u32* bitmap, Arena* arena, cudaStream_t s);
void launch_reset_identities(Arena* arena, cudaStream_t s);
// Opcode distribution and work-item count in one launch; the counted bitmap words are cleared.
void launch_tail_counts(const u64* hist, u32 n_opcodes, u32* bitmap, u64* over, u64 over_cap, Arena* arena,
                        cudaStream_t s);
// Arena (with the identities), opcode histogram and sbt_words words of the superblock table to their start.
void launch_reset(Arena* arena, u64* hist, u32 n_opcodes, u64* sbt, u64 sbt_words, cudaStream_t s);

struct FinalizeArgs {
  const u64* over_a{};
  const u64* over_b{};
  const u32* over_cur{};
  u64 over_cap{};
  Arena* arena{};
  Result* result{};
  u32 cover_num{}, cover_den{};
  u32 precision{};
  u32 history_len{};
};
void launch_finalize(const FinalizeArgs& a, cudaStream_t s);
// Partitioned invocations: adds one partition's arena (and overflow entries) to the total's.
void launch_merge_partition(const Arena* part, const u64* part_over, u64 part_cap, Arena* total, u64* total_over,
                            u64 total_cap, cudaStream_t s);
// Sharded invocations: dst[i] += src[i] (opcode histograms), dst[i] |= src[i] (work-item bitmap words).
void launch_add_u64(u64* dst, const u64* src, u64 n, int sm_count, cudaStream_t s);
void launch_or_u32(u32* dst, const u32* src, u64 n, int sm_count, cudaStream_t s);

}  // namespace aiwc
