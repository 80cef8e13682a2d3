/*
 * aiwc.h -- C ABI of a GB300-native reduction of one OpenCL kernel
 * invocation's event traces to the architecture-independent workload
 * characterization (AIWC) metrics of Johnston & Milthorpe (arXiv 1805.04207).
 *
 * The paper collects events inside an OpenCL simulator through per-
 * instruction callbacks and reduces them when the kernel ends (Sec. V). This
 * library replaces the callbacks with bulk pushes of already-collected event
 * streams and performs the end-of-kernel reduction (Table I) on the GPU.
 *
 * Conventions for every entry point:
 *   - Return value: an aiwc_status. Nothing aborts, traps or exits.
 *   - Pointers flagged `on_device` are CUDA device pointers on the handle's
 *     device; otherwise they are host pointers. Host data is copied (or fully
 *     consumed) before the call returns. Device data must stay valid and
 *     unmodified until the next aiwc_compute on that handle returns, because
 *     work is queued on the handle's CUDA stream.
 *   - All GPU work of a handle is ordered on the stream given in
 *     aiwc_config.cuda_stream: the handle's own streams (copies of host data;
 *     the branch reduction, which runs beside the memory reduction) fork from
 *     it and join it again with events before a call's work there ends. The
 *     library owns all of its device scratch.
 *   - After an error other than AIWC_EINVAL the handle answers AIWC_ESTATE
 *     until aiwc_compute (which then resets it) or aiwc_destroy.
 *     AIWC_EINVAL found inside event data is reported by aiwc_compute, which
 *     still resets the handle for the next invocation.
 *   - A handle is not thread-safe; distinct handles are independent.
 */
#ifndef AIWC_H
#define AIWC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- events */

/* One memory access (Sec. V: memoryLoad / memoryStore / memoryAtomicLoad /
 * memoryAtomicStore notifications). 16 bytes, little-endian.
 *   addr       start address; must be < 2^61 (the 61-bit address domain);
 *              with byte_addresses = 1 the last byte, addr + size - 1, must be.
 *   work_item  id of the issuing work-item.
 *   size       access size in bytes: used only with byte_addresses = 1, where
 *              every byte it covers counts; otherwise carried and unused.
 *   flags      bit 0: 1 = store (write), 0 = load (read);
 *              bits 1-2: OpenCL address space (0 global, 1 local,
 *              2 constant, 3 private); other bits ignored.
 * An atomic read-modify-write is pushed as one load and one store. */
typedef struct aiwc_mem_event {
  uint64_t addr;
  uint32_t work_item;
  uint8_t size;
  uint8_t flags;
  uint16_t reserved;
} aiwc_mem_event;

/* One conditional-branch outcome (Sec. V, Listing 1: the taken / not-taken
 * result recorded per branch location). 8 bytes.
 *   site       id of the static branch (the paper keys branches by source
 *              line; any 32-bit id works).
 *   wi_taken   bits 0-30: work-item id; bit 31: 1 = taken. */
typedef struct aiwc_branch_event {
  uint32_t site;
  uint32_t wi_taken;
} aiwc_branch_event;

/* Barrier marker in the 16-bit opcode stream (Sec. V: a barrier ends the
 * running instructions-to-barrier tally). It is not counted as an
 * instruction. */
#define AIWC_BARRIER 0xFFFFu
#define AIWC_ADDR_LIMIT (1ull << 61)
#define AIWC_MAX_SKIP 10 /* local memory address entropy skips 1..10 bits (Sec. III) */

typedef enum aiwc_status {
  AIWC_OK = 0,
  AIWC_EINVAL = 1,   /* invalid argument or invalid event data */
  AIWC_ENOMEM = 2,   /* device memory or the HBM budget is exhausted */
  AIWC_ECUDA = 3,    /* a CUDA call failed; see aiwc_last_error */
  AIWC_ESTATE = 4,   /* handle unusable after an earlier error */
  AIWC_ETIMEOUT = 5, /* a bounded device-side wait gave up */
  AIWC_EAGAIN = 6    /* serving: not admitted now, retry later */
} aiwc_status;

/* ---------------------------------------------------------------- config */

typedef struct aiwc_config {
  int device;             /* CUDA device ordinal */
  void* cuda_stream;      /* cudaStream_t for all work of the handle; NULL = legacy default stream */
  uint32_t history_len;   /* branch history length, 1..31 (Sec. III fixes 16) */
  uint32_t cover_num;     /* coverage fraction numerator (Table I "90%": 9) */
  uint32_t cover_den;     /* coverage fraction denominator (10) */
  uint32_t n_opcodes;     /* valid opcodes are 0..n_opcodes-1, n_opcodes <= 65535 */
  uint32_t space_mask;    /* bit s set: address space s takes part in the memory metrics (0xF) */
  uint32_t precision;     /* entropy finalisation: 0 = FP64, 1 = FP32 compensated sums (each entropy
                             within 2^-22 bits of FP64; every count identical; the linear branch
                             entropy, one division of exact integers, is FP64 in both modes) */
  uint32_t plan;          /* distinct-address counting: 0 = automatic, per invocation, from its first
                             memory push of n events: n <= 2^15 takes the sort plan, larger ones the
                             hash plan (the sort plan finishes one whose table overflowed);
                             1 = sort (and the radix-sort branch path); 2 = hash */
  uint64_t max_work_items;/* work-item ids must be < this (sizes the work-item bitmap); 0 = 2^32 */
  uint64_t hbm_budget;    /* bytes of device scratch the handle may hold; 0 = unlimited */
  uint64_t table_slots;   /* hash plan: initial superblock-table slots (power of two); 0 = automatic:
                             at least n slots for a first memory push of n events, 2^12 .. 2^20,
                             never shrinking. An invocation that overflows the table is finished by
                             the sort plan and the next one gets a 4x larger table */
  uint32_t partitions;    /* invocations larger than device memory (Sec. VI names the trace size as the
                             tool's limit): 0 or 1 = off; P > 1 (a power of two <= 256) routes pushes on
                             the host into P partitions that keep every unit of the method whole --
                             memory superblocks of 2^11 addresses, branch sites, work-items' runs --
                             and aiwc_compute reduces one partition at a time on the device, adds their
                             exact distributions and finalises once. Device memory then scales with the
                             largest partition; host memory holds the pushed events until compute.
                             Not for aiwc_compute_batch or server jobs. */
  uint32_t byte_addresses;/* address granularity (the paper records each access's address and size
                             but keys its memory metrics by address only): 0 = an access counts once,
                             at its start address; 1 = every byte it touches, addr .. addr + size - 1,
                             counts as one access of the same kind and space (size 0 touches none), so
                             every memory metric counts bytes. A push then learns its byte count on the
                             device before ingesting: one stream synchronisation per 2^26 device events
                             (per 2^22 host events, which are staged in 64 MiB pieces). An
                             access whose last byte is outside the address domain is invalid data. */
  uint32_t history_scope; /* whose branch history (Sec. III, Sec. V): 0 = one history per site, the
                             work-items' outcomes one after another (ids ascending, program order
                             inside each); 1 = one history per (site, work-item), that work-item's
                             outcomes in program order. Patterns stay keyed by (site, history); the
                             first history_len outcomes of every history predict nothing. */
  uint32_t defer_pushes;  /* 1: pushes of DEVICE data (memory events without byte_addresses, branch
                             events, instruction run tables, widths) are recorded and ingested when
                             the invocation is computed -- aiwc_compute_batch then ingests every
                             handle's pushes on parallel streams, so that many small invocations
                             share the GPU. The data must stay unmodified until the compute (the
                             ownership rule of device pointers already asks this). A host push first
                             ingests the recorded ones, so order is kept. Results are identical;
                             push-time data errors surface at the compute. Not with partitions. */
} aiwc_config;

/* Fills the paper's defaults: history 16, 90% coverage, all address spaces,
 * 65535 opcodes, FP64, automatic plan, device 0, default stream. */
void aiwc_config_default(aiwc_config* cfg);

/* --------------------------------------------------------------- metrics */

/* Table I metrics for one invocation (all integers exact).
 * Readings where the paper is silent are stated per field. */
typedef struct aiwc_metrics {
  /* Compute (Table I): */
  uint64_t total_instructions;  /* non-barrier instructions */
  uint64_t unique_opcodes;      /* opcodes executed at least once */
  uint64_t opcode_cover;        /* "Opcode": fewest opcodes covering cover_num/cover_den of instructions */
  /* Parallelism (Table I): */
  uint64_t work_items;          /* distinct work-item ids over all three streams */
  uint64_t barriers;            /* barrier markers */
  uint64_t itb_count, itb_min, itb_max, itb_median_lo, itb_median_hi;
  double itb_median;            /* instructions to barrier; each work-item's final tally counts (implicit barrier) */
  uint64_t ipt_count, ipt_min, ipt_max, ipt_median_lo, ipt_median_hi;
  double ipt_median;            /* instructions per thread, over work-items of the instruction stream */
  /* Memory (Table I): */
  uint64_t total_reads, total_writes;
  uint64_t footprint;           /* unique (address space, address) pairs */
  uint64_t footprint_cover;     /* "90% Memory Footprint" */
  uint64_t unique_reads, unique_writes;
  double entropy[AIWC_MAX_SKIP + 1]; /* [0] global memory address entropy; [n] local entropy with n low bits skipped */
  /* Control (Table I): */
  uint64_t branch_events;
  uint64_t branch_sites;        /* "Total Unique Branch Instructions" */
  uint64_t branch_cover;        /* "90% Branch Instructions" */
  uint64_t branch_patterns;     /* N': outcomes that have a full history */
  uint64_t branch_minsum;       /* M = sum over history patterns of min(taken, not taken) */
  double albe;                  /* average linear branch entropy = 2 M / N' */
  double yokota;                /* Yokota branch entropy. Reading (the paper gives no normalisation): the entropy
                                 * of the h-outcome history given the site, over the N' predicted outcomes,
                                 * divided by h -- in [0, 1] */
  /* Ratios as printed in Table I (IEEE division: x/0 gives inf or NaN). */
  double unique_rw_ratio;       /* unique reads / unique writes */
  double reread_ratio;          /* unique reads / total reads */
  double rewrite_ratio;         /* unique writes / total writes */
  /* Parallelism, SIMD (Table I; Sec. III, Sec. V): over the result widths of
   * executed instructions pushed with aiwc_push_widths. Sums are exact below
   * 2^64 (at most 2^32 widths of at most 65535 each). */
  uint64_t simd_count;          /* widths pushed */
  uint64_t simd_max;            /* "Max SIMD Width" */
  uint64_t simd_sum;            /* sum of widths */
  uint64_t simd_sumsq;          /* sum of squared widths */
  double simd_mean;             /* "Mean SIMD Width" = simd_sum / simd_count */
  double simd_sd;               /* "SD SIMD Width": population standard deviation (divides by simd_count) */
  /* Derived parallelism quantities of the Kiviat diagrams (Sec. VI), IEEE division: */
  double granularity;               /* 1 / work_items */
  double barriers_per_instruction;  /* 1 / mean ITB = itb_count / total_instructions */
  double instructions_per_operand;  /* 1 / simd_sum */
  double load_imbalance;            /* ipt_max - ipt_min */
  /* In: optional caller buffer of n_opcodes counts (NULL to skip). */
  uint64_t* opcode_hist;
} aiwc_metrics;

/* ------------------------------------------------------- single invocation */

typedef struct aiwc_handle aiwc_handle;

/* kernelBegin (Sec. V): creates the state of one invocation at a time.
 * Errors: AIWC_EINVAL (cfg NULL or out of range), AIWC_ECUDA, AIWC_ENOMEM. */
aiwc_status aiwc_create(const aiwc_config* cfg, aiwc_handle** out);

/* Memory notifications (Sec. V) in bulk: n events, in any order (the memory
 * metrics do not depend on event order). Device events must be 16-byte
 * aligned. Invalid addresses are reported by aiwc_compute as AIWC_EINVAL.
 * Errors: AIWC_EINVAL (ev NULL with n > 0, misaligned device events),
 * AIWC_ENOMEM, AIWC_ECUDA, AIWC_ESTATE. */
aiwc_status aiwc_push_mem(aiwc_handle* h, const aiwc_mem_event* ev, size_t n, int on_device);

/* Branch outcomes (Sec. III, Sec. V) in bulk. Each site's history is ordered
 * by (work-item id, push order): events of one work-item must be pushed in
 * program order; different work-items may interleave freely. Device events
 * must be 8-byte aligned.
 * Errors: AIWC_EINVAL (ev NULL with n > 0, misaligned device events),
 * AIWC_ENOMEM, AIWC_ECUDA, AIWC_ESTATE. */
aiwc_status aiwc_push_branch(aiwc_handle* h, const aiwc_branch_event* ev, size_t n, int on_device);

/* Instruction stream of one work-item (Sec. V: instructionExecuted), n
 * opcodes in program order with AIWC_BARRIER markers. Successive pushes for
 * the same work-item continue its stream; n = 0 still makes the work-item one
 * of the instruction stream's (its final tally, 0, counts). Device opcodes
 * must be 2-byte aligned. Invalid opcodes are reported by aiwc_compute.
 * Errors: AIWC_EINVAL (ops NULL with n > 0, misaligned device opcodes),
 * AIWC_ENOMEM, AIWC_ECUDA, AIWC_ESTATE. */
aiwc_status aiwc_push_instr(aiwc_handle* h, uint32_t work_item, const uint16_t* ops, size_t n, int on_device);

/* Bulk form of aiwc_push_instr: n_runs runs, run r covering
 * ops[run_off[r] .. run_off[r] + run_len[r]) for work-item run_wi[r], in
 * push order. All five arrays are on the same side (on_device), device
 * arrays aligned to their element size. A run reaching past n_ops is
 * invalid: this call refuses it in a host table, aiwc_compute reports it
 * from a device table.
 * Errors: AIWC_EINVAL (a NULL table with n_runs > 0, ops NULL with n_ops > 0,
 * misaligned device arrays, a host run past n_ops, more than 2^32 - 1 runs in
 * one invocation), AIWC_ENOMEM, AIWC_ECUDA, AIWC_ESTATE. */
aiwc_status aiwc_push_instr_runs(aiwc_handle* h, const uint32_t* run_wi, const uint64_t* run_off,
                                 const uint64_t* run_len, size_t n_runs, const uint16_t* ops,
                                 size_t n_ops, int on_device);

/* The result width (number of data items) of executed instructions (Sec. V:
 * the width of each instruction's result is recorded for the SIMD metrics of
 * Table I), one u16 per counted instruction, in any order; barrier markers
 * have no width. `widths` is host or device memory (on_device = 1), owned by
 * the caller, and device memory must stay valid until the next compute.
 * Errors: AIWC_EINVAL (null pointer with n > 0), AIWC_ECUDA, AIWC_ESTATE. */
aiwc_status aiwc_push_widths(aiwc_handle* h, const uint16_t* widths, size_t n, int on_device);

/* kernelEnd (Sec. V): reduces everything pushed since the last compute to the
 * Table I metrics, writes them to *out (and out->opcode_hist when non-NULL),
 * then resets the handle for the next invocation. Blocks until done.
 * Errors: AIWC_EINVAL (invalid event data: an address >= 2^61 or an opcode
 * >= n_opcodes that is not AIWC_BARRIER, a run past its opcode array, a
 * work-item >= max_work_items), AIWC_ECUDA, AIWC_ESTATE, AIWC_ETIMEOUT (a radix
 * sort pass gave up its bounded wait for an earlier tile's digit counts; valid
 * launches always finish those waits). */
aiwc_status aiwc_compute(aiwc_handle* h, aiwc_metrics* out);

/* Several invocations at once: outs[i] receives the metrics of hs[i], exactly
 * as aiwc_compute(hs[i]) would. After one synchronisation that reads every
 * handle's ingest-time counters, the remaining stages of all handles are
 * captured as one CUDA graph -- each handle a branch on one of 16 forked
 * streams, so small invocations run side by side -- and the graph is
 * replayed while the batch keeps the same handles, sizes and plans. Choices
 * that depend on device results (the branch-history path) are taken on the
 * device inside the graph. All handles must share one device and stream;
 * a handle may appear once. Returns the first non-OK status (each outs[i]
 * is still written for handles that succeeded). */
aiwc_status aiwc_compute_batch(aiwc_handle* const* hs, size_t n, aiwc_metrics* outs);

aiwc_status aiwc_destroy(aiwc_handle* h);

/* Whole-application view over several invocations of one kernel (Sec. VI):
 * AIWC_AGG_SUM adds every numeric field over runs[0..n) (the paper presents
 * "the summation of all metrics for a kernel"), AIWC_AGG_MEDIAN takes each
 * field's median over the runs (the figures show medians across iterations):
 * for floating-point fields the mean of the two middle values when n is
 * even, for integer fields the lower middle value. out->opcode_hist is left
 * as the caller set it. Host-only arithmetic: needs no device and no handle.
 * Errors: AIWC_EINVAL (null pointers with n > 0, unknown mode). */
#define AIWC_AGG_SUM 0
#define AIWC_AGG_MEDIAN 1
aiwc_status aiwc_aggregate(const aiwc_metrics* runs, size_t n, int mode, aiwc_metrics* out);

/* ------------------------------------------------------- sharded invocations
 *
 * One invocation reduced by several ranks (one process per GPU). Sec. V adds
 * each work-group's results into the kernel's global state; every metric is a
 * function of distributions that add exactly over any split of the events
 * into whole units -- memory superblocks of 2^11 addresses (with their space),
 * branch sites, work-items' instruction runs -- so ranks that each reduce
 * whole units and add their exact distributions reproduce the single-device
 * result bit for bit. The protocol, for N ranks that each hold any slice of
 * the invocation's streams (in push order, rank r's slice before rank r+1's):
 *   1. route: each rank splits its slice into N shards with the calls below;
 *   2. exchange (all-to-all): rank s receives shard s of every rank;
 *   3. push the received slices in source-rank order, then aiwc_shard_export;
 *   4. gather the N blobs (in rank order) on one or every rank and call
 *      aiwc_shard_merge, which finalises once.
 * Routing is host code (no device, no handle); the collective is the
 * caller's (NCCL on device buffers, gloo on host buffers). */

/* Stable split of host memory events into n_shards (1..256) shards by
 * superblock. With byte_addresses, an access whose bytes cross a superblock
 * boundary becomes two accesses, one on each side (as aiwc_config.
 * byte_addresses reads the stream), so *n_out may exceed n. out == NULL:
 * size query (*n_out and counts only). Else out (host, out_cap events)
 * receives shard 0's events, then shard 1's, ..., counts[s] of them each.
 * Errors: AIWC_EINVAL (bad n_shards, null pointers, out_cap < *n_out). */
aiwc_status aiwc_shard_route_mem(uint32_t n_shards, int byte_addresses, const aiwc_mem_event* ev, size_t n,
                                 aiwc_mem_event* out, size_t out_cap, uint64_t* counts, size_t* n_out);

/* Stable split of host branch events by site into out (n events, shard 0's
 * first) with counts[s] per shard. Errors: AIWC_EINVAL. */
aiwc_status aiwc_shard_route_branch(uint32_t n_shards, const aiwc_branch_event* ev, size_t n, aiwc_branch_event* out,
                                    uint64_t* counts);

/* Stable split of host instruction runs (as aiwc_push_instr_runs) by
 * work-item: out_wi / out_off / out_len receive shard 0's runs, then shard
 * 1's, ... (run_counts[s] each); out_ops receives each shard's opcodes as one
 * segment (op_counts[s] opcodes; the segments follow each other) and out_off
 * is relative to the start of the run's own shard segment, so that a shard's
 * run table and segment can be sent and pushed as they are. out_ops holds
 * the sum of run_len. Errors: AIWC_EINVAL (null pointers, a run past n_ops). */
aiwc_status aiwc_shard_route_runs(uint32_t n_shards, const uint32_t* run_wi, const uint64_t* run_off,
                                  const uint64_t* run_len, size_t n_runs, const uint16_t* ops, size_t n_ops,
                                  uint32_t* out_wi, uint64_t* out_off, uint64_t* out_len, uint16_t* out_ops,
                                  uint64_t* run_counts, uint64_t* op_counts);

/* Ends this rank's part of a sharded invocation: reduces what was pushed with
 * the finalisation deferred and writes the exact distributions (dense
 * count-of-counts and value bins, counters, overflow entries, opcode
 * histogram, the rank's work-item bitmap words) as a host blob. The first call
 * after the pushes reduces, keeps the blob on the host and resets the handle
 * for its next invocation; *size is then the blob's size. blob == NULL: only
 * *size (the blob stays held). blob with cap >= *size: the blob is copied
 * there and released. The blob is valid for aiwc_shard_merge of the same
 * library build and metric configuration. Invalid event data is carried in
 * the blob and reported by the merge. Errors: AIWC_EINVAL (null pointers, cap
 * too small, a partitioned handle), AIWC_ENOMEM, AIWC_ECUDA, AIWC_ESTATE. */
aiwc_status aiwc_shard_export(aiwc_handle* h, void* blob, size_t cap, size_t* size);

/* Adds n ranks' blobs (host pointers, sizes from aiwc_shard_export) into the
 * handle's device state and finalises the invocation once: *out is the
 * metric set of the whole sharded invocation (out->opcode_hist as for
 * aiwc_compute). h must hold no pushed events and share the blobs' metric
 * configuration (history length, opcodes, space mask, byte addresses,
 * history scope, max_work_items); precision and coverage fraction are h's.
 * Errors: AIWC_EINVAL (a blob of another build or configuration, inconsistent
 * sizes, invalid event data), AIWC_ESTATE (pushed events pending),
 * AIWC_ENOMEM, AIWC_ECUDA. */
aiwc_status aiwc_shard_merge(aiwc_handle* h, const void* const* blobs, const size_t* sizes, size_t n,
                             aiwc_metrics* out);

/* Text of the last error on h (or of the last global error when h is NULL). */
const char* aiwc_last_error(const aiwc_handle* h);

/* Device bytes currently held by h. */
uint64_t aiwc_device_bytes(const aiwc_handle* h);

/* ----------------------------------------------------------- diagnostics */

/* Number of CUDA kernels this library has launched in this process (all
 * handles). The paper has no counterpart; it exists so that callers can
 * check which work ran on the GPU. */
uint64_t aiwc_kernel_launches(void);

/* Stage timing: when on, every push and aiwc_compute brackets its stages with
 * CUDA events on the stream each stage runs on (no extra synchronisation);
 * after aiwc_compute returns, aiwc_stage_times reports the elapsed
 * milliseconds of each stage of that invocation, summed over pushes. Stages
 * that run at the same time on two streams each include the other's share of
 * the GPU. Stages, in order:
 *   0 mem_ingest    1 branch_ingest  2 instr_runs    3 mem_sort
 *   4 mem_scatter   5 mem_levels     6 branch_sort   7 windows
 *   8 pattern_sort  9 pattern_runs  10 run_sort     11 run_combine
 *  12 finalize     13 mem_expand
 * Returns the number of stages written (at most n); names may be NULL.
 * Whether timing is on or off, each stage is also an NVTX range with the
 * stage's name, for profilers that record NVTX (nsys; ncu --nvtx). */
aiwc_status aiwc_set_stage_timing(aiwc_handle* h, int on);
int aiwc_stage_times(const aiwc_handle* h, double* ms, const char** names, int n);

/* --------------------------------------------------------------- serving */

/* Many characterization jobs at once, each streaming its trace in chunks
 * (the low-memory streaming the paper leaves to future work, Sec. VII, and
 * the failures on large traces it reports, Sec. VI). A server owns
 * `max_jobs` slots; each slot is a handle with its own CUDA stream, so the
 * chunks of one job are ingested while other jobs are reduced. A job is
 * admitted only when a slot is free and its reservation fits `hbm_budget`
 * next to what running jobs reserve (device memory of idle slots is released
 * first); otherwise aiwc_job_open returns AIWC_EAGAIN and the caller retries.
 * A job's results equal those of aiwc_compute on the same events. */
typedef struct aiwc_server_config {
  int device;
  uint32_t max_jobs;     /* slots: jobs in flight at once (1..4096) */
  uint32_t workers;      /* host threads running reductions (1..64) */
  uint64_t hbm_budget;   /* bytes of device scratch all jobs together may hold */
} aiwc_server_config;

typedef struct aiwc_server aiwc_server;
typedef struct aiwc_job aiwc_job;

/* Defaults: device 0, 32 slots, 4 workers, 120 GiB. */
void aiwc_server_config_default(aiwc_server_config* cfg);
aiwc_status aiwc_server_create(const aiwc_server_config* cfg, aiwc_server** out);

/* Opens a job with the metric configuration job_cfg (its device, stream and
 * hbm_budget are replaced by the slot's) and a scratch reservation of
 * reserve_bytes, which bounds what the job may allocate (pushes beyond it fail
 * with AIWC_ENOMEM; the work-item bitmap is max_work_items / 8 bytes of it).
 * AIWC_EAGAIN: no slot or not enough budget now. AIWC_ENOMEM: the
 * reservation exceeds the whole budget. */
aiwc_status aiwc_job_open(aiwc_server* s, const aiwc_config* job_cfg, uint64_t reserve_bytes, aiwc_job** out);

/* Chunk pushes, with the semantics of aiwc_push_mem / _branch / _instr_runs.
 * A job is used by one thread at a time. */
aiwc_status aiwc_job_push_mem(aiwc_job* j, const aiwc_mem_event* ev, size_t n, int on_device);
aiwc_status aiwc_job_push_branch(aiwc_job* j, const aiwc_branch_event* ev, size_t n, int on_device);
aiwc_status aiwc_job_push_widths(aiwc_job* j, const uint16_t* widths, size_t n, int on_device);
aiwc_status aiwc_job_push_instr_runs(aiwc_job* j, const uint32_t* run_wi, const uint64_t* run_off,
                                     const uint64_t* run_len, size_t n_runs, const uint16_t* ops, size_t n_ops,
                                     int on_device);

/* Queues the job's reduction on a worker and returns at once. */
aiwc_status aiwc_job_finish(aiwc_job* j);

/* When the reduction is done: writes the metrics (and out->opcode_hist when
 * non-NULL), releases the slot, frees j and returns the reduction's status;
 * otherwise AIWC_EAGAIN and j stays valid. aiwc_job_wait blocks instead (and
 * finishes the job first if needed). */
aiwc_status aiwc_job_poll(aiwc_job* j, aiwc_metrics* out);
aiwc_status aiwc_job_wait(aiwc_job* j, aiwc_metrics* out);

/* Counters since creation, and the device bytes slots hold now. */
aiwc_status aiwc_server_stats(const aiwc_server* s, uint64_t* admitted, uint64_t* rejected, uint64_t* completed,
                              uint64_t* device_bytes);

/* Waits for queued reductions, then frees everything, jobs not yet collected
 * included (their pointers become invalid). */
aiwc_status aiwc_server_destroy(aiwc_server* s);

/* ------------------------------------------------- without any allocation */

/* The memory metrics (Table I memory rows: totals, unique reads and writes,
 * footprint, 90% footprint, global and local address entropies) and the
 * work-item count of one invocation's memory events, computed without any
 * device allocation. The paper has no counterpart: this entry point exists
 * for callers that may not call cudaMalloc or cudaFree -- code whose device
 * memory belongs to another allocator (a framework's caching allocator or a
 * fixed pool it must stay inside) and code that must not trigger the
 * device-wide synchronisation that freeing device memory implies.
 *
 *   device       CUDA device ordinal; events must live on it.
 *   cuda_stream  cudaStream_t the work is ordered on (NULL = default stream).
 *   events       DEVICE pointer to n aiwc_mem_event records, 16-byte aligned,
 *                owned by the caller and only read; device memory of another
 *                device or pageable host memory -> AIWC_EINVAL.
 *   n            at most 262144 (2^18) events; larger n -> AIWC_EINVAL.
 *   space_mask   as aiwc_config.space_mask.
 *   out          HOST pointer; the memory fields and work_items are written,
 *                every other field is zero (out->opcode_hist is left as is);
 *                on any status but AIWC_OK every field is zero.
 * Work-item ids must be below 2^20. Blocks until the result is on the host.
 *
 * Scratch: one file-scope device array of about 24 MiB inside the library
 * (every device that loads the library holds it until the process exits),
 * shared by all calls on a device and keeping the last call's contents, which
 * each call clears where it must start at zero. Calls whose GPU work overlaps
 * (concurrent streams, or threads) race on that array and give wrong results:
 * serialise them. The first call on a device looks the array's address up
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture. No cudaMalloc, cudaFree or allocating library
 * routine is called. Errors: AIWC_EINVAL (bad arguments or event data),
 * AIWC_ENOMEM (the fixed scratch overflowed), AIWC_ECUDA. */
aiwc_status aiwc_mem_metrics_noalloc(int device, void* cuda_stream, const aiwc_mem_event* events, size_t n,
                                     uint32_t space_mask, aiwc_metrics* out);

#ifdef __cplusplus
}
#endif
#endif /* AIWC_H */
