// Routing of an invocation's events to shards (one per rank), host code.
//
// A rank that holds an arbitrary slice of an invocation's streams routes every
// event to the shard that owns its unit (route.h): memory events by
// superblock, branch events by site, instruction runs by work-item. After the
// ranks exchange the routed slices (an all-to-all), each rank holds whole
// units only, reduces them with the finalisation deferred and exports its
// exact distributions (aiwc_shard_export); adding the ranks' distributions
// (aiwc_shard_merge) gives the invocation's, as Sec. V adds each work-group's
// results into the kernel's global state.
#include <cstring>
#include <string>
#include <vector>

#include "aiwc_internal.cuh"
#include "route.h"

using namespace aiwc;

namespace {

aiwc_status bad(const std::string& msg) {
  set_last_error(msg);
  return AIWC_EINVAL;
}

bool shards_ok(uint32_t n_shards) { return n_shards >= 1 && n_shards <= 256; }

}  // namespace

extern "C" {

aiwc_status aiwc_shard_route_mem(uint32_t n_shards, int byte_addresses, const aiwc_mem_event* ev, size_t n,
                                 aiwc_mem_event* out, size_t out_cap, uint64_t* counts, size_t* n_out) {
  if (!shards_ok(n_shards)) return bad("aiwc_shard_route_mem: n_shards must be 1..256");
  if (!counts || !n_out || (n && !ev)) return bad("aiwc_shard_route_mem: null argument");
  const aiwc_mem_event* e = ev;
  std::vector<aiwc_mem_event> split;
  if (byte_addresses && split_at_superblocks(ev, n, &split)) {
    e = split.data();
    n = split.size();
  }
  *n_out = n;
  std::vector<uint32_t> sid(n);
  for (uint32_t s = 0; s < n_shards; ++s) counts[s] = 0;
  for (size_t i = 0; i < n; ++i) ++counts[sid[i] = shard_of(mem_route_key(e[i]), n_shards)];
  if (!out) return AIWC_OK;  // size query
  if (out_cap < n) return bad("aiwc_shard_route_mem: out holds fewer events than the routed stream");
  std::vector<uint64_t> at(n_shards, 0);
  for (uint32_t s = 1; s < n_shards; ++s) at[s] = at[s - 1] + counts[s - 1];
  for (size_t i = 0; i < n; ++i) out[at[sid[i]]++] = e[i];
  return AIWC_OK;
}

aiwc_status aiwc_shard_route_branch(uint32_t n_shards, const aiwc_branch_event* ev, size_t n, aiwc_branch_event* out,
                                    uint64_t* counts) {
  if (!shards_ok(n_shards)) return bad("aiwc_shard_route_branch: n_shards must be 1..256");
  if (!counts || (n && (!ev || !out))) return bad("aiwc_shard_route_branch: null argument");
  std::vector<uint32_t> sid(n);
  for (uint32_t s = 0; s < n_shards; ++s) counts[s] = 0;
  for (size_t i = 0; i < n; ++i) ++counts[sid[i] = shard_of(ev[i].site, n_shards)];
  std::vector<uint64_t> at(n_shards, 0);
  for (uint32_t s = 1; s < n_shards; ++s) at[s] = at[s - 1] + counts[s - 1];
  for (size_t i = 0; i < n; ++i) out[at[sid[i]]++] = ev[i];
  return AIWC_OK;
}

aiwc_status aiwc_shard_route_runs(uint32_t n_shards, const uint32_t* run_wi, const uint64_t* run_off,
                                  const uint64_t* run_len, size_t n_runs, const uint16_t* ops, size_t n_ops,
                                  uint32_t* out_wi, uint64_t* out_off, uint64_t* out_len, uint16_t* out_ops,
                                  uint64_t* run_counts, uint64_t* op_counts) {
  if (!shards_ok(n_shards)) return bad("aiwc_shard_route_runs: n_shards must be 1..256");
  if (!run_counts || !op_counts) return bad("aiwc_shard_route_runs: null argument");
  if (n_runs && (!run_wi || !run_off || !run_len || !out_wi || !out_off || !out_len))
    return bad("aiwc_shard_route_runs: null argument");
  for (size_t r = 0; r < n_runs; ++r)
    if (run_off[r] > n_ops || run_len[r] > n_ops - run_off[r])
      return bad("aiwc_shard_route_runs: a run reaches past its opcode array");
  std::vector<uint32_t> sid(n_runs);
  for (uint32_t s = 0; s < n_shards; ++s) run_counts[s] = op_counts[s] = 0;
  for (size_t r = 0; r < n_runs; ++r) {
    sid[r] = shard_of(run_wi[r], n_shards);
    ++run_counts[sid[r]];
    op_counts[sid[r]] += run_len[r];
  }
  uint64_t total_ops = 0;
  for (uint32_t s = 0; s < n_shards; ++s) total_ops += op_counts[s];
  if (total_ops && (!ops || !out_ops)) return bad("aiwc_shard_route_runs: null opcode array");
  std::vector<uint64_t> at(n_shards, 0), op_at(n_shards, 0), op_base(n_shards, 0);
  for (uint32_t s = 1; s < n_shards; ++s) {
    at[s] = at[s - 1] + run_counts[s - 1];
    op_base[s] = op_base[s - 1] + op_counts[s - 1];
  }
  for (size_t r = 0; r < n_runs; ++r) {
    const uint32_t s = sid[r];
    const uint64_t k = at[s]++;
    out_wi[k] = run_wi[r];
    out_len[k] = run_len[r];
    out_off[k] = op_at[s];  // relative to the shard's own opcode segment
    if (run_len[r]) memcpy(out_ops + op_base[s] + op_at[s], ops + run_off[r], run_len[r] * 2);
    op_at[s] += run_len[r];
  }
  return AIWC_OK;
}

}  // extern "C"
