// AIWC metric oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, obviously correct CPU restatement of the architecture-
// independent workload metrics of Johnston & Milthorpe, "AIWC: OpenCL-based
// Architecture-Independent Workload Characterization" (arXiv 1805.04207),
// Table I and Sec. III, for one kernel invocation. Only the test suite, the
// smoke check and the benchmark's CPU-baseline leg use it; the product
// library never links, loads or calls it, and it shares no code, header or
// constant table with the CUDA path.
//
// Every step is the plain definition: collect, std::sort, walk. Where the
// paper is silent the reading used is stated beside the step (the same
// readings the design notes list).
//
// Parity status of each function (what pins it; see tests/test_oracle_pins.py):
//   memory metrics   -- brute force, closed forms, invariants
//   branch metrics   -- brute force, closed forms (constant, alternating,
//                       period-32 loop), invariants
//   instruction/ITB  -- brute force, closed forms, invariants
//   work-items       -- brute force
//   SIMD widths      -- closed forms (constant widths, two-value mix), brute force
//   Yokota entropy   -- closed forms (constant branch 0, de Bruijn sequence 1), brute force;
//                       parity unpinned for the normalisation, which is a reading
//   byte addresses   -- equal to the start-address metrics of the events split into
//                       one-byte accesses; closed forms (arrays read once); brute force
//   per-work-item    -- equal to the per-site metrics when every site has one work-item;
//     histories         closed forms (short per-work-item sequences predict nothing,
//                       interleaved loops); brute force
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <utility>
#include <vector>

namespace {

// Input layouts (little-endian bytes).
//   memory event, 16 B: u64 addr | u32 work_item | u8 size | u8 flags | u16 rsvd
//     flags bit 0 = store, bits 1-2 = address space.
//   branch event, 8 B: u32 site | u32 (work_item | taken << 31)
//   instruction opcodes: u16, 0xFFFF = barrier marker.
constexpr uint16_t kBarrier = 0xFFFFu;
constexpr uint64_t kAddrLimit = 1ull << 61;  // 61-bit address domain

struct OracleConfig {
  uint32_t history_len;  // branch history length (16 in Sec. III)
  uint32_t cover_num;    // coverage fraction numerator   (90%: 9)
  uint32_t cover_den;    // coverage fraction denominator (90%: 10)
  uint32_t n_opcodes;    // valid opcodes are 0..n_opcodes-1
  uint32_t space_mask;   // bit s set: address space s takes part in memory metrics
  uint32_t byte_addresses;  // 0: an access is its start address; 1: every byte it touches
  uint32_t history_scope;   // 0: one history per site; 1: one per (site, work-item)
};

struct OracleMetrics {
  uint64_t total_instructions, unique_opcodes, opcode_cover;
  uint64_t work_items, barriers;
  uint64_t itb_count, itb_min, itb_max, itb_median_lo, itb_median_hi;
  double itb_median;
  uint64_t ipt_count, ipt_min, ipt_max, ipt_median_lo, ipt_median_hi;
  double ipt_median;
  uint64_t total_reads, total_writes, footprint, footprint_cover, unique_reads, unique_writes;
  double entropy[11];
  uint64_t branch_events, branch_sites, branch_cover, branch_patterns, branch_minsum;
  double albe;
  double yokota;
  double unique_rw_ratio, reread_ratio, rewrite_ratio;
};

// Neumaier's compensated sum (a textbook summation, no reordering).
struct CompensatedSum {
  double s = 0.0, c = 0.0;
  void add(double x) {
    double t = s + x;
    if (std::fabs(s) >= std::fabs(x)) c += (s - t) + x; else c += (x - t) + s;
    s = t;
  }
  double value() const { return s + c; }
};

// Table I "Opcode", "90% Memory Footprint", "90% Branch Instructions": the
// fewest items whose counts cover num/den of all occurrences. Reading: the
// smallest k with den * (sum of the k largest counts) >= num * total; 0 when
// there is nothing to cover.
uint64_t cover_count(std::vector<uint64_t> counts, uint32_t num, uint32_t den) {
  unsigned __int128 total = 0;
  for (uint64_t c : counts) total += c;
  if (total == 0) return 0;
  std::sort(counts.begin(), counts.end(), std::greater<uint64_t>());
  unsigned __int128 cum = 0;
  for (size_t k = 0; k < counts.size(); ++k) {
    cum += counts[k];
    if ((unsigned __int128)den * cum >= (unsigned __int128)num * total) return k + 1;
  }
  return counts.size();
}

// Min / max / median of a multiset (Table I ITB and IPT rows). Reading: the
// median of an even-sized set is the mean of the two middle values.
void order_stats(std::vector<uint64_t> v, uint64_t* cnt, uint64_t* mn, uint64_t* mx,
                 uint64_t* lo, uint64_t* hi, double* med) {
  *cnt = v.size();
  if (v.empty()) { *mn = *mx = *lo = *hi = 0; *med = 0.0; return; }
  std::sort(v.begin(), v.end());
  *mn = v.front();
  *mx = v.back();
  *lo = v[(v.size() - 1) / 2];
  *hi = v[v.size() / 2];
  *med = 0.5 * ((double)*lo + (double)*hi);
}

// Shannon entropy (base 2) of the empirical distribution given by counts of
// groups that sum to n: H = -sum_g p_g log2 p_g with p_g = c_g / n.
double shannon_bits(const std::vector<uint64_t>& group_counts, uint64_t n) {
  if (n == 0) return 0.0;
  CompensatedSum acc;
  for (uint64_t c : group_counts) {
    double p = (double)c / (double)n;
    acc.add(-p * std::log2(p));
  }
  return acc.value();
}

}  // namespace

extern "C" {

// Returns 0 on success, 1 when an input is invalid (an address outside the
// 61-bit domain, an opcode that is neither < n_opcodes nor the barrier
// marker, a history length outside 1..31, a coverage fraction outside
// (0, 1], a run that reaches past the opcode array, or -- with byte
// addresses -- an access whose last byte lies outside the domain).
int aiwc_oracle_compute(const uint8_t* mem, uint64_t n_mem,
                        const uint8_t* br, uint64_t n_br,
                        const uint16_t* ops, uint64_t n_ops,
                        const uint32_t* run_wi, const uint64_t* run_off, const uint64_t* run_len,
                        uint64_t n_runs,
                        const OracleConfig* cfg, OracleMetrics* out, uint64_t* opcode_hist) {
  std::memset(out, 0, sizeof(*out));
  if (cfg->history_len < 1 || cfg->history_len > 31) return 1;
  if (cfg->byte_addresses > 1 || cfg->history_scope > 1) return 1;
  if (cfg->cover_den == 0 || cfg->cover_num == 0 || cfg->cover_num > cfg->cover_den) return 1;
  std::set<uint32_t> work_items;  // Table I "Work-items": every id seen in any stream

  // ---------------- memory (Table I memory rows; Sec. III, Sec. V) ----------
  // Each access is keyed by (address space, start address): the space tag
  // keeps equal numbers in different OpenCL address spaces apart. Reads and
  // writes are kept apart for the unique/total counts and combined for the
  // footprints and entropies ("stored separately and later combined", Sec. III).
  // Address granularity (the paper records the address of each access and
  // its size): by default an access counts once, at its start address. With
  // byte_addresses every byte an access touches, addr .. addr + size - 1,
  // counts as one access of its own, with the access's kind and space; an
  // access of size 0 touches no byte (its work-item still counts).
  std::vector<uint64_t> all_keys, read_keys, write_keys;
  for (uint64_t i = 0; i < n_mem; ++i) {
    const uint8_t* e = mem + 16 * i;
    uint64_t addr;
    uint32_t wi;
    std::memcpy(&addr, e, 8);
    std::memcpy(&wi, e + 8, 4);
    uint8_t size = e[12];
    uint8_t flags = e[13];
    work_items.insert(wi);
    if (addr >= kAddrLimit) return 1;
    if (cfg->byte_addresses && size > 0 && addr + size - 1 >= kAddrLimit) return 1;
    uint32_t space = (flags >> 1) & 3u;
    if (!((cfg->space_mask >> space) & 1u)) continue;
    const uint64_t touched = cfg->byte_addresses ? size : 1;
    for (uint64_t b = 0; b < touched; ++b) {
      uint64_t key = ((uint64_t)space << 61) | (addr + b);
      all_keys.push_back(key);
      if (flags & 1u) write_keys.push_back(key); else read_keys.push_back(key);
    }
  }
  out->total_reads = read_keys.size();
  out->total_writes = write_keys.size();
  std::sort(all_keys.begin(), all_keys.end());
  std::sort(read_keys.begin(), read_keys.end());
  std::sort(write_keys.begin(), write_keys.end());
  out->unique_reads = std::unique(read_keys.begin(), read_keys.end()) - read_keys.begin();
  out->unique_writes = std::unique(write_keys.begin(), write_keys.end()) - write_keys.begin();
  const uint64_t n_acc = all_keys.size();
  // Local memory address entropy skips n = 1..10 low address bits (Sec. III);
  // n = 0 is the global memory address entropy. Groups are equal key >> n.
  for (int n = 0; n <= 10; ++n) {
    std::vector<uint64_t> groups;
    for (uint64_t i = 0; i < n_acc;) {
      uint64_t g = all_keys[i] >> n;
      uint64_t j = i;
      while (j < n_acc && (all_keys[j] >> n) == g) ++j;
      groups.push_back(j - i);
      i = j;
    }
    if (n == 0) {
      out->footprint = groups.size();  // "Total Memory Footprint"
      out->footprint_cover = cover_count(groups, cfg->cover_num, cfg->cover_den);
    }
    out->entropy[n] = shannon_bits(groups, n_acc);
  }

  // ---------------- branches (Table I control rows; Sec. III, Sec. V) ------
  // Each site's outcomes form one history, ordered as the simulator would
  // produce them: work-items one after another, program order within each.
  std::map<uint32_t, std::vector<std::pair<uint32_t, uint8_t>>> per_site;  // (wi, taken) in push order
  for (uint64_t i = 0; i < n_br; ++i) {
    uint32_t site, wt;
    std::memcpy(&site, br + 8 * i, 4);
    std::memcpy(&wt, br + 8 * i + 4, 4);
    uint32_t wi = wt & 0x7FFFFFFFu;
    work_items.insert(wi);
    per_site[site].push_back({wi, (uint8_t)(wt >> 31)});
  }
  out->branch_events = n_br;
  std::vector<uint64_t> site_counts;
  const uint32_t h = cfg->history_len;
  std::map<std::pair<uint32_t, uint64_t>, std::pair<uint64_t, uint64_t>> patterns;  // -> (taken, total)
  // Outcome j of a history is predicted from the h outcomes before it in the
  // same history (oldest in the high bit); the first h outcomes of a history
  // have no full history and are skipped. Patterns are keyed by (site,
  // history) in both scopes.
  auto predict = [&](uint32_t site, const std::vector<uint8_t>& seq) {
    for (size_t j = h; j < seq.size(); ++j) {
      uint64_t hist = 0;
      for (size_t k = j - h; k < j; ++k) hist = (hist << 1) | seq[k];
      auto& tn = patterns[{site, hist}];
      tn.first += seq[j];
      tn.second += 1;
    }
  };
  for (auto& kv : per_site) {
    auto& seq = kv.second;
    site_counts.push_back(seq.size());
    std::stable_sort(seq.begin(), seq.end(),
                     [](const std::pair<uint32_t, uint8_t>& a, const std::pair<uint32_t, uint8_t>& b) {
                       return a.first < b.first;
                     });
    if (cfg->history_scope == 0) {
      // one history per site: its work-items' outcomes one after another
      std::vector<uint8_t> outcomes;
      for (auto& e : seq) outcomes.push_back(e.second);
      predict(kv.first, outcomes);
    } else {
      // one history per (site, work-item): that work-item's outcomes at the
      // site in program order (a per-thread history register)
      std::map<uint32_t, std::vector<uint8_t>> per_wi;
      for (auto& e : seq) per_wi[e.first].push_back(e.second);
      for (auto& w : per_wi) predict(kv.first, w.second);
    }
  }
  out->branch_sites = site_counts.size();
  out->branch_cover = cover_count(site_counts, cfg->cover_num, cfg->cover_den);
  // Average linear branch entropy (De Pestel et al., cited in Sec. II):
  // E(p) = 2 min(p, 1 - p) per history pattern, averaged with weights equal
  // to the pattern's share of all predicted outcomes.
  uint64_t minsum = 0, npat = 0;
  for (auto& kv : patterns) {
    uint64_t t = kv.second.first, n = kv.second.second;
    minsum += std::min(t, n - t);
    npat += n;
  }
  out->branch_minsum = minsum;
  out->branch_patterns = npat;
  out->albe = npat ? 2.0 * (double)minsum / (double)npat : 0.0;
  // Yokota branch (history) entropy (Table I; Yokota et al., cited in Sec. II),
  // whose normalisation the paper does not print. Reading: the Shannon
  // entropy of the h-outcome history given the site, over the predicted
  // outcomes, divided by h so that it lies in [0, 1]:
  //   H(history | site) = H(site, history) - H(site)
  //                     = (1/N') [ sum_s N'_s log2 N'_s - sum_P n_P log2 n_P ],
  // with N'_s the predicted outcomes of site s and n_P those of pattern P.
  {
    std::map<uint32_t, uint64_t> per_site_pred;
    CompensatedSum pat_sum, site_sum;
    for (auto& kv : patterns) {
      const double n = (double)kv.second.second;
      pat_sum.add(n * std::log2(n));
      per_site_pred[kv.first.first] += kv.second.second;
    }
    for (auto& kv : per_site_pred) {
      const double n = (double)kv.second;
      site_sum.add(n * std::log2(n));
    }
    double y = npat ? (site_sum.value() - pat_sum.value()) / ((double)npat * (double)h) : 0.0;
    out->yokota = y < 0.0 ? 0.0 : y;
  }

  // ---------------- instructions (Table I compute/parallelism; Sec. III) ---
  // Runs arrive in push order; a work-item's runs continue one another. A
  // barrier marker ends the running ITB tally (it is not itself counted as an
  // instruction); every work-item's last tally is recorded at kernel end
  // (the final implicit barrier), even when it is zero.
  std::vector<uint64_t> hist(cfg->n_opcodes, 0);
  std::map<uint32_t, std::pair<uint64_t, uint64_t>> wi_state;  // wi -> (open tally, instructions)
  std::vector<uint64_t> itb;
  uint64_t barriers = 0;
  for (uint64_t r = 0; r < n_runs; ++r) {
    if (run_off[r] > n_ops || run_len[r] > n_ops - run_off[r]) return 1;
    auto& st = wi_state[run_wi[r]];
    work_items.insert(run_wi[r]);
    for (uint64_t k = 0; k < run_len[r]; ++k) {
      uint16_t op = ops[run_off[r] + k];
      if (op == kBarrier) {
        itb.push_back(st.first);
        st.first = 0;
        ++barriers;
      } else {
        if (op >= cfg->n_opcodes) return 1;
        ++hist[op];
        ++st.first;
        ++st.second;
      }
    }
  }
  std::vector<uint64_t> ipt;
  for (auto& kv : wi_state) {
    itb.push_back(kv.second.first);
    ipt.push_back(kv.second.second);
  }
  uint64_t total = 0, unique_ops = 0;
  std::vector<uint64_t> nonzero;
  for (uint32_t o = 0; o < cfg->n_opcodes; ++o) {
    total += hist[o];
    if (hist[o]) { ++unique_ops; nonzero.push_back(hist[o]); }
    if (opcode_hist) opcode_hist[o] = hist[o];
  }
  out->total_instructions = total;
  out->unique_opcodes = unique_ops;
  out->opcode_cover = cover_count(nonzero, cfg->cover_num, cfg->cover_den);
  out->barriers = barriers;
  order_stats(itb, &out->itb_count, &out->itb_min, &out->itb_max, &out->itb_median_lo,
              &out->itb_median_hi, &out->itb_median);
  order_stats(ipt, &out->ipt_count, &out->ipt_min, &out->ipt_max, &out->ipt_median_lo,
              &out->ipt_median_hi, &out->ipt_median);
  out->work_items = work_items.size();

  // Table I ratios, as printed: unique reads / unique writes, unique reads /
  // total reads, unique writes / total writes (IEEE division: x/0 is inf or NaN).
  out->unique_rw_ratio = (double)out->unique_reads / (double)out->unique_writes;
  out->reread_ratio = (double)out->unique_reads / (double)out->total_reads;
  out->rewrite_ratio = (double)out->unique_writes / (double)out->total_writes;
  return 0;
}

// Group-count multiset ("count of counts") of the memory accesses at skip
// level n: pairs (c, m_c) with m_c groups of exactly c accesses, ascending c.
// Used by the tests to compare exact integer intermediates. Returns the
// number of pairs written (at most cap), or -1 on invalid input.
int64_t aiwc_oracle_count_of_counts(const uint8_t* mem, uint64_t n_mem, uint32_t space_mask, int n,
                                    uint64_t* c_out, uint64_t* m_out, uint64_t cap) {
  std::vector<uint64_t> keys;
  for (uint64_t i = 0; i < n_mem; ++i) {
    const uint8_t* e = mem + 16 * i;
    uint64_t addr;
    std::memcpy(&addr, e, 8);
    if (addr >= kAddrLimit) return -1;
    uint32_t space = (e[13] >> 1) & 3u;
    if (!((space_mask >> space) & 1u)) continue;
    keys.push_back((((uint64_t)space << 61) | addr) >> n);
  }
  std::sort(keys.begin(), keys.end());
  std::map<uint64_t, uint64_t> coc;
  for (size_t i = 0; i < keys.size();) {
    size_t j = i;
    while (j < keys.size() && keys[j] == keys[i]) ++j;
    coc[j - i] += 1;
    i = j;
  }
  int64_t w = 0;
  for (auto& kv : coc) {
    if ((uint64_t)w < cap) { c_out[w] = kv.first; m_out[w] = kv.second; }
    ++w;
  }
  return w;
}

// SIMD width statistics (Table I "Max / Mean / SD SIMD Width"; Sec. V: the
// result width of every executed instruction is recorded): count, maximum,
// sum and sum of squares as exact integers. The mean and the population
// standard deviation follow from them in the caller.
void aiwc_oracle_simd(const uint16_t* widths, uint64_t n, uint64_t* count, uint64_t* mx, uint64_t* sum,
                      uint64_t* sumsq) {
  uint64_t m = 0, s = 0, q = 0;
  for (uint64_t i = 0; i < n; ++i) {
    const uint64_t w = widths[i];
    if (w > m) m = w;
    s += w;
    q += w * w;
  }
  *count = n;
  *mx = m;
  *sum = s;
  *sumsq = q;
}

}  // extern "C"
