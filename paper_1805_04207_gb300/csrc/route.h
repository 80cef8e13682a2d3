// Host routing of events to partitions and shards.
//
// Every metric is a function of distributions that add exactly over a split
// of the events into whole units (Sec. V adds each work-group's results into
// the invocation's global state; the same holds for any split that keeps the
// units whole): memory groups of every skip level lie inside one superblock
// of 2^11 addresses (space, address >> 11), a branch history inside one site,
// an ITB chain inside one work-item. A partition (one device, reduced one
// after another) and a shard (one rank) are both such splits; they differ only
// in how many there are and where each one is reduced.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <thread>
#include <vector>

#include "aiwc.h"

namespace aiwc {

// SplitMix64's output function (Steele, Lea & Flood 2014) as the routing hash.
inline uint64_t route_hash(uint64_t key) {
  uint64_t z = key + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Partition of a routing key; n_parts is a power of two.
inline uint32_t part_of(uint64_t key, uint32_t n_parts) {
  return (uint32_t)(route_hash(key) & (uint64_t)(n_parts - 1));
}

// Shard of a routing key; any number of shards.
inline uint32_t shard_of(uint64_t key, uint32_t n_shards) { return (uint32_t)(route_hash(key) % n_shards); }

// Routing key of a memory event: its superblock, with the space tag.
inline uint64_t mem_route_key(const aiwc_mem_event& e) {
  return ((uint64_t)((e.flags >> 1) & 3u) << 56) | ((e.addr & (AIWC_ADDR_LIMIT - 1)) >> 11);
}

// Byte-granular addresses: an access whose bytes cross a superblock boundary
// travels as two accesses, one on each side, so that every unit stays whole.
// Writes the split stream to *out and returns true when some access crosses.
inline bool split_at_superblocks(const aiwc_mem_event* e, size_t n, std::vector<aiwc_mem_event>* out) {
  auto crosses = [](const aiwc_mem_event& x) {
    return x.addr < AIWC_ADDR_LIMIT && x.size > 1 && (x.addr >> 11) != ((x.addr + x.size - 1) >> 11);
  };
  size_t cross = 0;
  for (size_t i = 0; i < n; ++i) cross += crosses(e[i]) ? 1 : 0;
  if (!cross) return false;
  out->clear();
  out->reserve(n + cross);
  for (size_t i = 0; i < n; ++i) {
    if (!crosses(e[i])) {
      out->push_back(e[i]);
      continue;
    }
    const uint64_t b = ((e[i].addr >> 11) + 1) << 11;
    aiwc_mem_event lo = e[i], hi = e[i];
    lo.size = (uint8_t)(b - e[i].addr);
    hi.addr = b;
    hi.size = (uint8_t)(e[i].size - lo.size);
    out->push_back(lo);
    out->push_back(hi);
  }
  return true;
}

// A stable partition of n items over the host's cores: the partition of
// each item, per-thread counts, offsets by (partition, thread), then each
// thread copies its items in order. `key(i)` names item i's partition (below
// P <= 256); `size(i)` its length in units; `copy(i, p, at)` writes item i to
// partition p at unit offset `at`; `grow(p, units)` resizes partition p (and
// returns its current length when units is 0).
template <typename Key, typename Size, typename Grow, typename Copy>
void stable_partition(size_t n, uint32_t P, Key key, Size size, Grow grow, Copy copy) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t T = n < (1u << 16) ? 1 : std::min<size_t>(hw, 32);
  std::vector<uint8_t> pid(n);
  std::vector<std::vector<uint64_t>> cnt(T, std::vector<uint64_t>(P, 0));
  auto range = [&](size_t t) { return std::make_pair(n * t / T, n * (t + 1) / T); };
  auto par = [&](auto fn) {
    std::vector<std::thread> ts;
    for (size_t t = 1; t < T; ++t) ts.emplace_back(fn, t);
    fn(0);
    for (auto& th : ts) th.join();
  };
  par([&](size_t t) {
    auto r = range(t);
    for (size_t i = r.first; i < r.second; ++i) {
      const uint32_t p = key(i);
      pid[i] = (uint8_t)p;
      cnt[t][p] += size(i);
    }
  });
  std::vector<std::vector<uint64_t>> at(T, std::vector<uint64_t>(P, 0));
  for (uint32_t p = 0; p < P; ++p) {
    uint64_t base = grow(p, 0);  // current length
    for (size_t t = 0; t < T; ++t) {
      at[t][p] = base;
      base += cnt[t][p];
    }
    grow(p, base);
  }
  par([&](size_t t) {
    auto r = range(t);
    for (size_t i = r.first; i < r.second; ++i) {
      const uint32_t p = pid[i];
      copy(i, p, at[t][p]);
      at[t][p] += size(i);
    }
  });
}

}  // namespace aiwc
