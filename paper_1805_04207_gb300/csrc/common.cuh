// Small device helpers shared by the kernels.
#pragma once

#include "aiwc_internal.cuh"

namespace aiwc {

template <typename T, typename Op>
__device__ __forceinline__ T warp_reduce(T x, Op op) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = op(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

struct OpAdd { template <typename T> __device__ T operator()(T a, T b) const { return a + b; } };
struct OpOr { template <typename T> __device__ T operator()(T a, T b) const { return a | b; } };
struct OpAnd { template <typename T> __device__ T operator()(T a, T b) const { return a & b; } };
struct OpMin { template <typename T> __device__ T operator()(T a, T b) const { return a < b ? a : b; } };
struct OpMax { template <typename T> __device__ T operator()(T a, T b) const { return a > b ? a : b; } };

// Block-wide reduction; every thread gets the result. scratch: 32 entries.
template <typename T, typename Op>
__device__ __forceinline__ T block_reduce(T x, Op op, T identity, T* scratch) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  x = warp_reduce(x, op);
  __syncthreads();
  if (lane == 0) scratch[w] = x;
  __syncthreads();
  T v = lane < nw ? scratch[lane] : identity;
  v = warp_reduce(v, op);
  return v;
}

// Marks work-item ids in a bitmap, one atomicOr per distinct bitmap word in
// the warp. All 32 lanes must call it; lanes with valid == false add nothing.
// Ids >= max_wi are not marked and raise *err_bits |= kErrWorkItem.
__device__ __forceinline__ void mark_work_items(u32* bitmap, u64 max_wi, u32 wi, bool valid, u32* err_bits) {
  const int lane = threadIdx.x & 31;
  if (valid && (u64)wi >= max_wi) {
    *err_bits |= kErrWorkItem;
    valid = false;
  }
  u32 todo = __ballot_sync(0xffffffffu, valid);
  const u32 word = wi >> 5;
  const u32 bit = 1u << (wi & 31);
  // common case: every valid lane's id falls in one bitmap word
  const int first = todo ? __ffs(todo) - 1 : 0;
  const u32 w0 = __shfl_sync(0xffffffffu, word, first);
  if (__all_sync(0xffffffffu, !valid || word == w0)) {
    const u32 bits = __reduce_or_sync(0xffffffffu, valid ? bit : 0u);
    if (todo && lane == first) atomicOr(&bitmap[w0], bits);
    return;
  }
  while (todo) {
    const int leader = __ffs(todo) - 1;
    const u32 lw = __shfl_sync(0xffffffffu, word, leader);
    const bool mine = ((todo >> lane) & 1u) && word == lw;
    const u32 grp = __ballot_sync(0xffffffffu, mine);
    const u32 bits = __reduce_or_sync(0xffffffffu, mine ? bit : 0u);
    if (lane == leader) atomicOr(&bitmap[lw], bits);
    todo &= ~grp;
  }
}

// Appends a tagged value to the overflow list.
__device__ __forceinline__ void overflow_append(u64* over, u64 cap, DevState* st, int tag, u64 value) {
  const u64 e = ((u64)tag << 56) | (value & kValueMask);
  const u64 idx = atomicAdd(&st->n_over, 1ull);
  if (idx < cap) {
    over[idx] = e;
    atomicOr(&st->over_or, e);
    atomicAnd(&st->over_and, e);
  } else {
    atomicOr(&st->err, kErrOverflow);
  }
}

__device__ __forceinline__ u64 umin64(u64 a, u64 b) { return a < b ? a : b; }
__device__ __forceinline__ u64 umax64(u64 a, u64 b) { return a > b ? a : b; }

__device__ __forceinline__ bool gate_open(const u32* gate, u32 want) { return !gate || *gate == want; }

// Home slot of a superblock key: fold to 32 bits, multiply by a 32-bit odd
// constant (Knuth's multiplicative hashing) and keep the high bits through
// the caller's mask after a final mix of the high half into the low half.
__device__ __forceinline__ u64 sbt_hash(u64 k) {
  const u32 x = (u32)k ^ (u32)(k >> 32) * 0x85EBCA6Bu;
  const u32 y = x * 0x9E3779B1u;
  return (u64)(y ^ (y >> 15));
}

// Slot of key k (> 0), inserting it if absent; kNoSlot when the probe limit is
// reached. `first` is keys[pos] already loaded for the home position pos.
__device__ __forceinline__ u32 sbt_place(const SbTable& t, u64 k, u64 pos, u64 first) {
  u64 cur = first;
  for (int p = 0; p < kMaxProbe; ++p) {
    if (cur == k) return (u32)pos;
    if (cur == 0ull) {
      const u64 old = atomicCAS(&t.keys[pos], 0ull, k);
      if (old == 0ull || old == k) return (u32)pos;
    }
    pos = (pos + 1) & t.mask;
    cur = __ldcg(&t.keys[pos]);
  }
  return kNoSlot;
}

// Slot of key k, which must already be in the table; kNoSlot if absent.
__device__ __forceinline__ u32 sbt_find(const SbTable& t, u64 k) {
  u64 pos = sbt_hash(k) & t.mask;
  for (int p = 0; p < kMaxProbe; ++p) {
    const u64 cur = t.keys[pos];
    if (cur == k) return (u32)pos;
    if (cur == 0ull) return kNoSlot;
    pos = (pos + 1) & t.mask;
  }
  return kNoSlot;
}

}  // namespace aiwc
