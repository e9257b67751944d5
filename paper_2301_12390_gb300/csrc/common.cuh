// common.cuh — device-side building blocks shared by the engine's kernels.
//
// Exact integer arithmetic for the modularity gain (Section 3.2 of the paper:
// each vertex moves to the neighbouring community of greatest modularity
// increase), hashing for per-vertex community-weight tables, and warp
// reductions.  Nothing here is shared with the CPU oracle.
#pragma once
#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

namespace gbl {

// Host-side count of the engine's kernel launches (every launch site is
// written as `(count_launch(), kernel<<<...>>>(...))`).
void count_launch();
long long launches_so_far();

typedef __int128 i128;
typedef unsigned __int128 u128;

constexpr int kWarp = 32;
constexpr int32_t kEmpty = -1;

// ---------------------------------------------------------------- errors

// Device-side error codes, OR-ed into DevCounters::error.
enum : int {
  kErrProbe = 1,      // a hash table ran out of free slots (capacity too small)
  kErrRange = 2,      // an index was out of range (bad input that slipped through)
};

// Per-iteration counters written by the local-moving kernels.
struct DevCounters {
  unsigned long long moves;
  unsigned long long s_lo, s_hi;   // sum of the gains of the moves (u128)
  unsigned long long edges;        // CSR entries scanned
  unsigned long long visited;      // vertices visited
  unsigned long long nmoves_list;  // entries in the synchronous move list
  unsigned long long cands;        // distinct candidate communities evaluated (other than the own)
  int error;
  int pad;
};

// Raises a kernel's dynamic shared-memory limit on the current device the
// first time a call site launches it there (`done`: the call site's bit per
// device; several host threads may race to set it, which is harmless).
template <typename K>
inline void smem_limit_once(std::atomic<unsigned long long>& done, K kernel, size_t smem) {
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (bit) done.fetch_or(bit, std::memory_order_acq_rel);
}

// ---------------------------------------------------------- 128-bit sums

// Unsigned 128-bit atomic add from two 64-bit atomics: the low word wraps
// modulo 2^64 and the add that wraps it carries one into the high word, so
// the pair always ends at the exact total.
__device__ __forceinline__ void atomic_add_u128(unsigned long long* lo, unsigned long long* hi, u128 v) {
  unsigned long long vlo = (unsigned long long)v, vhi = (unsigned long long)(v >> 64);
  if (vlo) {
    unsigned long long old = atomicAdd(lo, vlo);
    if (old + vlo < old) vhi += 1ull;
  }
  if (vhi) atomicAdd(hi, vhi);
}

// ------------------------------------------------------------- the gain

// score(x) = M * K_{i->x} - K_i * Sigma'_x, Sigma'_x the total of community x
// without vertex i; moving i from d to c gains score(c) - score(d), which is
// M^2/2 times the modularity change.  With M^2 < 2^62 every term fits in
// int64 (Narrow); otherwise 128-bit (Wide).
template <bool WIDE> struct Arith;
template <> struct Arith<false> {
  typedef long long S;
  __device__ __forceinline__ static S lowest() { return (S)(-0x7fffffffffffffffll - 1); }
  __device__ __forceinline__ static S score(long long M, long long kix, long long Ki, long long sig) {
    return M * kix - Ki * sig;
  }
  __device__ __forceinline__ static u128 to_u128(S g) { return (u128)(unsigned long long)g; }
};
template <> struct Arith<true> {
  typedef i128 S;
  __device__ __forceinline__ static S lowest() { return (S)((u128)1 << 127); }
  __device__ __forceinline__ static S score(long long M, long long kix, long long Ki, long long sig) {
    return (i128)M * kix - (i128)Ki * sig;
  }
  __device__ __forceinline__ static u128 to_u128(S g) { return (u128)g; }
};

// (score, community) ordering: larger first, ties to the lower id.  Since
// every candidate's gain is its score minus the same score(d), the best score
// is the best gain, and ties agree.
template <typename S>
__device__ __forceinline__ bool better(S g1, int32_t c1, S g2, int32_t c2) {
  return g1 > g2 || (g1 == g2 && (unsigned)c1 < (unsigned)c2);
}

__device__ __forceinline__ long long shfl_xor_ll(long long v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
__device__ __forceinline__ i128 shfl_xor_i128(i128 v, int m) {
  unsigned long long lo = (unsigned long long)v;
  long long hi = (long long)(v >> 64);
  lo = __shfl_xor_sync(0xffffffffu, lo, m);
  hi = __shfl_xor_sync(0xffffffffu, hi, m);
  return ((i128)hi << 64) | (i128)lo;
}
__device__ __forceinline__ long long shfl_xor_s(long long v, int m) { return shfl_xor_ll(v, m); }
__device__ __forceinline__ i128 shfl_xor_s(i128 v, int m) { return shfl_xor_i128(v, m); }

// Warp-wide argmax of (gain, community) with the tie rule; every lane ends
// with the result.
template <typename S>
__device__ __forceinline__ void warp_argmax(S& g, int32_t& c) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    S g2 = shfl_xor_s(g, m);
    int32_t c2 = __shfl_xor_sync(0xffffffffu, c, m);
    if (better(g2, c2, g, c)) { g = g2; c = c2; }
  }
}

// The same with a payload that travels with the winner.
template <typename S>
__device__ __forceinline__ void warp_argmax_carry(S& g, int32_t& c, int32_t& pay) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    S g2 = shfl_xor_s(g, m);
    int32_t c2 = __shfl_xor_sync(0xffffffffu, c, m);
    int32_t p2 = __shfl_xor_sync(0xffffffffu, pay, m);
    if (better(g2, c2, g, c)) { g = g2; c = c2; pay = p2; }
  }
}

// ------------------------------------------------- block-to-item maps

// Blocks are handed out to items by prefix sums: item h owns blocks
// [pre[h] - pre[0], pre[h + 1] - pre[0]).  The item of block blk is the last
// h with pre[h] - pre[0] <= blk.  With at most CACHE items the block first
// copies pre into shared memory (`cache`, CACHE + 1 entries): one coalesced
// load instead of log2(nitems) dependent global loads at the head of every
// block.  Every thread of the block calls it (it holds a barrier).
template <int CACHE>
__device__ __forceinline__ int block_item(const int64_t* __restrict__ pre, int nitems, int64_t blk,
                                          int64_t* cache) {
  const int64_t* p = pre;
  if (nitems <= CACHE) {
    for (int t = threadIdx.x; t <= nitems; t += blockDim.x) cache[t] = pre[t];
    __syncthreads();
    p = cache;
  }
  const int64_t p0 = p[0];
  int lo = 0, hi = nitems;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (p[mid] - p0 <= blk) lo = mid; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------- hashing

__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  x ^= x >> 16; x *= 0x7feb352du;
  x ^= x >> 15; x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// Open-addressing insert-or-add into a power-of-two table (shared or global
// memory): keys int32 (kEmpty = free), values u64.  Returns false if the
// table is full (the caller records kErrProbe).
// Shared tables hold u32 sums when every sum fits (narrow arithmetic: M <
// 2^31, so any K_{i->c} <= M fits), else u64.
template <bool WIDE> struct TableVal { typedef unsigned long long T; };
template <> struct TableVal<false> { typedef unsigned int T; };

// Home slot of a key in a power-of-two shared table: multiplicative
// (Fibonacci) hashing, the top log2(CAP) bits of key * 2^32 / golden ratio
// (two instructions; consecutive community ids land far apart).
constexpr int log2_pow2(int x) { return x <= 1 ? 0 : 1 + log2_pow2(x >> 1); }
template <int CAP>
__device__ __forceinline__ uint32_t table_home(int32_t key) {
  static_assert(CAP >= 2 && (CAP & (CAP - 1)) == 0, "power-of-two table");
  return ((uint32_t)key * 0x9E3779B9u) >> (32 - log2_pow2(CAP));
}

template <int CAP, typename V>
__device__ __forceinline__ bool table_add_pow2(int32_t* keys, V* vals, int32_t key, unsigned long long w) {
  uint32_t h = table_home<CAP>(key);
#pragma unroll 1
  for (int probe = 0; probe < CAP; ++probe) {
    int32_t k = keys[h];
    if (k == kEmpty) k = atomicCAS(&keys[h], kEmpty, key);
    if (k == kEmpty || k == key) {
      atomicAdd(&vals[h], (V)w);
      return true;
    }
    h = (h + 1) & (CAP - 1);
  }
  return false;
}

// Same, also reporting the slot and whether the key is new (for touched-slot
// lists).  Returns -1 if the table is full.
template <int CAP, typename V>
__device__ __forceinline__ int table_add_pow2_slot(int32_t* keys, V* vals, int32_t key, unsigned long long w,
                                                   bool* fresh) {
  uint32_t h = table_home<CAP>(key);
  *fresh = false;
#pragma unroll 1
  for (int probe = 0; probe < CAP; ++probe) {
    int32_t k = keys[h];
    if (k == kEmpty) {
      k = atomicCAS(&keys[h], kEmpty, key);
      if (k == kEmpty) *fresh = true;
    }
    if (k == kEmpty || k == key) {
      atomicAdd(&vals[h], (V)w);
      return (int)h;
    }
    h = (h + 1) & (CAP - 1);
  }
  return -1;
}

// Lookup in a power-of-two table; 0 if absent.
template <int CAP, typename V>
__device__ __forceinline__ unsigned long long table_get_pow2(const int32_t* keys, const V* vals, int32_t key) {
  uint32_t h = table_home<CAP>(key);
#pragma unroll 1
  for (int probe = 0; probe < CAP; ++probe) {
    int32_t k = keys[h];
    if (k == key) return vals[h];
    if (k == kEmpty) return 0;
    h = (h + 1) & (CAP - 1);
  }
  return 0;
}

// Same for a table of arbitrary capacity `cap` in global memory; the slot is
// the high half of hash * cap.  `fresh` reports a key seen for the first time.
__device__ __forceinline__ bool gtable_add(int32_t* keys, unsigned long long* vals, uint32_t cap, int32_t key,
                                           unsigned long long w, bool* fresh) {
  uint32_t h = __umulhi(hash32((uint32_t)key), cap);
  *fresh = false;
#pragma unroll 1
  for (uint32_t probe = 0; probe < cap; ++probe) {
    int32_t k = *(volatile int32_t*)&keys[h];
    if (k == kEmpty) {
      k = atomicCAS(&keys[h], kEmpty, key);
      if (k == kEmpty) *fresh = true;
    }
    if (k == kEmpty || k == key) {
      atomicAdd(&vals[h], w);
      return true;
    }
    h = (h + 1 == cap) ? 0 : h + 1;
  }
  return false;
}

// gtable_add for J entries of one thread at once (k[j] = kEmpty: none): each
// round issues the compare-and-swaps of every pending entry before looking at
// any result, so J probes are in flight together instead of one.
template <int J>
__device__ __forceinline__ bool gtable_add_many(int32_t* keys, unsigned long long* vals, uint32_t cap,
                                                const int32_t* k, const unsigned long long* v) {
  uint32_t h[J];
  bool pend[J];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    pend[j] = k[j] != kEmpty;
    h[j] = pend[j] ? __umulhi(hash32((uint32_t)k[j]), cap) : 0u;
  }
#pragma unroll 1
  for (uint32_t probe = 0; probe < cap; ++probe) {
    int32_t old[J];
#pragma unroll
    for (int j = 0; j < J; ++j) old[j] = pend[j] ? atomicCAS(&keys[h[j]], kEmpty, k[j]) : kEmpty;
    bool any = false;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      if (!pend[j]) continue;
      if (old[j] == kEmpty || old[j] == k[j]) {
        atomicAdd(&vals[h[j]], v[j]);
        pend[j] = false;
      } else {
        h[j] = h[j] + 1 == cap ? 0u : h[j] + 1;
        any = true;
      }
    }
    if (!any) return true;
  }
  return false;
}

__device__ __forceinline__ unsigned long long gtable_get(const int32_t* keys, const unsigned long long* vals,
                                                         uint32_t cap, int32_t key) {
  uint32_t h = __umulhi(hash32((uint32_t)key), cap);
#pragma unroll 1
  for (uint32_t probe = 0; probe < cap; ++probe) {
    int32_t k = keys[h];
    if (k == key) return vals[h];
    if (k == kEmpty) return 0;
    h = (h + 1 == cap) ? 0 : h + 1;
  }
  return 0;
}

// ------------------------------------------------------ kernel parameters

// What every local-moving launch needs for one (class, bucket) list.
template <typename W>
struct LMArgs {
  const int64_t* off;
  const int32_t* col;
  const W* wt;
  const long long* K;        // vertex degrees (row sums)
  int32_t* memb;             // community of each vertex
  long long* sig;            // community totals Sigma_c
  int32_t* csize;            // community sizes (for the singleton guard)
  const int* d_iter;         // the iteration number, read from device memory so that one
                             // captured launch sequence serves every iteration of a pass
  int32_t* stamps[2];        // pruning: active in iteration t iff stamps[t & 1][i] == t;
                             // a move marks stamps[(t + 1) & 1] with t + 1
  int2* moves;               // synchronous: (vertex, target) of every move of the class
  DevCounters* ctr;
  long long M;
  // several graphs in one run (block-diagonal CSR); gid == nullptr means one graph
  const int32_t* gid;        // graph of each vertex
  const long long* Mg;       // total weight M of each graph
  const int32_t* g_on;       // graph still iterating in this pass
  unsigned long long* g_moves;  // per-graph moves of the iteration
  unsigned long long* g_s;      // per-graph S of the iteration (lo, hi)
  int prune;
  int guard;
  // hub path: per-hub global tables (2 deg slots each, per class from slot 0)
  int32_t* hkeys;
  unsigned long long* hvals;
  const int64_t* hbase;      // table offset of hub h (the class's first hub at hbase[0])
  const int64_t* spre;       // first slot chunk of hub h (absolute within the pass)
  unsigned long long* hkid;  // K_{i->d} of hub h, looked up before the scan clears the table
  int32_t* hdone;            // scan blocks of hub h finished so far (back to 0 by the last one)
  int32_t* hmoved;           // iteration + 1 when hub h moved in that iteration
  long long* hpart;          // per slot chunk: best gain (lo, hi)
  int32_t* hpart_c;          // per slot chunk: its community
};

}  // namespace gbl
