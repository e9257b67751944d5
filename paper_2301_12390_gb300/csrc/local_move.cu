// local_move.cu — the local-moving phase (Section 3.2 of the paper).
//
// For every visited vertex i: sum the edge weight from i to each neighbouring
// community (K_{i->c}, self-loop excluded), evaluate the exact gain of moving
// to each of them, and move to the best one if its gain is positive (ties to
// the lowest community id).  The paper's per-thread hashtable becomes, here,
// one table per vertex sized to its degree class:
//
//   bucket 0  degree 1..8       one thread per vertex, table in registers
//   bucket 1  degree 9..32      one warp per vertex, 64-slot shared table
//   bucket 2  degree 33..128    one warp per vertex, 256-slot shared table
//   bucket 3  degree 129..1024  one block per vertex, 2048-slot shared table
//   bucket 4  degree 1025..4096 one block per vertex, 8192-slot shared table
//   bucket 5  degree > 4096     hub: several blocks insert into a global
//                               table of 2*degree slots, one block decides
//
// Synchronous mode (Jacobi): decisions read the state at the start of the
// class and append (vertex, target) to a move list; lm_commit applies the
// list afterwards.  Asynchronous mode (Gauss-Seidel-like): a decision is
// applied at once (memberships stored, totals and sizes updated with
// atomics), so later decisions may see it.
#include <climits>
#include "common.cuh"
#include "engine.h"

namespace gbl {

// --------------------------------------------------------- small helpers

// Synchronous launches never write memberships, totals or sizes, so they
// read them through the read-only path; asynchronous launches use plain
// loads, which may return a value that another vertex has since changed —
// exactly the staleness the asynchronous variant allows.
template <bool ASYNC>
__device__ __forceinline__ int32_t ld_memb(const int32_t* p) {
  if (ASYNC) return *p;
  return __ldg(p);
}
template <bool ASYNC>
__device__ __forceinline__ long long ld_sig(const long long* p) {
  if (ASYNC) return *p;
  return __ldg(p);
}
template <bool ASYNC>
__device__ __forceinline__ int32_t ld_size(const int32_t* p) {
  if (ASYNC) return *p;
  return __ldg(p);
}

// Block-level accumulators, flushed once per block.
struct BlockAcc {
  unsigned long long moves, edges, s_lo, s_hi;
  int error;
};

__device__ __forceinline__ void acc_init(BlockAcc& b) {
  if (threadIdx.x == 0) { b.moves = 0; b.edges = 0; b.s_lo = 0; b.s_hi = 0; b.error = 0; }
}
__device__ __forceinline__ void acc_flush(BlockAcc& b, DevCounters* ctr) {
  if (threadIdx.x == 0) {
    if (b.moves) atomicAdd(&ctr->moves, b.moves);
    if (b.edges) atomicAdd(&ctr->edges, b.edges);
    u128 s = ((u128)b.s_hi << 64) | (u128)b.s_lo;
    if (s) atomic_add_u128(&ctr->s_lo, &ctr->s_hi, s);
    if (b.error) atomicOr(&ctr->error, b.error);
  }
}

// Decide-and-apply for vertex i (called by one thread): guard, then either
// an in-place move (asynchronous) or an entry in the move list (synchronous).
// Returns whether the vertex moves.
template <typename W, bool WIDE, bool ASYNC>
__device__ __forceinline__ bool commit_choice(const LMArgs<W>& a, BlockAcc& acc, int32_t i, int32_t d, long long Ki,
                                              typename Arith<WIDE>::S g, int32_t c) {
  if (c < 0 || !(g > 0)) return false;
  if (a.guard && c > d && ld_size<ASYNC>(a.csize + d) == 1 && ld_size<ASYNC>(a.csize + c) == 1) return false;
  if (ASYNC) {
    a.memb[i] = c;
    atomicAdd((unsigned long long*)(a.sig + d), (unsigned long long)(-Ki));
    atomicAdd((unsigned long long*)(a.sig + c), (unsigned long long)Ki);
    atomicSub(a.csize + d, 1);
    atomicAdd(a.csize + c, 1);
  } else {
    unsigned long long pos = atomicAdd(&a.ctr->nmoves_list, 1ull);
    a.moves[pos] = make_int2(i, c);
  }
  atomicAdd(&acc.moves, 1ull);
  u128 gv = Arith<WIDE>::to_u128(g);
  atomic_add_u128(&acc.s_lo, &acc.s_hi, gv);
  return true;
}

template <typename W>
__device__ __forceinline__ bool is_active(const LMArgs<W>& a, int32_t i) {
  return !a.prune || a.iter == 0 || a.stamp_r[i] == a.iter;
}

// --------------------------------------------- bucket 0: thread per vertex

template <typename W, bool WIDE, bool ASYNC>
__global__ void __launch_bounds__(256) lm_thread(LMArgs<W> a, const int32_t* __restrict__ verts, int nverts) {
  typedef typename Arith<WIDE>::S S;
  __shared__ BlockAcc acc;
  acc_init(acc);
  __syncthreads();
  for (int vi = blockIdx.x * blockDim.x + threadIdx.x; vi < nverts; vi += gridDim.x * blockDim.x) {
    int32_t i = verts[vi];
    if (!is_active(a, i)) continue;
    int64_t b = a.off[i], e = a.off[i + 1];
    int32_t d = a.memb[i];
    long long Ki = a.K[i];
    int32_t ck[8];
    unsigned long long cw[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) { ck[k] = kEmpty; cw[k] = 0; }
    int cnt = 0;
    for (int64_t x = b; x < e; ++x) {
      int32_t j = a.col[x];
      if (j == i) continue;
      int32_t c = ld_memb<ASYNC>(a.memb + j);
      unsigned long long w = (unsigned long long)a.wt[x];
      bool found = false;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (ck[k] == c) { cw[k] += w; found = true; }
      if (!found) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (k == cnt) { ck[k] = c; cw[k] = w; }
        ++cnt;
      }
    }
    unsigned long long kid = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (ck[k] == d) kid = cw[k];
    S score_d = Arith<WIDE>::score(a.M, (long long)kid, Ki, ld_sig<ASYNC>(a.sig + d) - Ki);
    S bg = 0;
    int32_t bc = -1;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      int32_t c = ck[k];
      if (c != kEmpty && c != d) {
        S g = Arith<WIDE>::score(a.M, (long long)cw[k], Ki, ld_sig<ASYNC>(a.sig + c)) - score_d;
        if (better(g, c, bg, bc)) { bg = g; bc = c; }
      }
    }
    atomicAdd(&acc.edges, (unsigned long long)(e - b));
    if (commit_choice<W, WIDE, ASYNC>(a, acc, i, d, Ki, bg, bc) && a.prune) {
      a.stamp_w[i] = a.iter + 1;
      for (int64_t x = b; x < e; ++x) a.stamp_w[a.col[x]] = a.iter + 1;
    }
  }
  __syncthreads();
  acc_flush(acc, a.ctr);
}

// ------------------------------------------ buckets 1-2: warp per vertex

template <typename W, bool WIDE, bool ASYNC, int CAP>
__global__ void __launch_bounds__(256) lm_warp(LMArgs<W> a, const int32_t* __restrict__ verts, int nverts) {
  typedef typename Arith<WIDE>::S S;
  constexpr int WPB = 8;
  __shared__ int32_t skeys[WPB][CAP];
  __shared__ unsigned long long svals[WPB][CAP];
  __shared__ BlockAcc acc;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* keys = skeys[wib];
  unsigned long long* vals = svals[wib];
  acc_init(acc);
  for (int t = lane; t < CAP; t += kWarp) { keys[t] = kEmpty; vals[t] = 0; }
  __syncthreads();
  bool ok = true;
  for (int vi = blockIdx.x * WPB + wib; vi < nverts; vi += gridDim.x * WPB) {
    int32_t i = verts[vi];
    if (!is_active(a, i)) continue;
    int64_t b = a.off[i], e = a.off[i + 1];
    int32_t d = a.memb[i];
    long long Ki = a.K[i];
    for (int64_t x = b + lane; x < e; x += kWarp) {
      int32_t j = a.col[x];
      if (j != i) ok &= table_add_pow2<CAP>(keys, vals, ld_memb<ASYNC>(a.memb + j), (unsigned long long)a.wt[x]);
    }
    __syncwarp();
    unsigned long long kid = table_get_pow2<CAP>(keys, vals, d);
    S score_d = Arith<WIDE>::score(a.M, (long long)kid, Ki, ld_sig<ASYNC>(a.sig + d) - Ki);
    __syncwarp();
    S bg = 0;
    int32_t bc = -1;
    for (int t = lane; t < CAP; t += kWarp) {
      int32_t c = keys[t];
      if (c != kEmpty) {
        if (c != d) {
          S g = Arith<WIDE>::score(a.M, (long long)vals[t], Ki, ld_sig<ASYNC>(a.sig + c)) - score_d;
          if (better(g, c, bg, bc)) { bg = g; bc = c; }
        }
        keys[t] = kEmpty;
        vals[t] = 0;
      }
    }
    warp_argmax(bg, bc);
    bool moved = false;
    if (lane == 0) {
      atomicAdd(&acc.edges, (unsigned long long)(e - b));
      moved = commit_choice<W, WIDE, ASYNC>(a, acc, i, d, Ki, bg, bc);
    }
    moved = __shfl_sync(0xffffffffu, moved, 0);
    if (moved && a.prune) {
      if (lane == 0) a.stamp_w[i] = a.iter + 1;
      for (int64_t x = b + lane; x < e; x += kWarp) a.stamp_w[a.col[x]] = a.iter + 1;
    }
    __syncwarp();
  }
  if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicOr(&acc.error, kErrProbe);
  __syncthreads();
  acc_flush(acc, a.ctr);
}

// ----------------------------------------- buckets 3-4: block per vertex

template <typename W, bool WIDE, bool ASYNC, int CAP, int THREADS>
__global__ void __launch_bounds__(THREADS) lm_block(LMArgs<W> a, const int32_t* __restrict__ verts, int nverts) {
  typedef typename Arith<WIDE>::S S;
  constexpr int NW = THREADS / kWarp;
  // dynamic shared memory: values (CAP u64), keys (CAP i32), touched slots (CAP/2 i32)
  extern __shared__ unsigned long long dyn[];
  unsigned long long* vals = dyn;
  int32_t* keys = (int32_t*)(dyn + CAP);
  int32_t* touched = keys + CAP;
  __shared__ BlockAcc acc;
  __shared__ S red_g[NW];
  __shared__ int32_t red_c[NW];
  __shared__ unsigned long long s_kid;
  __shared__ int s_moved, s_nt;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  acc_init(acc);
  if (threadIdx.x == 0) s_nt = 0;
  for (int t = threadIdx.x; t < CAP; t += THREADS) { keys[t] = kEmpty; vals[t] = 0; }
  __syncthreads();
  bool ok = true;
  for (int vi = blockIdx.x; vi < nverts; vi += gridDim.x) {
    int32_t i = verts[vi];
    if (!is_active(a, i)) continue;   // uniform across the block
    int64_t b = a.off[i], e = a.off[i + 1];
    int32_t d = a.memb[i];
    long long Ki = a.K[i];
    for (int64_t x = b + threadIdx.x; x < e; x += THREADS) {
      int32_t j = a.col[x];
      if (j != i) {
        bool fresh;
        int h = table_add_pow2_slot<CAP>(keys, vals, ld_memb<ASYNC>(a.memb + j), (unsigned long long)a.wt[x], &fresh);
        if (h < 0) ok = false;
        else if (fresh) touched[atomicAdd(&s_nt, 1)] = h;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) s_kid = table_get_pow2<CAP>(keys, vals, d);
    __syncthreads();
    const int nt = s_nt;
    S score_d = Arith<WIDE>::score(a.M, (long long)s_kid, Ki, ld_sig<ASYNC>(a.sig + d) - Ki);
    S bg = 0;
    int32_t bc = -1;
    for (int t = threadIdx.x; t < nt; t += THREADS) {
      int h = touched[t];
      int32_t c = keys[h];
      if (c != d) {
        S g = Arith<WIDE>::score(a.M, (long long)vals[h], Ki, ld_sig<ASYNC>(a.sig + c)) - score_d;
        if (better(g, c, bg, bc)) { bg = g; bc = c; }
      }
      keys[h] = kEmpty;
      vals[h] = 0;
    }
    warp_argmax(bg, bc);
    if (lane == 0) { red_g[wid] = bg; red_c[wid] = bc; }
    __syncthreads();
    if (wid == 0) {
      bg = lane < NW ? red_g[lane] : (S)0;
      bc = lane < NW ? red_c[lane] : -1;
      warp_argmax(bg, bc);
      if (lane == 0) {
        atomicAdd(&acc.edges, (unsigned long long)(e - b));
        s_moved = commit_choice<W, WIDE, ASYNC>(a, acc, i, d, Ki, bg, bc);
        s_nt = 0;
      }
    }
    __syncthreads();
    if (s_moved && a.prune) {
      if (threadIdx.x == 0) a.stamp_w[i] = a.iter + 1;
      for (int64_t x = b + threadIdx.x; x < e; x += THREADS) a.stamp_w[a.col[x]] = a.iter + 1;
    }
  }
  if (!ok) atomicOr(&acc.error, kErrProbe);
  __syncthreads();
  acc_flush(acc, a.ctr);
}

// ------------------------------------------------- bucket 5: hub vertices

constexpr int kHubChunk = 2048;

// hub h of the launch's list owns table slots [hbase[h], hbase[h] + 2 deg).
// Blocks are (hub, chunk) pairs; chunk_pre[h] is the first block of hub h.
template <typename W, bool ASYNC>
__global__ void __launch_bounds__(256) lm_hub_insert(LMArgs<W> a, const int32_t* __restrict__ hubs, int nhubs,
                                                     const int64_t* __restrict__ chunk_pre) {
  // a chunk's entries are first summed per community in a shared table, then
  // each distinct community is added once to the hub's global table
  constexpr int CAP = 2 * kHubChunk;
  extern __shared__ unsigned long long hdyn[];
  unsigned long long* svals = hdyn;
  int32_t* skeys = (int32_t*)(hdyn + CAP);
  // find the hub of this block: last h with chunk_pre[h] - chunk_pre[0] <= blockIdx.x
  const int64_t cb = chunk_pre[0];
  int lo = 0, hi = nhubs;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (chunk_pre[mid] - cb <= (int64_t)blockIdx.x) lo = mid; else hi = mid;
  }
  const int h = lo;
  const int32_t i = hubs[h];
  if (!is_active(a, i)) return;   // uniform across the block
  const int64_t q = (int64_t)blockIdx.x - (chunk_pre[h] - cb);
  for (int t = threadIdx.x; t < CAP; t += blockDim.x) { skeys[t] = kEmpty; svals[t] = 0; }
  __syncthreads();
  const int64_t b = a.off[i], e = a.off[i + 1];
  const int64_t base = a.hbase[h];
  const uint32_t cap = (uint32_t)(2 * (e - b));
  int32_t* keys = a.hkeys + base;
  unsigned long long* vals = a.hvals + base;
  const int64_t x0 = b + q * kHubChunk, x1 = min(e, x0 + kHubChunk);
  bool ok = true;
  for (int64_t x = x0 + threadIdx.x; x < x1; x += blockDim.x) {
    int32_t j = a.col[x];
    if (j == i) continue;
    ok &= table_add_pow2<CAP>(skeys, svals, ld_memb<ASYNC>(a.memb + j), (unsigned long long)a.wt[x]);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < CAP; t += blockDim.x) {
    int32_t c = skeys[t];
    if (c == kEmpty) continue;
    bool fresh;
    ok &= gtable_add(keys, vals, cap, c, svals[t], &fresh);
    if (fresh) {
      int pos = atomicAdd(a.hcount + h, 1);
      a.hslots[base + pos] = c;   // record the key; the decide step looks it up
    }
  }
  if (!ok) atomicOr(&a.ctr->error, kErrProbe);
}

// One block per hub: evaluate every distinct neighbour community, choose,
// commit, reset the table.
template <typename W, bool WIDE, bool ASYNC>
__global__ void __launch_bounds__(256) lm_hub_decide(LMArgs<W> a, const int32_t* __restrict__ hubs, int nhubs) {
  typedef typename Arith<WIDE>::S S;
  constexpr int NW = 256 / kWarp;
  __shared__ BlockAcc acc;
  __shared__ S red_g[NW];
  __shared__ int32_t red_c[NW];
  __shared__ int s_moved;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  acc_init(acc);
  __syncthreads();
  for (int h = blockIdx.x; h < nhubs; h += gridDim.x) {
    const int32_t i = hubs[h];
    if (!is_active(a, i)) continue;
    const int64_t b = a.off[i], e = a.off[i + 1];
    const int64_t base = a.hbase[h];
    const uint32_t cap = (uint32_t)(2 * (e - b));
    int32_t* keys = a.hkeys + base;
    unsigned long long* vals = a.hvals + base;
    const int32_t d = a.memb[i];
    const long long Ki = a.K[i];
    const int cnt = a.hcount[h];
    unsigned long long kid = gtable_get(keys, vals, cap, d);
    S score_d = Arith<WIDE>::score(a.M, (long long)kid, Ki, ld_sig<ASYNC>(a.sig + d) - Ki);
    S bg = 0;
    int32_t bc = -1;
    for (int t = threadIdx.x; t < cnt; t += 256) {
      int32_t c = a.hslots[base + t];
      if (c == d) continue;
      unsigned long long v = gtable_get(keys, vals, cap, c);
      S g = Arith<WIDE>::score(a.M, (long long)v, Ki, ld_sig<ASYNC>(a.sig + c)) - score_d;
      if (better(g, c, bg, bc)) { bg = g; bc = c; }
    }
    warp_argmax(bg, bc);
    if (lane == 0) { red_g[wid] = bg; red_c[wid] = bc; }
    __syncthreads();
    if (wid == 0) {
      bg = lane < NW ? red_g[lane] : (S)0;
      bc = lane < NW ? red_c[lane] : -1;
      warp_argmax(bg, bc);
      if (lane == 0) {
        atomicAdd(&acc.edges, (unsigned long long)(e - b));
        s_moved = commit_choice<W, WIDE, ASYNC>(a, acc, i, d, Ki, bg, bc);
      }
    }
    __syncthreads();
    // reset the table: clear the slot of every recorded key
    for (int t = threadIdx.x; t < cnt; t += 256) {
      int32_t c = a.hslots[base + t];
      uint32_t hs = __umulhi(hash32((uint32_t)c), cap);
      for (uint32_t probe = 0; probe < cap; ++probe) {
        if (keys[hs] == c) { keys[hs] = kEmpty; vals[hs] = 0; break; }
        hs = (hs + 1 == cap) ? 0 : hs + 1;
      }
    }
    if (s_moved && a.prune) {
      if (threadIdx.x == 0) a.stamp_w[i] = a.iter + 1;
      for (int64_t x = b + threadIdx.x; x < e; x += 256) a.stamp_w[a.col[x]] = a.iter + 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) a.hcount[h] = 0;
  }
  __syncthreads();
  acc_flush(acc, a.ctr);
}

// ----------------------------------------------- synchronous commit step

template <typename W>
__global__ void __launch_bounds__(256) lm_commit(LMArgs<W> a) {
  const unsigned long long n = a.ctr->nmoves_list;
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < n;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    int2 mv = a.moves[t];
    int32_t i = mv.x, c = mv.y, d = a.memb[i];
    long long Ki = a.K[i];
    a.memb[i] = c;
    atomicAdd((unsigned long long*)(a.sig + d), (unsigned long long)(-Ki));
    atomicAdd((unsigned long long*)(a.sig + c), (unsigned long long)Ki);
    atomicSub(a.csize + d, 1);
    atomicAdd(a.csize + c, 1);
  }
}

__global__ void reset_move_list(DevCounters* ctr) { ctr->nmoves_list = 0; }

// ---------------------------------------------------------------- launch

namespace {

template <typename K>
int grid_for(K kernel, int threads, size_t smem, int work_blocks) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  int g = sms * per_sm;
  if (work_blocks < g) g = work_blocks;
  return g < 1 ? 1 : g;
}

template <typename W, bool WIDE, bool ASYNC>
void launch_bucket_t(const LMArgs<W>& a, int bucket, const int32_t* verts, int nverts, cudaStream_t s) {
  if (nverts <= 0) return;
  switch (bucket) {
    case 0: {
      auto k = lm_thread<W, WIDE, ASYNC>;
      k<<<grid_for(k, 256, 0, (nverts + 255) / 256), 256, 0, s>>>(a, verts, nverts);
      break;
    }
    case 1: {
      auto k = lm_warp<W, WIDE, ASYNC, 64>;
      k<<<grid_for(k, 256, 0, (nverts + 7) / 8), 256, 0, s>>>(a, verts, nverts);
      break;
    }
    case 2: {
      auto k = lm_warp<W, WIDE, ASYNC, 256>;
      k<<<grid_for(k, 256, 0, (nverts + 7) / 8), 256, 0, s>>>(a, verts, nverts);
      break;
    }
    case 3: {
      constexpr int CAP = 2048;
      size_t smem = (size_t)CAP * 14;
      auto k = lm_block<W, WIDE, ASYNC, CAP, 128>;
      k<<<grid_for(k, 128, smem, nverts), 128, smem, s>>>(a, verts, nverts);
      break;
    }
    case 4: {
      constexpr int CAP = 8192;
      size_t smem = (size_t)CAP * 14;
      auto k = lm_block<W, WIDE, ASYNC, CAP, 256>;
      static bool attr = false;
      if (!attr) {
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
      }
      k<<<grid_for(k, 256, smem, nverts), 256, smem, s>>>(a, verts, nverts);
      break;
    }
    default: break;
  }
}

}  // namespace

template <typename W>
void lm_launch_bucket(const LMArgs<W>& a, bool wide, bool async, int bucket, const int32_t* verts, int nverts,
                      cudaStream_t s) {
  if (wide) {
    if (async) launch_bucket_t<W, true, true>(a, bucket, verts, nverts, s);
    else launch_bucket_t<W, true, false>(a, bucket, verts, nverts, s);
  } else {
    if (async) launch_bucket_t<W, false, true>(a, bucket, verts, nverts, s);
    else launch_bucket_t<W, false, false>(a, bucket, verts, nverts, s);
  }
}

template <typename W>
void lm_launch_hubs(const LMArgs<W>& a, bool wide, bool async, const int32_t* hubs, int nhubs,
                    const int64_t* chunk_pre, int64_t nchunks, cudaStream_t s) {
  if (nhubs <= 0 || nchunks <= 0) return;
  const size_t smem = (size_t)(2 * kHubChunk) * 12;
  if (async) lm_hub_insert<W, true><<<(unsigned)nchunks, 256, smem, s>>>(a, hubs, nhubs, chunk_pre);
  else lm_hub_insert<W, false><<<(unsigned)nchunks, 256, smem, s>>>(a, hubs, nhubs, chunk_pre);
  int g = nhubs < 4096 ? nhubs : 4096;
  if (wide) {
    if (async) lm_hub_decide<W, true, true><<<g, 256, 0, s>>>(a, hubs, nhubs);
    else lm_hub_decide<W, true, false><<<g, 256, 0, s>>>(a, hubs, nhubs);
  } else {
    if (async) lm_hub_decide<W, false, true><<<g, 256, 0, s>>>(a, hubs, nhubs);
    else lm_hub_decide<W, false, false><<<g, 256, 0, s>>>(a, hubs, nhubs);
  }
}

template <typename W>
void lm_launch_commit(const LMArgs<W>& a, int64_t max_moves, cudaStream_t s) {
  if (max_moves <= 0) return;
  int blocks = (int)((max_moves + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  lm_commit<W><<<blocks, 256, 0, s>>>(a);
  reset_move_list<<<1, 1, 0, s>>>(a.ctr);
}

template void lm_launch_bucket<int32_t>(const LMArgs<int32_t>&, bool, bool, int, const int32_t*, int, cudaStream_t);
template void lm_launch_bucket<int64_t>(const LMArgs<int64_t>&, bool, bool, int, const int32_t*, int, cudaStream_t);
template void lm_launch_hubs<int32_t>(const LMArgs<int32_t>&, bool, bool, const int32_t*, int, const int64_t*,
                                      int64_t, cudaStream_t);
template void lm_launch_hubs<int64_t>(const LMArgs<int64_t>&, bool, bool, const int32_t*, int, const int64_t*,
                                      int64_t, cudaStream_t);
template void lm_launch_commit<int32_t>(const LMArgs<int32_t>&, int64_t, cudaStream_t);
template void lm_launch_commit<int64_t>(const LMArgs<int64_t>&, int64_t, cudaStream_t);

}  // namespace gbl
