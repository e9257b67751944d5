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

__device__ __forceinline__ unsigned lanemask_lt_lm() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Synchronous launches never write memberships, totals or sizes, so they
// read them through the read-only path; asynchronous launches use plain
// loads, which may return a value that another vertex has since changed —
// exactly the staleness the asynchronous variant allows.
// Loads of memberships, community totals and sizes.  LD 0: read-only path
// (nothing writes them while the kernel runs: a synchronous class); 1: plain
// (asynchronous in-place updates, any recent value will do); 2: L2 only (the
// kernel itself updates them between its classes and must see the result).
template <int LD, typename T>
__device__ __forceinline__ T ld_state(const T* p) {
  if (LD == 0) return __ldg(p);
  if (LD == 2) return __ldcg(p);
  return *p;
}
template <bool ASYNC>
__device__ __forceinline__ int32_t ld_memb(const int32_t* p) {
  return ld_state<ASYNC ? 1 : 0>(p);
}
template <bool ASYNC>
__device__ __forceinline__ long long ld_sig(const long long* p) {
  return ld_state<ASYNC ? 1 : 0>(p);
}
template <bool ASYNC>
__device__ __forceinline__ int32_t ld_size(const int32_t* p) {
  return ld_state<ASYNC ? 1 : 0>(p);
}

// Block-level accumulators, flushed once per block.
struct BlockAcc {
  unsigned long long moves, edges, visited, s_lo, s_hi, cands;
  int error;
};

__device__ __forceinline__ void acc_init(BlockAcc& b) {
  if (threadIdx.x == 0) { b.moves = 0; b.edges = 0; b.visited = 0; b.s_lo = 0; b.s_hi = 0; b.cands = 0; b.error = 0; }
}
__device__ __forceinline__ void acc_flush(BlockAcc& b, DevCounters* ctr) {
  if (threadIdx.x == 0) {
    if (b.moves) atomicAdd(&ctr->moves, b.moves);
    if (b.edges) atomicAdd(&ctr->edges, b.edges);
    if (b.visited) atomicAdd(&ctr->visited, b.visited);
    if (b.cands) atomicAdd(&ctr->cands, b.cands);
    u128 s = ((u128)b.s_hi << 64) | (u128)b.s_lo;
    if (s) atomic_add_u128(&ctr->s_lo, &ctr->s_hi, s);
    if (b.error) atomicOr(&ctr->error, b.error);
  }
}

__device__ __forceinline__ u128 warp_sum_u128(u128 v) {
  unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long l2 = __shfl_xor_sync(0xffffffffu, lo, o), h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    const unsigned long long nl = lo + l2;
    hi = hi + h2 + (nl < lo ? 1ull : 0ull);
    lo = nl;
  }
  return ((u128)hi << 64) | (u128)lo;
}

// All 32 lanes of a warp: the moves and gains of the lanes that moved (gv of
// a lane that did not is ignored), summed per graph of a batch and added
// with one atomic per distinct graph, or to the block's accumulator.
template <typename W>
__device__ __forceinline__ void warp_move_totals(const LMArgs<W>& a, BlockAcc& acc, bool moved, int graph, u128 gv) {
  unsigned pend = __ballot_sync(0xffffffffu, moved);
  while (pend) {
    const int leader = __ffs(pend) - 1;
    const int gl = __shfl_sync(0xffffffffu, graph, leader);
    const bool in = moved && (!a.gid || graph == gl);
    const unsigned inm = __ballot_sync(0xffffffffu, in);
    const u128 sum = warp_sum_u128(in ? gv : (u128)0);
    if ((int)(threadIdx.x & 31) == leader) {
      if (a.gid) {
        atomicAdd(a.g_moves + gl, (unsigned long long)__popc(inm));
        atomic_add_u128(a.g_s + 2 * gl, a.g_s + 2 * gl + 1, sum);
      } else {
        atomicAdd(&acc.moves, (unsigned long long)__popc(inm));
        atomic_add_u128(&acc.s_lo, &acc.s_hi, sum);
      }
    }
    pend &= ~inm;
  }
}

// Decide-and-apply for vertex i (called by one thread): guard, then either
// an in-place move (asynchronous) or an entry in the move list (synchronous).
// Returns whether the vertex moves.
// `best` is the best candidate's score, `score_d` the vertex's own; the move
// needs gain = best - score_d > 0.
// sd, szd: Sigma_d and the size of d, loaded with the vertex's row (constant
// within a synchronous class; an asynchronous decision may use any recent
// value).  size_c: the size of c when the caller loaded it with the
// candidates (the guard's test), else -1 and it is loaded here.
template <typename W, bool WIDE, bool ASYNC, int LD = (ASYNC ? 1 : 0)>
__device__ __forceinline__ bool commit_choice(const LMArgs<W>& a, BlockAcc& acc, int32_t i, int32_t d, long long Ki,
                                              long long sd, int32_t szd, typename Arith<WIDE>::S best, int32_t c,
                                              unsigned long long kid, long long M, int graph,
                                              u128* defer_gain = nullptr, int32_t size_c = -1) {
  if (c < 0) return false;
  typedef typename Arith<WIDE>::S S;
  const S g = best - Arith<WIDE>::score(M, (long long)kid, Ki, sd - Ki);
  if (!(g > 0)) return false;
  if (a.guard && c > d && szd == 1 && (size_c >= 0 ? size_c : ld_state<LD>(a.csize + c)) == 1) return false;
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
  u128 gv = Arith<WIDE>::to_u128(g);   // g > 0 here
  if (defer_gain) {   // the caller adds the move and its gain
    *defer_gain = gv;
    return true;
  }
  if (a.gid) {
    atomicAdd(a.g_moves + graph, 1ull);
    atomic_add_u128(a.g_s + 2 * graph, a.g_s + 2 * graph + 1, gv);
  } else {
    atomicAdd(&acc.moves, 1ull);
    atomic_add_u128(&acc.s_lo, &acc.s_hi, gv);
  }
  return true;
}

// The graph of vertex i and its M; false if that graph has stopped
// iterating in this pass.
template <typename W>
__device__ __forceinline__ bool graph_of(const LMArgs<W>& a, int32_t i, long long* M, int* g) {
  if (!a.gid) {
    *M = a.M;
    *g = 0;
    return true;
  }
  const int gg = a.gid[i];
  *g = gg;
  if (!a.g_on[gg]) return false;
  *M = a.Mg[gg];
  return true;
}

// The iteration and its stamp buffers, read once at kernel start.
struct IterView {
  int iter;
  const int32_t* sr;   // read: active in this iteration
  int32_t* sw;         // write: active in the next one
};

template <typename W>
__device__ __forceinline__ IterView iter_view(const LMArgs<W>& a) {
  const int it = *a.d_iter;
  return IterView{it, a.stamps[it & 1], a.stamps[(it + 1) & 1]};
}

template <typename W>
__device__ __forceinline__ bool is_active(const LMArgs<W>& a, const IterView& iv, int32_t i) {
  return !a.prune || iv.iter == 0 || iv.sr[i] == iv.iter;
}

// What a per-vertex kernel needs of list entry vi before its row: loaded one
// vertex ahead so that these loads overlap the previous vertex.
struct VertexInfo {
  int32_t i, d, szd;
  bool on;        // in range, active and its graph still iterating
  int graph;
  int64_t b, e;
  long long Ki, M, sd;
};

template <typename W, bool ASYNC, int LD = (ASYNC ? 1 : 0)>
__device__ __forceinline__ VertexInfo vertex_info(const LMArgs<W>& a, const IterView& iv,
                                                  const int32_t* __restrict__ verts, int nverts, int vi) {
  VertexInfo v;
  v.on = false;
  v.i = 0;
  v.d = 0;
  v.szd = 0;
  v.graph = 0;
  v.b = v.e = 0;
  v.Ki = v.M = v.sd = 0;
  if (vi >= nverts) return v;
  v.i = verts[vi];
  v.b = a.off[v.i];
  v.e = a.off[v.i + 1];
  v.d = ld_state<LD == 2 ? 2 : 1>(a.memb + v.i);
  v.Ki = a.K[v.i];
  v.on = is_active(a, iv, v.i) && graph_of(a, v.i, &v.M, &v.graph);
  if (v.on) {   // the loads that depend on d, only for a vertex that is visited
    v.sd = ld_state<LD>(a.sig + v.d);
    v.szd = ld_state<LD>(a.csize + v.d);
  }
  return v;
}

// Pruning marks of a vertex that moved: the vertex and every neighbour are
// active in the next iteration.  The row's columns are loaded together
// before the marks are stored (a load after a store to the stamps would wait
// for it), U at a time per thread; the entries b + lane0, + step, ... are
// this thread's, and the thread with lane0 == 0 marks the vertex itself.
template <int U, typename W>
__device__ __forceinline__ void mark_row(const LMArgs<W>& a, const IterView& iv, int32_t i, int64_t b, int64_t e,
                                         int lane0 = 0, int step = 1, bool self = true) {
  if (self && lane0 == 0) iv.sw[i] = iv.iter + 1;
  for (int64_t x0 = b + lane0; x0 < e; x0 += (int64_t)U * step) {
    int32_t cc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t x = x0 + (int64_t)u * step;
      cc[u] = x < e ? __ldg(a.col + x) : -1;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (cc[u] >= 0) iv.sw[cc[u]] = iv.iter + 1;
  }
}

// --------------------------------------------- bucket 0: thread per vertex

// The row (<= 8 entries) is loaded first and its neighbours' communities
// gathered with all loads in flight; duplicates are then merged in registers.
// Lane l of the calling warp takes list entry vi (none if vi >= nverts); all
// 32 lanes call it.  Whole warps sum their counters, moves and gains over the
// warp: per-lane atomics on the block's counters serialise (measured: a third
// of the thread kernel's time).
template <typename W, bool WIDE, bool ASYNC>
__device__ __forceinline__ void thread_vertex(const LMArgs<W>& a, const IterView& iv, BlockAcc& acc,
                                              const int32_t* __restrict__ verts, int64_t nverts, int64_t vi) {
  typedef typename Arith<WIDE>::S S;
  {
    bool moved = false;
    u128 gv = 0;
    int graph = 0;
    unsigned n_edges = 0, n_visited = 0, n_cand = 0;
    do {
      if (vi >= nverts) break;
      int32_t i = verts[vi];
      // the vertex's row bounds, community and degree are loaded together
      // with its stamp, before the activity test
      const int64_t b = a.off[i], e = a.off[i + 1];
      const int32_t d = a.memb[i];
      const long long Ki = a.K[i];
      if (!is_active(a, iv, i)) break;
      long long M;
      if (!graph_of(a, i, &M, &graph)) break;
      const long long sd = ld_sig<ASYNC>(a.sig + d);
      const int32_t szd = ld_size<ASYNC>(a.csize + d);
      int32_t cc[8];
      unsigned long long ww[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const bool v = b + k < e;
        cc[k] = v ? a.col[b + k] : i;
        ww[k] = v ? (unsigned long long)a.wt[b + k] : 0ull;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) cc[k] = cc[k] != i ? ld_memb<ASYNC>(a.memb + cc[k]) : kEmpty;
#pragma unroll
      for (int k = 1; k < 8; ++k) {
        bool merged = false;
#pragma unroll
        for (int l = 0; l < k; ++l)
          if (!merged && cc[k] != kEmpty && cc[l] == cc[k]) { ww[l] += ww[k]; merged = true; }
        if (merged) cc[k] = kEmpty;
      }
      unsigned long long kid = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (cc[k] == d) kid = ww[k];
      // the candidates' totals, and for a singleton under the guard their
      // sizes too (loaded with the totals instead of after the choice)
      const bool want_size = a.guard && szd == 1;
      long long sg[8];
      int32_t sz[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const bool cand = cc[k] != kEmpty && cc[k] != d;
        sg[k] = cand ? ld_sig<ASYNC>(a.sig + cc[k]) : 0;
        sz[k] = cand && want_size && cc[k] > d ? ld_size<ASYNC>(a.csize + cc[k]) : 0;
      }
      S bg = Arith<WIDE>::lowest();
      int32_t bc = -1, bsz = 0;
      unsigned ncand = 0;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (cc[k] != kEmpty && cc[k] != d) {
          ++ncand;
          S g = Arith<WIDE>::score(M, (long long)ww[k], Ki, sg[k]);
          if (better(g, cc[k], bg, bc)) { bg = g; bc = cc[k]; bsz = sz[k]; }
        }
      }
      n_cand = ncand;
      n_edges = (unsigned)(e - b);
      n_visited = 1;
      moved = commit_choice<W, WIDE, ASYNC>(a, acc, i, d, Ki, sd, szd, bg, bc, kid, M, graph, &gv, bsz);
      if (moved && a.prune) mark_row<8>(a, iv, i, b, e);
    } while (false);
    n_edges = __reduce_add_sync(0xffffffffu, n_edges);
    n_visited = __reduce_add_sync(0xffffffffu, n_visited);
    n_cand = __reduce_add_sync(0xffffffffu, n_cand);
    if ((threadIdx.x & 31) == 0 && n_visited) {
      atomicAdd(&acc.edges, (unsigned long long)n_edges);
      atomicAdd(&acc.visited, (unsigned long long)n_visited);
      atomicAdd(&acc.cands, (unsigned long long)n_cand);
    }
    warp_move_totals(a, acc, moved, graph, gv);
  }
}

template <typename W, bool WIDE, bool ASYNC>
__global__ void __launch_bounds__(256, 3) lm_thread(LMArgs<W> a, const int32_t* __restrict__ verts, int nverts) {
  const IterView iv = iter_view(a);
  __shared__ BlockAcc acc;
  acc_init(acc);
  __syncthreads();
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < nverts; base += gridDim.x * blockDim.x)
    thread_vertex<W, WIDE, ASYNC>(a, iv, acc, verts, nverts, base + (int)(threadIdx.x & 31));
  __syncthreads();
  acc_flush(acc, a.ctr);
}

// --------------------- bucket 1, narrow arithmetic: thread per vertex, sorted

// A vertex of degree <= D by one lane: its row is loaded and the neighbours'
// communities gathered with all loads in flight, the (community, weight)
// pairs sorted by community with a bitonic network in registers (static
// indices), each run of one community summed into its first position, and the
// runs' totals gathered in two halves (bounded registers).  Same decisions as
// the warp kernel it replaces for narrow sums (K_{i->c} < 2^31).  All 32
// lanes call it.
template <typename W, bool ASYNC, int D>
__device__ __forceinline__ void thread_vertex_sorted(const LMArgs<W>& a, const IterView& iv, BlockAcc& acc,
                                                     const int32_t* __restrict__ verts, int64_t nverts, int64_t vi) {
  typedef typename Arith<false>::S S;
  static_assert((D & (D - 1)) == 0 && D <= 32, "power-of-two network of at most 32");
  constexpr int32_t kPast = 0x7fffffff;   // sorts after every community id
  constexpr int H = D / 2;
  bool moved = false;
  u128 gv = 0;
  int graph = 0;
  unsigned n_edges = 0, n_visited = 0, n_cand = 0;
  do {
    if (vi >= nverts) break;
    const int32_t i = verts[vi];
    const int64_t b = a.off[i], e = a.off[i + 1];
    const int32_t d = a.memb[i];
    const long long Ki = a.K[i];
    if (!is_active(a, iv, i)) break;
    long long M;
    if (!graph_of(a, i, &M, &graph)) break;
    const long long sd = ld_sig<ASYNC>(a.sig + d);
    const int32_t szd = ld_size<ASYNC>(a.csize + d);
    int32_t k[D];
    unsigned w[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const bool v = b + j < e;
      k[j] = v ? a.col[b + j] : i;
      w[j] = v ? (unsigned)a.wt[b + j] : 0u;
    }
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const bool other = k[j] != i;   // a self-loop adds to no K_{i->c}
      k[j] = other ? ld_memb<ASYNC>(a.memb + k[j]) : kPast;
      if (!other) w[j] = 0u;
    }
#pragma unroll
    for (int kk = 2; kk <= D; kk <<= 1) {
#pragma unroll
      for (int jj = kk >> 1; jj > 0; jj >>= 1) {
#pragma unroll
        for (int x = 0; x < D; ++x) {
          const int y = x ^ jj;
          if (y > x) {
            const bool up = (x & kk) == 0;
            if ((k[x] > k[y]) == up) {
              const int32_t tk = k[x]; k[x] = k[y]; k[y] = tk;
              const unsigned tw = w[x]; w[x] = w[y]; w[y] = tw;
            }
          }
        }
      }
    }
    // run heads (first position of each community) carry the run's sum
    unsigned heads = 0u, run = 0u;
#pragma unroll
    for (int j = D - 1; j >= 0; --j) {
      run += w[j];
      if (k[j] != kPast && (j == 0 || k[j] != k[j - 1])) {
        heads |= 1u << j;
        w[j] = run;
        run = 0u;
      }
    }
    unsigned long long kid = 0;
#pragma unroll
    for (int j = 0; j < D; ++j)
      if (((heads >> j) & 1u) && k[j] == d) kid = w[j];
    const bool want_size = a.guard && szd == 1;
    S bg = Arith<false>::lowest();
    int32_t bc = -1, bsz = 0;
    unsigned ncand = 0;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      long long sg[H];
      bool one[H];
#pragma unroll
      for (int t = 0; t < H; ++t) {
        const int j = half * H + t;
        const bool cand = ((heads >> j) & 1u) && k[j] != d;
        sg[t] = cand ? ld_sig<ASYNC>(a.sig + k[j]) : 0;
        one[t] = cand && want_size && k[j] > d && ld_size<ASYNC>(a.csize + k[j]) == 1;
      }
#pragma unroll
      for (int t = 0; t < H; ++t) {
        const int j = half * H + t;
        if (((heads >> j) & 1u) && k[j] != d) {
          ++ncand;
          const S g = Arith<false>::score(M, (long long)w[j], Ki, sg[t]);
          if (better(g, k[j], bg, bc)) { bg = g; bc = k[j]; bsz = one[t] ? 1 : 0; }
        }
      }
    }
    n_cand = ncand;
    n_edges = (unsigned)(e - b);
    n_visited = 1;
    moved = commit_choice<W, false, ASYNC>(a, acc, i, d, Ki, sd, szd, bg, bc, kid, M, graph, &gv, bsz);
    if (moved && a.prune) mark_row<8>(a, iv, i, b, e);
  } while (false);
  n_edges = __reduce_add_sync(0xffffffffu, n_edges);
  n_visited = __reduce_add_sync(0xffffffffu, n_visited);
  n_cand = __reduce_add_sync(0xffffffffu, n_cand);
  if ((threadIdx.x & 31) == 0 && n_visited) {
    atomicAdd(&acc.edges, (unsigned long long)n_edges);
    atomicAdd(&acc.visited, (unsigned long long)n_visited);
    atomicAdd(&acc.cands, (unsigned long long)n_cand);
  }
  warp_move_totals(a, acc, moved, graph, gv);
}

template <typename W, bool ASYNC, int D>
__global__ void __launch_bounds__(128) lm_thread_sorted(LMArgs<W> a, const int32_t* __restrict__ verts, int nverts) {
  const IterView iv = iter_view(a);
  __shared__ BlockAcc acc;
  acc_init(acc);
  __syncthreads();
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < nverts; base += gridDim.x * blockDim.x)
    thread_vertex_sorted<W, ASYNC, D>(a, iv, acc, verts, nverts, base + (int)(threadIdx.x & 31));
  __syncthreads();
  acc_flush(acc, a.ctr);
}

// ------------------------------------------ buckets 1-2: warp per vertex

// One vertex of degree <= U * 32 by one warp: its neighbour communities summed
// in the warp's shared table (CAP slots, left empty again), the best score
// against its own community's, the move committed and its neighbours marked.
// SIZES: a singleton under the guard loads its candidates' sizes with their
// totals (one dependent load less before the decision; off where the
// registers would spill).
template <typename W, bool WIDE, bool ASYNC, int CAP, int U, int LD, bool SIZES>
__device__ __forceinline__ void warp_vertex(const LMArgs<W>& a, const IterView& iv, BlockAcc& acc, int32_t* keys,
                                            typename TableVal<WIDE>::T* vals, const VertexInfo& cur, int lane,
                                            bool& ok) {
  typedef typename Arith<WIDE>::S S;
  typedef typename TableVal<WIDE>::T V;
  const int32_t i = cur.i, d = cur.d;
  const int64_t b = cur.b, e = cur.e;
  const long long Ki = cur.Ki, M = cur.M;
  const int graph = cur.graph;
  for (int64_t x0 = b; x0 < e; x0 += U * kWarp) {
    // rounds of 32 entries that hold at least one (the rest are skipped)
    const int nu = (int)min((int64_t)U, (e - x0 + kWarp - 1) / kWarp);
    int32_t cc[U];
    unsigned long long ww[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      cc[u] = i;
      ww[u] = 0ull;
      if (u < nu) {
        const int64_t x = x0 + u * kWarp + lane;
        if (x < e) {
          cc[u] = a.col[x];
          ww[u] = (unsigned long long)a.wt[x];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) cc[u] = cc[u] != i ? ld_state<LD>(a.memb + cc[u]) : kEmpty;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (cc[u] != kEmpty) ok &= table_add_pow2<CAP, V>(keys, vals, cc[u], ww[u]);
  }
  __syncwarp();
  // a singleton under the guard loads its candidates' sizes with their
  // totals and carries the best one's through the reduction
  const bool want_size = SIZES && a.guard && cur.szd == 1;
  unsigned long long kid = 0;
  S bg = Arith<WIDE>::lowest();
  int32_t bc = -1, bsz = 0;
  unsigned ncand = 0;
#pragma unroll
  for (int t0 = 0; t0 < CAP; t0 += kWarp * 4) {
    int32_t cs[4];
    long long sg[4];
    unsigned long long vs[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = t0 + u * kWarp + lane;
      cs[u] = t < CAP ? keys[t] : kEmpty;
      vs[u] = t < CAP ? vals[t] : 0ull;
    }
    bool one[4];   // the candidate is a singleton (asked only for the guard)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool cand = cs[u] != kEmpty && cs[u] != d;
      sg[u] = cand ? ld_state<LD>(a.sig + cs[u]) : 0;
      one[u] = cand && want_size && cs[u] > d && ld_state<LD>(a.csize + cs[u]) == 1;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int t = t0 + u * kWarp + lane;
      if (cs[u] != kEmpty) {
        if (cs[u] != d) {
          ++ncand;
          S g = Arith<WIDE>::score(M, (long long)vs[u], Ki, sg[u]);
          if (better(g, cs[u], bg, bc)) { bg = g; bc = cs[u]; bsz = one[u] ? 1 : 0; }
        } else {
          kid = vs[u];
        }
        keys[t] = kEmpty;
        vals[t] = 0;
      }
    }
  }
  if (want_size) warp_argmax_carry(bg, bc, bsz);
  else warp_argmax(bg, bc);
  ncand = __reduce_add_sync(0xffffffffu, ncand);
  {
    const unsigned has = __ballot_sync(0xffffffffu, kid != 0);
    kid = has ? __shfl_sync(0xffffffffu, kid, __ffs(has) - 1) : 0ull;
  }
  bool moved = false;
  if (lane == 0) {
    atomicAdd(&acc.cands, (unsigned long long)ncand);
    atomicAdd(&acc.edges, (unsigned long long)(e - b));
    atomicAdd(&acc.visited, 1ull);
    moved = commit_choice<W, WIDE, ASYNC, LD>(a, acc, i, d, Ki, cur.sd, cur.szd, bg, bc, kid, M, graph, nullptr,
                                              want_size ? bsz : -1);
  }
  moved = __shfl_sync(0xffffffffu, moved, 0);
  if (moved && a.prune) mark_row<U>(a, iv, i, b, e, lane, kWarp);
}

// U entries per lane are loaded and gathered before any insert (U * 32 covers
// the bucket's largest degree), so their memory latencies overlap.
template <typename W, bool WIDE, bool ASYNC, int CAP, int U>
__global__ void __launch_bounds__(256, 4) lm_warp(LMArgs<W> a, const int32_t* __restrict__ verts, int nverts) {
  const IterView iv = iter_view(a);
  typedef typename Arith<WIDE>::S S;
  typedef typename TableVal<WIDE>::T V;
  constexpr int WPB = 8;
  __shared__ int32_t skeys[WPB][CAP];
  __shared__ V svals[WPB][CAP];
  __shared__ BlockAcc acc;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* keys = skeys[wib];
  V* vals = svals[wib];
  acc_init(acc);
  for (int t = lane; t < CAP; t += kWarp) { keys[t] = kEmpty; vals[t] = 0; }
  __syncthreads();
  bool ok = true;
  const int stride = gridDim.x * WPB;
  VertexInfo nx = vertex_info<W, ASYNC>(a, iv, verts, nverts, blockIdx.x * WPB + wib);
  for (int vi = blockIdx.x * WPB + wib; vi < nverts; vi += stride) {
    const VertexInfo cur = nx;
    nx = vertex_info<W, ASYNC>(a, iv, verts, nverts, vi + stride);
    if (!cur.on) continue;
    warp_vertex<W, WIDE, ASYNC, CAP, U, (ASYNC ? 1 : 0), (CAP <= 64 && !WIDE)>(a, iv, acc, keys, vals, cur, lane,
                                                                                 ok);
    __syncwarp();
  }
  if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicOr(&acc.error, kErrProbe);
  __syncthreads();
  acc_flush(acc, a.ctr);
}

// ----------------------------- small pass graphs: one launch per class
//
// When no vertex of the pass graph has degree above 128 and the graph is
// small, the launches of a class are few microseconds of work each: one
// kernel then takes the whole class instead of one kernel per bucket on
// forked streams: a lane per vertex of bucket 0 (as lm_thread), a warp per
// vertex of buckets 1-2 (as lm_warp, 256-slot tables).  ko = the bucket
// offsets of the class lists (device).
template <typename W, bool WIDE, bool ASYNC>
__global__ void __launch_bounds__(256, 3) lm_class(LMArgs<W> a, const int32_t* __restrict__ list,
                                                   const int64_t* __restrict__ ko, int P, int ch) {
  const IterView iv = iter_view(a);
  typedef typename TableVal<WIDE>::T V;
  constexpr int WPB = 8, CAP = 256, U = 4;
  __shared__ int32_t skeys[WPB][CAP];
  __shared__ V svals[WPB][CAP];
  __shared__ BlockAcc acc;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* keys = skeys[wib];
  V* vals = svals[wib];
  acc_init(acc);
  for (int t = lane; t < CAP; t += kWarp) { keys[t] = kEmpty; vals[t] = 0; }
  __syncthreads();
  bool ok = true;
  const int64_t r0 = ko[ch], n0 = ko[ch + 1] - r0;
  const int64_t r1 = ko[P + ch], n1 = ko[P + ch + 1] - r1;
  const int64_t r2 = ko[2 * P + ch], n2 = ko[2 * P + ch + 1] - r2;
  // work items of a warp: 32 degree-<=8 vertices (a lane each, as the thread
  // kernel), then one vertex of degree 9-128 each
  const int64_t m0 = (n0 + kWarp - 1) / kWarp;
  const int64_t tot = m0 + n1 + n2;
  for (int64_t t = (int64_t)blockIdx.x * WPB + wib; t < tot; t += (int64_t)gridDim.x * WPB) {
    if (t < m0) {
      thread_vertex<W, WIDE, ASYNC>(a, iv, acc, list + r0, n0, t * kWarp + lane);
      continue;
    }
    const int64_t u = t - m0;
    const int64_t idx = u < n1 ? r1 + u : r2 + (u - n1);
    const VertexInfo cur = vertex_info<W, ASYNC>(a, iv, list + idx, 1, 0);
    if (!cur.on) continue;
    warp_vertex<W, WIDE, ASYNC, CAP, U, (ASYNC ? 1 : 0), !WIDE>(a, iv, acc, keys, vals, cur, lane, ok);
    __syncwarp();
  }
  if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicOr(&acc.error, kErrProbe);
  __syncthreads();
  acc_flush(acc, a.ctr);
}

// ----------------------------------------- buckets 3-4: block per vertex

// A decided move waiting for the block to commit it, with its row bounds
// (for the pruning marks).
struct PendingMove {
  int32_t i, c, d, pad;
  int64_t b, e;
};

// Commit and mark the pending moves of a block (all threads take part).
template <typename W, bool ASYNC>
__device__ __forceinline__ void flush_moves(const LMArgs<W>& a, const IterView& iv, const PendingMove* q, int n,
                                            int tid, int nthr) {
  for (int t = tid; t < n; t += nthr) {
    const PendingMove m = q[t];
    if (ASYNC) {
      const long long Ki = a.K[m.i];
      a.memb[m.i] = m.c;
      atomicAdd((unsigned long long*)(a.sig + m.d), (unsigned long long)(-Ki));
      atomicAdd((unsigned long long*)(a.sig + m.c), (unsigned long long)Ki);
      atomicSub(a.csize + m.d, 1);
      atomicAdd(a.csize + m.c, 1);
    } else {
      unsigned long long pos = atomicAdd(&a.ctr->nmoves_list, 1ull);
      a.moves[pos] = make_int2(m.i, m.c);
    }
  }
  if (a.prune)   // one warp per move, the warps' moves in parallel
    for (int t = tid >> 5; t < n; t += nthr >> 5) mark_row<8>(a, iv, q[t].i, q[t].b, q[t].e, tid & 31, kWarp);
}

// Decide (no commit yet): the exact gain of the best candidate against the
// vertex's own community, the guard, and the S / move counts.
// sd, szd: Sigma_d and the size of d, read when the vertex's row was
// (constant within a synchronous class; an asynchronous decision may use any
// recent value).
template <typename W, bool WIDE, bool ASYNC>
__device__ __forceinline__ bool decide_move(const LMArgs<W>& a, BlockAcc& acc, int32_t d, long long Ki, long long sd,
                                            int32_t szd, typename Arith<WIDE>::S best, int32_t c,
                                            unsigned long long kid, long long M, int graph) {
  if (c < 0) return false;
  typedef typename Arith<WIDE>::S S;
  const S g = best - Arith<WIDE>::score(M, (long long)kid, Ki, sd - Ki);
  if (!(g > 0)) return false;
  if (a.guard && c > d && szd == 1 && ld_size<ASYNC>(a.csize + c) == 1) return false;
  const u128 gv = Arith<WIDE>::to_u128(g);
  if (a.gid) {
    atomicAdd(a.g_moves + graph, 1ull);
    atomic_add_u128(a.g_s + 2 * graph, a.g_s + 2 * graph + 1, gv);
  } else {
    atomicAdd(&acc.moves, 1ull);
    atomic_add_u128(&acc.s_lo, &acc.s_hi, gv);
  }
  return true;
}

// Two barriers per vertex: the small shared values alternate between two
// copies by vertex parity, so the next vertex can start while warp 0 still
// reduces and decides; moves queue in shared memory and are committed by the
// whole block when the queue fills and at the end.
template <typename W, bool WIDE, bool ASYNC, int CAP, int THREADS>
__global__ void __launch_bounds__(THREADS, THREADS <= 128 ? 8 : 2)
    lm_block(LMArgs<W> a, const int32_t* __restrict__ verts, int nverts) {
  const IterView iv = iter_view(a);
  typedef typename Arith<WIDE>::S S;
  typedef typename TableVal<WIDE>::T V;
  constexpr int NW = THREADS / kWarp;
  constexpr int U = 4;
  constexpr int QCAP = 64;
  // dynamic shared memory: values (CAP V), keys (CAP i32), touched slots (CAP/2 u16)
  extern __shared__ unsigned long long dyn[];
  V* vals = (V*)dyn;
  int32_t* keys = (int32_t*)(vals + CAP);
  uint16_t* touched = (uint16_t*)(keys + CAP);
  __shared__ BlockAcc acc;
  __shared__ S red_g[2][NW];
  __shared__ int32_t red_c[2][NW];
  __shared__ unsigned long long s_kid[2];
  __shared__ int s_nt[2];
  __shared__ PendingMove queue[QCAP];
  __shared__ int q_n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  acc_init(acc);
  if (threadIdx.x == 0) { s_nt[0] = s_nt[1] = 0; s_kid[0] = s_kid[1] = 0; q_n = 0; }
  for (int t = threadIdx.x; t < CAP; t += THREADS) { keys[t] = kEmpty; vals[t] = 0; }
  __syncthreads();
  bool ok = true;
  int p = 0;
  // The next vertex's list entry, activity, row bounds, community and degree
  // are loaded while the current one is processed.
  VertexInfo nx = vertex_info<W, ASYNC>(a, iv, verts, nverts, blockIdx.x);
  for (int vi = blockIdx.x; vi < nverts; vi += gridDim.x) {
    const VertexInfo cur = nx;
    if (!cur.on) {   // uniform across the block
      nx = vertex_info<W, ASYNC>(a, iv, verts, nverts, vi + gridDim.x);
      continue;
    }
    const int32_t i = cur.i, d = cur.d;
    const int64_t b = cur.b, e = cur.e;
    const long long Ki = cur.Ki, M = cur.M;
    const int graph = cur.graph;
    for (int64_t x0 = b; x0 < e; x0 += U * THREADS) {
      // this warp's rounds that hold at least one entry (the rest skipped)
      const int64_t rem = e - x0 - wid * kWarp;
      const int nu = rem <= 0 ? 0 : (int)min((int64_t)U, (rem + THREADS - 1) / THREADS);
      int32_t cc[U];
      unsigned long long ww[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        cc[u] = i;
        ww[u] = 0ull;
        if (u < nu) {
          const int64_t x = x0 + u * THREADS + threadIdx.x;
          if (x < e) {
            cc[u] = a.col[x];
            ww[u] = (unsigned long long)a.wt[x];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) cc[u] = cc[u] != i ? ld_memb<ASYNC>(a.memb + cc[u]) : kEmpty;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (u >= nu) break;
        bool fresh = false;
        int h = -1;
        if (cc[u] != kEmpty) {
          h = table_add_pow2_slot<CAP, V>(keys, vals, cc[u], ww[u], &fresh);
          if (h < 0) ok = false;
        }
        // one append per warp for the new keys of its lanes
        const unsigned m = __ballot_sync(0xffffffffu, fresh);
        int base = 0;
        if (lane == 0 && m) base = atomicAdd(&s_nt[p], __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (fresh) touched[base + __popc(m & lanemask_lt_lm())] = (uint16_t)h;
      }
    }
    nx = vertex_info<W, ASYNC>(a, iv, verts, nverts, vi + gridDim.x);
    __syncthreads();   // B1: table complete; warp 0 has finished the previous vertex
    if (q_n >= QCAP) {   // uniform: q_n was last written before this barrier
      flush_moves<W, ASYNC>(a, iv, queue, q_n, threadIdx.x, THREADS);
      __syncthreads();
      if (threadIdx.x == 0) q_n = 0;
    }
    if (threadIdx.x == 0) { s_nt[p ^ 1] = 0; s_kid[p ^ 1] = 0; }   // the next vertex's copies
    const int nt = s_nt[p];
    S bg = Arith<WIDE>::lowest();
    int32_t bc = -1;
    for (int t0 = 0; t0 < nt; t0 += U * THREADS) {
      const int rem = nt - t0 - wid * kWarp;
      const int nu = rem <= 0 ? 0 : min(U, (rem + THREADS - 1) / THREADS);
      int hs[U];
      int32_t cs[U];
      long long sg[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int t = t0 + u * THREADS + threadIdx.x;
        hs[u] = u < nu && t < nt ? (int)touched[t] : -1;
        cs[u] = hs[u] >= 0 ? keys[hs[u]] : kEmpty;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) sg[u] = (cs[u] != kEmpty && cs[u] != d) ? ld_sig<ASYNC>(a.sig + cs[u]) : 0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (hs[u] < 0) continue;
        if (cs[u] != d) {
          S g = Arith<WIDE>::score(M, (long long)vals[hs[u]], Ki, sg[u]);
          if (better(g, cs[u], bg, bc)) { bg = g; bc = cs[u]; }
        } else {
          s_kid[p] = vals[hs[u]];
        }
        keys[hs[u]] = kEmpty;
        vals[hs[u]] = 0;
      }
    }
    warp_argmax(bg, bc);
    if (lane == 0) { red_g[p][wid] = bg; red_c[p][wid] = bc; }
    __syncthreads();   // B2: candidates evaluated, table clear
    if (wid == 0) {
      bg = lane < NW ? red_g[p][lane] : Arith<WIDE>::lowest();
      bc = lane < NW ? red_c[p][lane] : -1;
      warp_argmax(bg, bc);
      if (lane == 0) {
        atomicAdd(&acc.edges, (unsigned long long)(e - b));
        atomicAdd(&acc.visited, 1ull);
        atomicAdd(&acc.cands, (unsigned long long)(s_nt[p] - (s_kid[p] != 0 ? 1 : 0)));
        if (decide_move<W, WIDE, ASYNC>(a, acc, d, Ki, cur.sd, cur.szd, bg, bc, s_kid[p], M, graph))
          queue[q_n++] = PendingMove{i, bc, d, 0, b, e};
      }
    }
    p ^= 1;
  }
  __syncthreads();
  flush_moves<W, ASYNC>(a, iv, queue, q_n, threadIdx.x, THREADS);
  if (!ok) atomicOr(&acc.error, kErrProbe);
  __syncthreads();
  acc_flush(acc, a.ctr);
}

// ------------------------------------------------- bucket 5: hub vertices
//
// Hub h of a class owns global table slots [hbase[h] - hbase[0], + 2 deg):
// every class's tables start at slot 0, so a class reuses the slots the
// previous class's scan just cleared, which are still in L2.
// 1. insert: blocks are (hub, 2048-entry chunk) pairs; each sums its chunk
//    per community in shared memory, then adds each distinct community once
//    to the hub's global table;
// 2. scan: blocks are (hub, 4096-slot chunk) pairs; each evaluates the gain
//    of every occupied slot, clears it, and leaves its chunk's best (and
//    K_{i->d} of the slot holding d); the last block of a hub reduces the
//    chunk bests and commits;
// 3. mark (once per iteration, all classes): neighbours of the hubs that moved.

constexpr int kHubChunk = (int)kHubChunkEntries;

constexpr int kItemCache = 512;   // hub prefix entries a block copies to shared memory

template <typename W, bool WIDE, bool ASYNC>
__global__ void __launch_bounds__(256) lm_hub_insert(LMArgs<W> a, const int32_t* __restrict__ hubs, int nhubs,
                                                     const int64_t* __restrict__ chunk_pre) {
  typedef typename TableVal<WIDE>::T V;
  const IterView iv = iter_view(a);
  constexpr int CAP = 2 * kHubChunk;
  extern __shared__ unsigned long long hdyn[];
  V* svals = (V*)hdyn;
  int32_t* skeys = (int32_t*)(svals + CAP);
  __shared__ int64_t s_pre[kItemCache + 1];
  const int h = block_item<kItemCache>(chunk_pre, nhubs, blockIdx.x, s_pre);
  const int32_t i = hubs[h];
  if (!is_active(a, iv, i)) return;   // uniform across the block
  {
    long long M;
    int graph;
    if (!graph_of(a, i, &M, &graph)) return;
  }
  const int64_t q = (int64_t)blockIdx.x - (chunk_pre[h] - chunk_pre[0]);
  for (int t = threadIdx.x; t < CAP; t += blockDim.x) { skeys[t] = kEmpty; svals[t] = 0; }
  __syncthreads();
  const int64_t b = a.off[i], e = a.off[i + 1];
  const int64_t base = a.hbase[h] - a.hbase[0];   // the class's tables start at slot 0
  const uint32_t cap = (uint32_t)(2 * (e - b));
  const int64_t x0 = b + q * kHubChunk, x1 = min(e, x0 + kHubChunk);
  bool ok = true;
  constexpr int U = kHubChunk / 256;
  static_assert(U >= 1 && kHubChunk % 256 == 0, "a chunk covers whole rounds of 256 threads");
  for (int64_t y = x0; y < x1; y += U * 256) {
    int32_t cc[U];
    unsigned long long ww[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t x = y + u * 256 + threadIdx.x;
      const bool v = x < x1;
      cc[u] = v ? a.col[x] : i;
      ww[u] = v ? (unsigned long long)a.wt[x] : 0ull;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) cc[u] = cc[u] != i ? ld_memb<ASYNC>(a.memb + cc[u]) : kEmpty;
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (cc[u] != kEmpty) ok &= table_add_pow2<CAP, V>(skeys, svals, cc[u], ww[u]);
  }
  __syncthreads();
  int32_t* keys = a.hkeys + base;
  unsigned long long* vals = a.hvals + base;
  constexpr int J = 8;
  for (int t0 = 0; t0 < CAP; t0 += J * 256) {
    int32_t kk[J];
    unsigned long long vv[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {   // slots past CAP (a table smaller than J * 256) read as empty
      const int t = t0 + j * 256 + (int)threadIdx.x;
      kk[j] = t < CAP ? skeys[t] : kEmpty;
      vv[j] = t < CAP ? (unsigned long long)svals[t] : 0ull;
    }
    ok &= gtable_add_many<J>(keys, vals, cap, kk, vv);
  }
  if (!ok) atomicOr(&a.ctr->error, kErrProbe);
}

// Scan blocks are (hub, kSlotChunk-slot chunk) pairs: each evaluates the
// gain of every occupied slot of its chunk, clears it, and leaves its chunk's
// best; the block that finishes a hub's last chunk (a per-hub counter after a
// fence) reduces the hub's chunk bests and commits the hub's move, so the
// decision needs no launch of its own.  No block waits for another.
template <typename W, bool WIDE, bool ASYNC>
__global__ void __launch_bounds__(256) lm_hub_scan(LMArgs<W> a, const int32_t* __restrict__ hubs, int nhubs) {
  const IterView iv = iter_view(a);
  typedef typename Arith<WIDE>::S S;
  constexpr int NW = 256 / kWarp;
  __shared__ S red_g[NW];
  __shared__ int32_t red_c[NW];
  __shared__ unsigned red_n[NW];
  __shared__ BlockAcc acc;
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __shared__ int64_t s_pre[kItemCache + 1];
  const int h = block_item<kItemCache>(a.spre, nhubs, blockIdx.x, s_pre);
  const int32_t i = hubs[h];
  if (!is_active(a, iv, i)) return;   // uniform across the block
  long long M;
  int graph;
  if (!graph_of(a, i, &M, &graph)) return;
  acc_init(acc);
  const int64_t q = (int64_t)blockIdx.x - (a.spre[h] - a.spre[0]);
  const int64_t b = a.off[i], e = a.off[i + 1];
  const int64_t cap = 2 * (e - b);
  const int64_t base = a.hbase[h] - a.hbase[0];
  const int32_t d = a.memb[i];
  const long long Ki = a.K[i];
  const int64_t t0 = q * kSlotChunk, t1 = min(cap, t0 + kSlotChunk);
  S bg = Arith<WIDE>::lowest();
  int32_t bc = -1;
  unsigned ncand = 0;
  constexpr int U = 4;
  for (int64_t y = t0; y < t1; y += U * 256) {
    int32_t cs[U];
    unsigned long long vs[U];
    long long sg[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t t = y + u * 256 + threadIdx.x;
      cs[u] = t < t1 ? a.hkeys[base + t] : kEmpty;
      vs[u] = cs[u] != kEmpty ? a.hvals[base + t] : 0ull;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) sg[u] = (cs[u] != kEmpty && cs[u] != d) ? ld_sig<ASYNC>(a.sig + cs[u]) : 0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (cs[u] == kEmpty) continue;
      const int64_t t = y + u * 256 + threadIdx.x;
      if (cs[u] != d) {
        ++ncand;
        S g = Arith<WIDE>::score(M, (long long)vs[u], Ki, sg[u]);
        if (better(g, cs[u], bg, bc)) { bg = g; bc = cs[u]; }
      } else {
        a.hkid[h] = vs[u];   // K_{i->d}; only one slot holds d
      }
      a.hkeys[base + t] = kEmpty;
      a.hvals[base + t] = 0;
    }
  }
  ncand = __reduce_add_sync(0xffffffffu, ncand);
  warp_argmax(bg, bc);
  if (lane == 0) { red_g[wid] = bg; red_c[wid] = bc; red_n[wid] = ncand; }
  __syncthreads();
  if (wid == 0) {
    bg = lane < NW ? red_g[lane] : Arith<WIDE>::lowest();
    bc = lane < NW ? red_c[lane] : -1;
    warp_argmax(bg, bc);
    ncand = __reduce_add_sync(0xffffffffu, lane < NW ? red_n[lane] : 0u);
    if (lane == 0) {
      if (ncand) atomicAdd(&a.ctr->cands, (unsigned long long)ncand);
      const int64_t slot = a.spre[h] + q;
      u128 gu = (u128)(i128)bg;
      a.hpart[2 * slot] = (long long)(unsigned long long)gu;
      a.hpart[2 * slot + 1] = (long long)(unsigned long long)(gu >> 64);
      a.hpart_c[slot] = bc;
      __threadfence();   // the chunk best (and K_{i->d}) before the count
      const int nck = (int)(a.spre[h + 1] - a.spre[h]);
      s_last = atomicAdd(a.hdone + h, 1) == nck - 1;
    }
  }
  __syncthreads();
  if (s_last && wid == 0) {   // every chunk of this hub is done: decide
    __threadfence();
    S hg = Arith<WIDE>::lowest();
    int32_t hc = -1;
    for (int64_t t = a.spre[h] + lane; t < a.spre[h + 1]; t += kWarp) {
      const i128 g = ((i128)__ldcg(a.hpart + 2 * t + 1) << 64) | (i128)(unsigned long long)__ldcg(a.hpart + 2 * t);
      const int32_t c = __ldcg(a.hpart_c + t);
      if (c >= 0 && better((S)g, c, hg, hc)) { hg = (S)g; hc = c; }
    }
    warp_argmax(hg, hc);
    if (lane == 0) {
      atomicAdd(&acc.edges, (unsigned long long)(e - b));
      atomicAdd(&acc.visited, 1ull);
      const bool moved = commit_choice<W, WIDE, ASYNC>(a, acc, i, d, Ki, ld_sig<ASYNC>(a.sig + d),
                                                       ld_size<ASYNC>(a.csize + d), hg, hc, __ldcg(a.hkid + h), M,
                                                       graph);
      a.hkid[h] = 0;
      a.hdone[h] = 0;
      if (moved && a.prune) a.hmoved[h] = iv.iter + 1;   // lm_hub_mark marks its neighbours
    }
  }
  __syncthreads();
  acc_flush(acc, a.ctr);
}

// Pruning marks of the hubs that moved in this iteration (all classes at
// once; the marks only feed the next iteration's active set): blocks are
// (hub, kHubChunkEntries-entry chunk) pairs of the pass's whole hub list.
template <typename W>
__global__ void __launch_bounds__(256) lm_hub_mark(LMArgs<W> a, const int32_t* __restrict__ hubs, int nhubs,
                                                   const int64_t* __restrict__ chunk_pre) {
  const IterView iv = iter_view(a);
  __shared__ int64_t s_pre[kItemCache + 1];
  const int h = block_item<kItemCache>(chunk_pre, nhubs, blockIdx.x, s_pre);
  if (a.hmoved[h] != iv.iter + 1) return;
  const int32_t i = hubs[h];
  const int64_t q = (int64_t)blockIdx.x - (chunk_pre[h] - chunk_pre[0]);
  const int64_t b = a.off[i], e = a.off[i + 1];
  const int64_t x0 = b + q * kHubChunk, x1 = min(e, x0 + kHubChunk);
  if (q == 0 && threadIdx.x == 0) iv.sw[i] = iv.iter + 1;
  mark_row<4>(a, iv, i, x0, x1, (int)threadIdx.x, 256, false);   // the hub itself: marked above
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
  const int per_sm = blocks_per_sm(kernel, threads, smem);
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
      (count_launch(), k<<<grid_for(k, 256, 0, (nverts + 255) / 256), 256, 0, s>>>(a, verts, nverts));
      break;
    }
    case 1: {
      if (!WIDE) {   // narrow sums: a lane per vertex, its row sorted in registers
        auto k = lm_thread_sorted<W, ASYNC, 32>;
        (count_launch(), k<<<grid_for(k, 128, 0, (nverts + 127) / 128), 128, 0, s>>>(a, verts, nverts));
      } else {
        auto k = lm_warp<W, WIDE, ASYNC, 64, 1>;
        (count_launch(), k<<<grid_for(k, 256, 0, (nverts + 7) / 8), 256, 0, s>>>(a, verts, nverts));
      }
      break;
    }
    case 2: {
      auto k = lm_warp<W, WIDE, ASYNC, 256, 4>;
      (count_launch(), k<<<grid_for(k, 256, 0, (nverts + 7) / 8), 256, 0, s>>>(a, verts, nverts));
      break;
    }
    case 3: {
      constexpr int CAP = 2048;
      size_t smem = (size_t)CAP * (sizeof(typename TableVal<WIDE>::T) + 4 + 1);
      auto k = lm_block<W, WIDE, ASYNC, CAP, 128>;
      (count_launch(), k<<<grid_for(k, 128, smem, nverts), 128, smem, s>>>(a, verts, nverts));
      break;
    }
    case 4: {
      constexpr int CAP = 8192;
      size_t smem = (size_t)CAP * (sizeof(typename TableVal<WIDE>::T) + 4 + 1);
      auto k = lm_block<W, WIDE, ASYNC, CAP, 512>;
      static std::atomic<unsigned long long> attr{0};
      smem_limit_once(attr, k, smem);
      (count_launch(), k<<<grid_for(k, 512, smem, nverts), 512, smem, s>>>(a, verts, nverts));
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
                    const int64_t* chunk_pre, int64_t nchunks, const int64_t* spre, int64_t nslotchunks,
                    cudaStream_t s) {
  if (nhubs <= 0 || nchunks <= 0) return;
  const size_t smem = (size_t)(2 * kHubChunk) * (wide ? 12 : 8);
  if (wide) {
    if (async) (count_launch(), lm_hub_insert<W, true, true><<<(unsigned)nchunks, 256, smem, s>>>(a, hubs, nhubs, chunk_pre));
    else (count_launch(), lm_hub_insert<W, true, false><<<(unsigned)nchunks, 256, smem, s>>>(a, hubs, nhubs, chunk_pre));
  } else {
    if (async) (count_launch(), lm_hub_insert<W, false, true><<<(unsigned)nchunks, 256, smem, s>>>(a, hubs, nhubs, chunk_pre));
    else (count_launch(), lm_hub_insert<W, false, false><<<(unsigned)nchunks, 256, smem, s>>>(a, hubs, nhubs, chunk_pre));
  }
  if (wide) {
    if (async) (count_launch(), lm_hub_scan<W, true, true><<<(unsigned)nslotchunks, 256, 0, s>>>(a, hubs, nhubs));
    else (count_launch(), lm_hub_scan<W, true, false><<<(unsigned)nslotchunks, 256, 0, s>>>(a, hubs, nhubs));
  } else {
    if (async) (count_launch(), lm_hub_scan<W, false, true><<<(unsigned)nslotchunks, 256, 0, s>>>(a, hubs, nhubs));
    else (count_launch(), lm_hub_scan<W, false, false><<<(unsigned)nslotchunks, 256, 0, s>>>(a, hubs, nhubs));
  }
}

template <typename W>
void lm_launch_class(const LMArgs<W>& a, bool wide, bool async, const int32_t* list, const int64_t* ko, int P,
                     int ch, int64_t nverts, cudaStream_t s) {
  if (nverts <= 0) return;
  int64_t blocks = (nverts + 7) / 8;
  if (blocks > 152 * 3) blocks = 152 * 3;   // resident blocks (three per SM)
  const unsigned g = (unsigned)blocks;
  if (wide) {
    if (async) (count_launch(), lm_class<W, true, true><<<g, 256, 0, s>>>(a, list, ko, P, ch));
    else (count_launch(), lm_class<W, true, false><<<g, 256, 0, s>>>(a, list, ko, P, ch));
  } else {
    if (async) (count_launch(), lm_class<W, false, true><<<g, 256, 0, s>>>(a, list, ko, P, ch));
    else (count_launch(), lm_class<W, false, false><<<g, 256, 0, s>>>(a, list, ko, P, ch));
  }
}

template <typename W>
void lm_launch_hub_mark(const LMArgs<W>& a, const int32_t* hubs, int nhubs, const int64_t* chunk_pre, int64_t nchunks,
                        cudaStream_t s) {
  if (nhubs <= 0 || nchunks <= 0 || !a.prune) return;
  (count_launch(), lm_hub_mark<W><<<(unsigned)nchunks, 256, 0, s>>>(a, hubs, nhubs, chunk_pre));
}

template <typename W>
void lm_launch_commit(const LMArgs<W>& a, int64_t max_moves, cudaStream_t s) {
  if (max_moves <= 0) return;
  int blocks = (int)((max_moves + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  (count_launch(), lm_commit<W><<<blocks, 256, 0, s>>>(a));
  (count_launch(), reset_move_list<<<1, 1, 0, s>>>(a.ctr));
}

template void lm_launch_bucket<int32_t>(const LMArgs<int32_t>&, bool, bool, int, const int32_t*, int, cudaStream_t);
template void lm_launch_bucket<int64_t>(const LMArgs<int64_t>&, bool, bool, int, const int32_t*, int, cudaStream_t);
template void lm_launch_hubs<int32_t>(const LMArgs<int32_t>&, bool, bool, const int32_t*, int, const int64_t*,
                                      int64_t, const int64_t*, int64_t, cudaStream_t);
template void lm_launch_hubs<int64_t>(const LMArgs<int64_t>&, bool, bool, const int32_t*, int, const int64_t*,
                                      int64_t, const int64_t*, int64_t, cudaStream_t);
template void lm_launch_class<int32_t>(const LMArgs<int32_t>&, bool, bool, const int32_t*, const int64_t*, int,
                                       int, int64_t, cudaStream_t);
template void lm_launch_class<int64_t>(const LMArgs<int64_t>&, bool, bool, const int32_t*, const int64_t*, int,
                                       int, int64_t, cudaStream_t);
template void lm_launch_hub_mark<int32_t>(const LMArgs<int32_t>&, const int32_t*, int, const int64_t*, int64_t,
                                          cudaStream_t);
template void lm_launch_hub_mark<int64_t>(const LMArgs<int64_t>&, const int32_t*, int, const int64_t*, int64_t,
                                          cudaStream_t);
template void lm_launch_commit<int32_t>(const LMArgs<int32_t>&, int64_t, cudaStream_t);
template void lm_launch_commit<int64_t>(const LMArgs<int64_t>&, int64_t, cudaStream_t);

}  // namespace gbl
