// graph_ops.cu — everything around local-moving: scans, partitions, row
// sums, modularity, renumbering and the aggregation phase (Section 3.2 of the
// paper: each community becomes a super-vertex, edges between communities
// are merged with summed weights, edges inside one become a summed
// self-loop).  No library primitives: scan and partition are our own.
#include <type_traits>
#include "common.cuh"
#include "engine.h"

namespace gbl {

constexpr int kT = 256;          // threads of the generic kernels
constexpr int kScanTile = 2048;  // elements per scan / partition tile (8 per thread)

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Inclusive block scan of one value per thread (kT threads); returns the
// thread's inclusive prefix and the block total in *total.
__device__ __forceinline__ long long block_inclusive_scan(long long v, long long* total) {
  __shared__ long long wsum[kT / kWarp];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    long long u = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += u;
  }
  if (lane == 31) wsum[wid] = v;
  __syncthreads();
  if (wid == 0) {
    long long s = lane < kT / kWarp ? wsum[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      long long u = __shfl_up_sync(0xffffffffu, s, d);
      if (lane >= d) s += u;
    }
    if (lane < kT / kWarp) wsum[lane] = s;
  }
  __syncthreads();
  long long add = wid > 0 ? wsum[wid - 1] : 0;
  *total = wsum[kT / kWarp - 1];
  __syncthreads();
  return v + add;
}

// Sum of a u128 per thread into the block; thread 0 adds it to lo/hi.
__device__ __forceinline__ void block_add_u128(u128 v, unsigned long long* lo, unsigned long long* hi) {
  __shared__ unsigned long long slo[kT / kWarp], shi[kT / kWarp];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    unsigned long long a = __shfl_xor_sync(0xffffffffu, (unsigned long long)v, m);
    unsigned long long b = __shfl_xor_sync(0xffffffffu, (unsigned long long)(v >> 64), m);
    v += ((u128)b << 64) | (u128)a;
  }
  if (lane == 0) { slo[wid] = (unsigned long long)v; shi[wid] = (unsigned long long)(v >> 64); }
  __syncthreads();
  if (threadIdx.x == 0) {
    u128 s = 0;
    for (int w = 0; w < kT / kWarp; ++w) s += ((u128)shi[w] << 64) | (u128)slo[w];
    if (s) atomic_add_u128(lo, hi, s);
  }
  __syncthreads();
}

// ---------------------------------------------------------------- scans

template <typename Tin>
__global__ void __launch_bounds__(kT) scan_reduce_k(const Tin* __restrict__ in, int64_t n, long long* bsum) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  long long s = 0;
#pragma unroll
  for (int k = 0; k < kScanTile / kT; ++k) {
    int64_t idx = base + k * kT + threadIdx.x;
    if (idx < n) s += (long long)in[idx];
  }
  long long tot;
  block_inclusive_scan(s, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kT) scan_bsums_k(long long* bsum, int64_t nb, int64_t* total) {
  long long carry = 0;
  for (int64_t c0 = 0; c0 < nb; c0 += kT) {
    int64_t idx = c0 + threadIdx.x;
    long long v = idx < nb ? bsum[idx] : 0;
    long long tot;
    long long inc = block_inclusive_scan(v, &tot);
    if (idx < nb) bsum[idx] = carry + inc - v;
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kT) scan_final_k(const Tin* in, Tout* out, int64_t n, const long long* bsum) {
  __shared__ long long tile[kScanTile];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  constexpr int PER = kScanTile / kT;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    int64_t idx = base + k * kT + threadIdx.x;
    tile[k * kT + threadIdx.x] = idx < n ? (long long)in[idx] : 0;
  }
  __syncthreads();
  long long loc[PER], s = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) { loc[k] = s; s += tile[threadIdx.x * PER + k]; }
  long long tot;
  long long inc = block_inclusive_scan(s, &tot);
  long long ex = inc - s + bsum[blockIdx.x];
#pragma unroll
  for (int k = 0; k < PER; ++k) tile[threadIdx.x * PER + k] = ex + loc[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    int64_t idx = base + k * kT + threadIdx.x;
    if (idx < n) out[idx] = (Tout)tile[k * kT + threadIdx.x];
  }
}

// A short input (at most kScanOneTiles tiles) in one launch: one block takes
// the tiles in order, each offset by the sum of those before it (the three
// kernels above cost more in launches than in work at these sizes).
constexpr int64_t kScanOneTiles = 4;
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kT) scan_one_k(const Tin* in, Tout* out, int64_t n, int64_t* total) {
  __shared__ long long tile[kScanTile];
  constexpr int PER = kScanTile / kT;
  long long carry = 0;
  for (int64_t base = 0; base < n; base += kScanTile) {
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int64_t idx = base + k * kT + threadIdx.x;
      tile[k * kT + threadIdx.x] = idx < n ? (long long)in[idx] : 0;
    }
    __syncthreads();
    long long loc[PER], v = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) { loc[k] = v; v += tile[threadIdx.x * PER + k]; }
    long long tot;
    const long long ex = block_inclusive_scan(v, &tot) - v + carry;
#pragma unroll
    for (int k = 0; k < PER; ++k) tile[threadIdx.x * PER + k] = ex + loc[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int64_t idx = base + k * kT + threadIdx.x;
      if (idx < n) out[idx] = (Tout)tile[k * kT + threadIdx.x];
    }
    carry += tot;
    __syncthreads();   // the tile is loaded again
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

size_t scan_tmp_bytes(int64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile + 1) * sizeof(long long); }

template <typename Tin, typename Tout>
static void scan_any(const Tin* in, Tout* out, int64_t n, int64_t* total, void* tmp, cudaStream_t s) {
  if (n <= 0) {
    if (total) cudaMemsetAsync(total, 0, sizeof(int64_t), s);
    return;
  }
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb <= kScanOneTiles) {
    (count_launch(), scan_one_k<Tin, Tout><<<1, kT, 0, s>>>(in, out, n, total));
    return;
  }
  long long* bsum = (long long*)tmp;
  (count_launch(), scan_reduce_k<Tin><<<(unsigned)nb, kT, 0, s>>>(in, n, bsum));
  (count_launch(), scan_bsums_k<<<1, kT, 0, s>>>(bsum, nb, total));
  (count_launch(), scan_final_k<Tin, Tout><<<(unsigned)nb, kT, 0, s>>>(in, out, n, bsum));
}

void scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, int64_t* total, void* tmp, cudaStream_t s) {
  scan_any<int32_t, int64_t>(in, out, n, total, tmp, s);
}
void scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total, void* tmp, cudaStream_t s) {
  scan_any<int64_t, int64_t>(in, out, n, total, tmp, s);
}
void scan_i32(const int32_t* in, int32_t* out, int64_t n, int64_t* total, void* tmp, cudaStream_t s) {
  scan_any<int32_t, int32_t>(in, out, n, total, tmp, s);
}

// ------------------------------------------------------ stable partition

__global__ void __launch_bounds__(kT) part_count_k(const int32_t* __restrict__ key, int64_t n, int nkeys,
                                                   int64_t* counts, int64_t nblk) {
  extern __shared__ int hist[];
  for (int t = threadIdx.x; t < nkeys; t += kT) hist[t] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int k = 0; k < kScanTile / kT; ++k) {
    int64_t idx = base + k * kT + threadIdx.x;
    if (idx < n) atomicAdd(&hist[key[idx]], 1);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nkeys; t += kT) counts[(int64_t)t * nblk + blockIdx.x] = hist[t];
}

__global__ void part_key_off_k(const int64_t* offs, int nkeys, int64_t nblk, int64_t n, int64_t* key_off) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t <= nkeys; t += gridDim.x * blockDim.x)
    key_off[t] = t < nkeys ? offs[(int64_t)t * nblk] : n;
}

__global__ void __launch_bounds__(kT) part_scatter_k(const int32_t* __restrict__ key, int64_t n, int nkeys,
                                                     const int64_t* offs, int64_t nblk, int32_t* out) {
  extern __shared__ long long psm[];
  long long* running = psm;               // nkeys
  long long* wcnt = psm + nkeys;          // (kT / 32) * nkeys
  constexpr int NW = kT / kWarp;
  const int wid = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < nkeys; t += kT) running[t] = offs[(int64_t)t * nblk + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int r = 0; r < kScanTile / kT; ++r) {
    for (int t = threadIdx.x; t < NW * nkeys; t += kT) wcnt[t] = 0;
    __syncthreads();
    int64_t idx = base + r * kT + threadIdx.x;
    bool valid = idx < n;
    int k = valid ? key[idx] : -1;
    unsigned peers = __match_any_sync(0xffffffffu, k);
    int rank = __popc(peers & lanemask_lt());
    if (valid && rank == 0) wcnt[wid * nkeys + k] = __popc(peers);
    __syncthreads();
    for (int t = threadIdx.x; t < nkeys; t += kT) {
      long long b = running[t];
      for (int w = 0; w < NW; ++w) {
        long long c = wcnt[w * nkeys + t];
        wcnt[w * nkeys + t] = b;
        b += c;
      }
      running[t] = b;
    }
    __syncthreads();
    if (valid) out[wcnt[wid * nkeys + k] + rank] = (int32_t)idx;
    __syncthreads();
  }
}

// One tile (n <= kScanTile) in one launch: the counts, their scan over the
// keys, the key offsets and the stable scatter above, in the same order.
__global__ void __launch_bounds__(kT) part_one_k(const int32_t* __restrict__ key, int64_t n, int nkeys,
                                                 int64_t* key_off, int32_t* out) {
  extern __shared__ long long psm[];
  long long* running = psm;               // nkeys
  long long* wcnt = psm + nkeys;          // (kT / 32) * nkeys
  constexpr int NW = kT / kWarp;
  const int wid = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < nkeys; t += kT) running[t] = 0;
  __syncthreads();
  for (int64_t idx = threadIdx.x; idx < n; idx += kT) atomicAdd((unsigned long long*)&running[key[idx]], 1ull);
  __syncthreads();
  long long carry = 0;   // exclusive scan of the counts over the keys
  for (int c0 = 0; c0 < nkeys; c0 += kT) {
    const int t = c0 + threadIdx.x;
    const long long v = t < nkeys ? running[t] : 0;
    long long tot;
    const long long ex = block_inclusive_scan(v, &tot) - v + carry;
    if (t < nkeys) {
      running[t] = ex;
      key_off[t] = ex;
    }
    carry += tot;
  }
  if (threadIdx.x == 0) key_off[nkeys] = n;
  __syncthreads();
  for (int64_t base = 0; base < n; base += kT) {
    for (int t = threadIdx.x; t < NW * nkeys; t += kT) wcnt[t] = 0;
    __syncthreads();
    const int64_t idx = base + threadIdx.x;
    const bool valid = idx < n;
    const int k = valid ? key[idx] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, k);
    const int rank = __popc(peers & lanemask_lt());
    if (valid && rank == 0) wcnt[wid * nkeys + k] = __popc(peers);
    __syncthreads();
    for (int t = threadIdx.x; t < nkeys; t += kT) {
      long long b = running[t];
      for (int w = 0; w < NW; ++w) {
        const long long c = wcnt[w * nkeys + t];
        wcnt[w * nkeys + t] = b;
        b += c;
      }
      running[t] = b;
    }
    __syncthreads();
    if (valid) out[wcnt[wid * nkeys + k] + rank] = (int32_t)idx;
    __syncthreads();
  }
}

size_t partition_tmp_bytes(int64_t n, int nkeys) {
  int64_t nblk = (n + kScanTile - 1) / kScanTile;
  if (nblk < 1) nblk = 1;
  int64_t m = (int64_t)nkeys * nblk;
  return (size_t)m * 8 * 2 + scan_tmp_bytes(m) + 256;
}

void stable_partition(const int32_t* key, int64_t n, int nkeys, int32_t* out, int64_t* key_off, void* tmp,
                      cudaStream_t s) {
  int64_t nblk = (n + kScanTile - 1) / kScanTile;
  if (nblk < 1) nblk = 1;
  int64_t m = (int64_t)nkeys * nblk;
  int64_t* counts = (int64_t*)tmp;
  int64_t* offs = counts + m;
  void* stmp = (void*)(offs + m);
  if (n > 0 && n <= kScanTile) {
    const size_t smem = (size_t)nkeys * (1 + kT / kWarp) * sizeof(long long);
    (count_launch(), part_one_k<<<1, kT, smem, s>>>(key, n, nkeys, key_off, out));
    return;
  }
  if (n > 0) {
    (count_launch(), part_count_k<<<(unsigned)nblk, kT, nkeys * sizeof(int), s>>>(key, n, nkeys, counts, nblk));
    scan_i64(counts, offs, m, nullptr, stmp, s);
  } else {
    cudaMemsetAsync(offs, 0, m * sizeof(int64_t), s);
  }
  (count_launch(), part_key_off_k<<<(nkeys + 1 + 255) / 256, 256, 0, s>>>(offs, nkeys, nblk, n, key_off));
  if (n > 0) {
    size_t smem = (size_t)nkeys * (1 + kT / kWarp) * sizeof(long long);
    (count_launch(), part_scatter_k<<<(unsigned)nblk, kT, smem, s>>>(key, n, nkeys, offs, nblk, out));
  }
}

// --------------------------------------------------- local-moving lists

// With `active` (the stamps read in this iteration), vertices that are not
// active, or whose graph has stopped (g_on), get the trailing key too, so the
// lists hold only the vertices the iteration visits.
__global__ void lm_keys_k(const int64_t* __restrict__ off, int64_t n, int P, int32_t* key,
                          const int32_t* __restrict__ gid, const int64_t* __restrict__ vo,
                          const int32_t* __restrict__ gcat, ClassSpec cs, const int* __restrict__ d_iter,
                          LMThresholds th, const int32_t* __restrict__ active, const int32_t* __restrict__ g_on) {
  const int iter = *d_iter;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int b = lm_bucket_of(off[i + 1] - off[i], th);
    if (active && (active[i] != iter || (gid && !g_on[gid[i]]))) b = -1;
    key[i] = b < 0 ? kBuckets * P : b * P + (P > 1 ? vertex_class(i, gid, vo, gcat, cs, iter) : 0);
  }
}

// The same keys for the vertices of a subset (key[j] for vertex sub[j]);
// with `active`, inactive vertices and vertices of stopped graphs get the
// key past every bucket.
__global__ void lm_keys_sub_k(const int64_t* __restrict__ off, const int32_t* __restrict__ sub, int64_t m, int P,
                              int32_t* key, const int32_t* __restrict__ gid, const int64_t* __restrict__ vo,
                              const int32_t* __restrict__ gcat, ClassSpec cs, const int* __restrict__ d_iter,
                              LMThresholds th, const int32_t* __restrict__ active, const int32_t* __restrict__ g_on) {
  const int iter = *d_iter;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t i = sub[j];
    int b = lm_bucket_of(off[i + 1] - off[i], th);
    if (active && (active[i] != iter || (gid && !g_on[gid[i]]))) b = -1;
    key[j] = b < 0 ? kBuckets * P : b * P + (P > 1 ? vertex_class(i, gid, vo, gcat, cs, iter) : 0);
  }
}

__global__ void gather_ids_k(const int32_t* __restrict__ idx, const int32_t* __restrict__ sub, int64_t m,
                             int32_t* out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
    out[j] = sub[idx[j]];
}

static unsigned grid1d(int64_t n, int per = kT) {
  int64_t b = (n + per - 1) / per;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)(b < 1 ? 1 : b);
}

void lm_keys(const int64_t* off, int64_t n, int P, int32_t* key, const int32_t* gid, const int64_t* vo,
             const int32_t* gcat, ClassSpec cs, const int* d_iter, LMThresholds th, const int32_t* active,
             const int32_t* g_on, cudaStream_t s) {
  if (n > 0)
    (count_launch(), lm_keys_k<<<grid1d(n), kT, 0, s>>>(off, n, P, key, gid, vo, gcat, cs, d_iter, th, active, g_on));
}

__global__ void hub_sizes_k(const int64_t* off, const int32_t* hubs, int64_t nhubs, int64_t* cap, int64_t* chunks,
                            int64_t* schunks) {
  for (int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; h < nhubs; h += (int64_t)gridDim.x * blockDim.x) {
    int64_t d = off[hubs[h] + 1] - off[hubs[h]];
    cap[h] = 2 * d;
    chunks[h] = (d + kHubChunkEntries - 1) / kHubChunkEntries;
    schunks[h] = (2 * d + kSlotChunk - 1) / kSlotChunk;
  }
}

void hub_layout(const int64_t* off, const int32_t* hubs, int64_t nhubs, int64_t* hbase, int64_t* chunk_pre,
                int64_t* spre, void* tmp, cudaStream_t s) {
  if (nhubs <= 0) {
    cudaMemsetAsync(hbase, 0, sizeof(int64_t), s);
    cudaMemsetAsync(chunk_pre, 0, sizeof(int64_t), s);
    cudaMemsetAsync(spre, 0, sizeof(int64_t), s);
    return;
  }
  int64_t* cap = (int64_t*)tmp;
  int64_t* chunks = cap + nhubs;
  int64_t* schunks = chunks + nhubs;
  void* stmp = (void*)(schunks + nhubs);
  (count_launch(), hub_sizes_k<<<grid1d(nhubs), kT, 0, s>>>(off, hubs, nhubs, cap, chunks, schunks));
  scan_i64(cap, hbase, nhubs, hbase + nhubs, stmp, s);
  scan_i64(chunks, chunk_pre, nhubs, chunk_pre + nhubs, stmp, s);
  scan_i64(schunks, spre, nhubs, spre + nhubs, stmp, s);
}

// -------------------------------------------- row-range load balancing

__global__ void chunk_rows_k(const int64_t* __restrict__ off, int64_t n, int64_t nchunks, int32_t* crow);

// Row sums over merge-path chunks (crow from chunk_rows_k: every warp gets
// kRelabelChunk rows + entries, however skewed the rows are).  A warp walks
// its chunk's rows 32 at a time and each lane finds its entry's row by a
// shuffle search over the 32 row starts; U rounds of 32 entries are loaded
// together.  Per round a segmented scan across the warp (rows are
// non-decreasing along the lanes) leaves each row's total on its last lane,
// which adds it to K (zeroed before).  M and the self-loop total are summed
// per lane and added once per warp.  With CHECK the same pass checks the
// columns' range and the weights' sign (flags 2 and 4; an entry out of range
// is not used further) and sums the two symmetry fingerprints (they wrap
// modulo 2^64 on both sides alike).
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ unsigned long long entry_hash(uint32_t u, uint32_t v, uint32_t w) {
  return mix64((((unsigned long long)u << 32) | v) ^ mix64(0xC0FFEEull + w));
}

template <typename W, bool CHECK>
__global__ void __launch_bounds__(256) row_sums_k(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                                                 const W* __restrict__ wt, int64_t n, int64_t nnz,
                                                 const int32_t* __restrict__ crow, int64_t nchunks,
                                                 unsigned long long* K, unsigned long long* acc, int* flags,
                                                 unsigned long long* hashes) {
  constexpr int U = 4;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  u128 mtot = 0, ltot = 0;   // this lane's share of M and of the self-loop total
  unsigned long long h1 = 0, h2 = 0;
  int f = 0;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks; c += warps) {
    const int64_t X0 = c * kRelabelChunk - crow[c];
    const int64_t X1 = min(nnz, (c + 1) * kRelabelChunk - crow[c + 1]);
    for (int64_t r = crow[c];; r += kWarp) {
      const int64_t o = off[min(r + lane, n)];
      const int64_t wend = __shfl_sync(0xffffffffu, off[min(r + kWarp, n)], 0);
      const int64_t xs = max(X0, __shfl_sync(0xffffffffu, o, 0)), xe = min(X1, wend);
      for (int64_t x0 = xs; x0 < xe; x0 += U * kWarp) {
        int rr[U];
        int32_t v[U];
        unsigned long long w[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
          const int64_t x = x0 + k * kWarp + lane;
          int q = 0;
#pragma unroll
          for (int step = 16; step >= 1; step >>= 1) {
            const int cand = q + step;
            if (__shfl_sync(0xffffffffu, o, cand) <= x) q = cand;
          }
          rr[k] = x < xe ? q : -1;
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
          const int64_t x = x0 + k * kWarp + lane;
          v[k] = rr[k] >= 0 ? col[x] : -1;
          w[k] = rr[k] >= 0 ? (unsigned long long)wt[x] : 0ull;
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
          const int64_t u = r + rr[k];
          if (rr[k] >= 0) {
            mtot += w[k];
            if (v[k] == u) ltot += w[k];
            if (CHECK) {
              if (v[k] < 0 || v[k] >= n) {
                f |= 2;
              } else {
                if ((long long)(W)w[k] <= 0) f |= 4;
                h1 += entry_hash((uint32_t)u, (uint32_t)v[k], (uint32_t)w[k]);
                h2 += entry_hash((uint32_t)v[k], (uint32_t)u, (uint32_t)w[k]);
              }
            }
          }
          unsigned long long sum = w[k];
          const int row = rr[k];
#pragma unroll
          for (int d = 1; d < kWarp; d <<= 1) {
            const unsigned long long up = __shfl_up_sync(0xffffffffu, sum, d);
            const int ru = __shfl_up_sync(0xffffffffu, row, d);
            if (lane >= d && ru == row) sum += up;
          }
          const int rn = __shfl_down_sync(0xffffffffu, row, 1);
          if (row >= 0 && (lane == kWarp - 1 || rn != row)) atomicAdd(K + (r + row), sum);
        }
      }
      if (wend >= X1) break;
    }
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) {
    mtot += ((u128)__shfl_xor_sync(0xffffffffu, (unsigned long long)(mtot >> 64), m) << 64) |
            (u128)__shfl_xor_sync(0xffffffffu, (unsigned long long)mtot, m);
    ltot += ((u128)__shfl_xor_sync(0xffffffffu, (unsigned long long)(ltot >> 64), m) << 64) |
            (u128)__shfl_xor_sync(0xffffffffu, (unsigned long long)ltot, m);
    if (CHECK) {
      h1 += __shfl_xor_sync(0xffffffffu, h1, m);
      h2 += __shfl_xor_sync(0xffffffffu, h2, m);
      f |= __shfl_xor_sync(0xffffffffu, f, m);
    }
  }
  if (lane == 0) {
    if (mtot) atomic_add_u128(acc, acc + 1, mtot);
    if (ltot) atomic_add_u128(acc + 2, acc + 3, ltot);
    if (CHECK) {
      if (f) atomicOr(flags, f);
      atomicAdd(hashes, h1);
      atomicAdd(hashes + 1, h2);
    }
  }
}

template <typename W>
void row_sums(const int64_t* off, const int32_t* col, const W* wt, int64_t n, int64_t nnz, int32_t* crow,
              long long* K, unsigned long long* acc, int* flags, unsigned long long* hashes, cudaStream_t s) {
  if (n <= 0) return;
  cudaMemsetAsync(K, 0, n * sizeof(long long), s);
  if (nnz <= 0) return;
  const int64_t nchunks = (n + nnz + kRelabelChunk - 1) / kRelabelChunk;
  (count_launch(), chunk_rows_k<<<grid1d(nchunks + 1), kT, 0, s>>>(off, n, nchunks, crow));
  int64_t blocks = (nchunks + 7) / 8;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (flags)
    (count_launch(), row_sums_k<W, true><<<(unsigned)blocks, 256, 0, s>>>(off, col, wt, n, nnz, crow, nchunks,
                                                                         (unsigned long long*)K, acc, flags, hashes));
  else
    (count_launch(), row_sums_k<W, false><<<(unsigned)blocks, 256, 0, s>>>(off, col, wt, n, nnz, crow, nchunks,
                                                                          (unsigned long long*)K, acc, nullptr,
                                                                          nullptr));
}
template void row_sums<int32_t>(const int64_t*, const int32_t*, const int32_t*, int64_t, int64_t, int32_t*,
                                long long*, unsigned long long*, int*, unsigned long long*, cudaStream_t);
template void row_sums<int64_t>(const int64_t*, const int32_t*, const int64_t*, int64_t, int64_t, int32_t*,
                                long long*, unsigned long long*, int*, unsigned long long*, cudaStream_t);

__global__ void pass_init_k(int64_t n, const long long* K, int32_t* memb, long long* sig, int32_t* csize,
                            int32_t* sa, int32_t* sb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    memb[i] = (int32_t)i;
    sig[i] = K[i];
    csize[i] = 1;
    sa[i] = -1;
    sb[i] = -1;
  }
}

void pass_init(int64_t n, const long long* K, int32_t* memb, long long* sig, int32_t* csize, int32_t* stampA,
               int32_t* stampB, cudaStream_t s) {
  if (n > 0) (count_launch(), pass_init_k<<<grid1d(n), kT, 0, s>>>(n, K, memb, sig, csize, stampA, stampB));
}

// ------------------------------------------------ partition, then merge
//
// Vertex u belongs to part floor(u * parts / n); the induced subgraphs keep
// the entries whose ends share a part, in order (a stable compaction).

void lm_keys_sub(const int64_t* off, const int32_t* sub, int64_t m, int P, int32_t* key, const int32_t* gid,
                 const int64_t* vo, const int32_t* gcat, ClassSpec cs, const int* d_iter, LMThresholds th,
                 const int32_t* active, const int32_t* g_on, cudaStream_t s) {
  if (m > 0)
    (count_launch(), lm_keys_sub_k<<<grid1d(m), kT, 0, s>>>(off, sub, m, P, key, gid, vo, gcat, cs, d_iter, th, active,
                                                             g_on));
}
void gather_ids(const int32_t* idx, const int32_t* sub, int64_t m, int32_t* out, cudaStream_t s) {
  if (m > 0) (count_launch(), gather_ids_k<<<grid1d(m), kT, 0, s>>>(idx, sub, m, out));
}

__device__ __forceinline__ int64_t part_of(int64_t u, int64_t n, int64_t parts) { return (u * parts) / n; }

__global__ void induced_flags_k(const int64_t* __restrict__ off, const int32_t* __restrict__ col, int64_t n,
                                int64_t parts, int64_t* flags) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
    const int64_t pu = part_of(u, n, parts);
    for (int64_t x = off[u] + lane; x < off[u + 1]; x += 32) flags[x] = part_of(col[x], n, parts) == pu ? 1 : 0;
  }
}

__global__ void induced_scatter_k(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                                  const int32_t* __restrict__ w, int64_t n, int64_t nnz, int64_t parts,
                                  const int64_t* __restrict__ pos, const int64_t* __restrict__ total, int64_t* off_sub,
                                  int32_t* col_sub, int32_t* w_sub) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
    const int64_t pu = part_of(u, n, parts);
    if (lane == 0) off_sub[u] = off[u] < nnz ? pos[off[u]] : *total;
    for (int64_t x = off[u] + lane; x < off[u + 1]; x += 32)
      if (part_of(col[x], n, parts) == pu) {
        col_sub[pos[x]] = col[x];
        w_sub[pos[x]] = w[x];
      }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) off_sub[n] = *total;
}

void induced_parts(const int64_t* off, const int32_t* col, const int32_t* w, int64_t n, int64_t nnz, int64_t parts,
                   int64_t* flags, int64_t* pos, int64_t* total, int64_t* off_sub, int32_t* col_sub, int32_t* w_sub,
                   void* tmp, cudaStream_t s) {
  if (n <= 0) return;
  int64_t blocks = (n + 7) / 8;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (nnz > 0) {
    (count_launch(), induced_flags_k<<<(unsigned)blocks, 256, 0, s>>>(off, col, n, parts, flags));
    scan_i64(flags, pos, nnz, total, tmp, s);
  } else {
    cudaMemsetAsync(total, 0, sizeof(int64_t), s);
  }
  (count_launch(), induced_scatter_k<<<(unsigned)blocks, 256, 0, s>>>(off, col, w, n, nnz, parts, pos, total, off_sub,
                                                                       col_sub, w_sub));
}

// memb[u] += first vertex of u's part (part-local community ids to global).
__global__ void part_base_k(int32_t* memb, int64_t n, int64_t parts) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = part_of(u, n, parts);
    memb[u] += (int32_t)((p * n + parts - 1) / parts);
  }
}
void part_base(int32_t* memb, int64_t n, int64_t parts, cudaStream_t s) {
  if (n > 0) (count_launch(), part_base_k<<<grid1d(n), kT, 0, s>>>(memb, n, parts));
}

// Several graphs copied side by side from separate CSRs: part g's offsets
// are shifted by its first entry eo[g] and its columns by its first vertex
// vo[g] (vo, eo: G + 1 prefixes); off[n] = nnz.
__global__ void rebase_parts_k(int64_t* off, int32_t* col, int64_t n, int64_t nnz, const int64_t* __restrict__ vo,
                               const int64_t* __restrict__ eo, int G) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n + nnz; t += stride) {
    const bool vertex = t < n;
    const int64_t x = vertex ? t : t - n;
    const int64_t* pre = vertex ? vo : eo;
    int lo = 0, hi = G;   // the last g with pre[g] <= x
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (pre[mid] <= x) lo = mid; else hi = mid;
    }
    if (vertex) off[x] += eo[lo];
    else col[x] += (int32_t)vo[lo];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) off[n] = nnz;
}

void rebase_parts(int64_t* off, int32_t* col, int64_t n, int64_t nnz, const int64_t* vo, const int64_t* eo, int G,
                  cudaStream_t s) {
  (count_launch(), rebase_parts_k<<<grid1d(n + nnz), kT, 0, s>>>(off, col, n, nnz, vo, eo, G));
}

// Pass 0 from a given membership (already in memb): ids must lie in the
// vertex's graph's range [vo[g], vo[g + 1]) (one graph: [0, n)); a bad id
// sets *flag and is replaced by the vertex itself.  Then Sigma and sizes.
__global__ void pass_init_from_k(int64_t n, int32_t* memb, int32_t* sa, int32_t* sb, const int32_t* __restrict__ gid,
                                 const int64_t* __restrict__ vo, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lo = gid ? vo[gid[i]] : 0, hi = gid ? vo[gid[i] + 1] : n;
    const int32_t c = memb[i];
    if (c < lo || c >= hi) {
      atomicOr(flag, 1);
      memb[i] = (int32_t)i;
    }
    sa[i] = -1;
    sb[i] = -1;
  }
}
__global__ void community_sizes_k(const long long* K, const int32_t* memb, int64_t n, long long* sig, int32_t* csize) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = memb[i];
    atomicAdd((unsigned long long*)(sig + c), (unsigned long long)K[i]);
    atomicAdd(csize + c, 1);
  }
}

__global__ void check_membership_k(int64_t n, const int32_t* __restrict__ memb, const int32_t* __restrict__ gid,
                                   const int64_t* __restrict__ vo, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lo = gid ? vo[gid[i]] : 0, hi = gid ? vo[gid[i] + 1] : n;
    if (memb[i] < lo || memb[i] >= hi) atomicOr(flag, 1);
  }
}

void check_membership(int64_t n, const int32_t* memb, const int32_t* gid, const int64_t* vo, int* flag,
                      cudaStream_t s) {
  if (n > 0) (count_launch(), check_membership_k<<<grid1d(n), kT, 0, s>>>(n, memb, gid, vo, flag));
}

void pass_init_from(int64_t n, const long long* K, int32_t* memb, long long* sig, int32_t* csize, int32_t* stampA,
                    int32_t* stampB, const int32_t* gid, const int64_t* vo, int* flag, cudaStream_t s) {
  if (n <= 0) return;
  cudaMemsetAsync(sig, 0, n * sizeof(long long), s);
  cudaMemsetAsync(csize, 0, n * sizeof(int32_t), s);
  (count_launch(), pass_init_from_k<<<grid1d(n), kT, 0, s>>>(n, memb, stampA, stampB, gid, vo, flag));
  (count_launch(), community_sizes_k<<<grid1d(n), kT, 0, s>>>(K, memb, n, sig, csize));
}

// L = sum of the weights of entries whose two ends share a community, over
// merge-path chunks of rows + entries (crow from chunk_rows_k, the walk of
// row_sums_k): every warp the same work however skewed the rows are.  A lane
// loads the community of one row of the warp's 32-row window; each entry
// takes its row's by a shuffle.
template <typename W>
__global__ void __launch_bounds__(256) intra_weight_k(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                                                     const W* __restrict__ wt, int64_t n, int64_t nnz,
                                                     const int32_t* __restrict__ memb,
                                                     const int32_t* __restrict__ crow, int64_t nchunks,
                                                     unsigned long long* acc) {
  constexpr int U = 4;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  u128 L = 0;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks; c += warps) {
    const int64_t X0 = c * kRelabelChunk - crow[c];
    const int64_t X1 = min(nnz, (c + 1) * kRelabelChunk - crow[c + 1]);
    for (int64_t r = crow[c];; r += kWarp) {
      const int64_t o = off[min(r + lane, n)];
      const int32_t mr = r + lane < n ? memb[r + lane] : -1;
      const int64_t wend = __shfl_sync(0xffffffffu, off[min(r + kWarp, n)], 0);
      const int64_t xs = max(X0, __shfl_sync(0xffffffffu, o, 0)), xe = min(X1, wend);
      for (int64_t x0 = xs; x0 < xe; x0 += U * kWarp) {
        int32_t cm[U], v[U];
        unsigned long long w[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
          const int64_t x = x0 + k * kWarp + lane;
          int q = 0;
#pragma unroll
          for (int step = 16; step >= 1; step >>= 1) {
            const int cand = q + step;
            if (__shfl_sync(0xffffffffu, o, cand) <= x) q = cand;
          }
          cm[k] = __shfl_sync(0xffffffffu, mr, q);
          v[k] = x < xe ? col[x] : -1;
          w[k] = x < xe ? (unsigned long long)wt[x] : 0ull;
        }
#pragma unroll
        for (int k = 0; k < U; ++k)
          if (v[k] >= 0 && memb[v[k]] == cm[k]) L += w[k];
      }
      if (wend >= X1) break;
    }
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1)
    L += ((u128)__shfl_xor_sync(0xffffffffu, (unsigned long long)(L >> 64), m) << 64) |
         (u128)__shfl_xor_sync(0xffffffffu, (unsigned long long)L, m);
  if (lane == 0 && L) atomic_add_u128(acc, acc + 3, L);   // acc[0] lo, acc[3] hi
}

__global__ void __launch_bounds__(kT) sum_squares_k(const long long* __restrict__ sig, int64_t n,
                                                    unsigned long long* lo, unsigned long long* hi) {
  u128 ss = 0;
  for (int64_t c = blockIdx.x * (int64_t)kT + threadIdx.x; c < n; c += (int64_t)gridDim.x * kT) {
    long long v = sig[c];
    ss += (u128)((unsigned long long)v) * (u128)((unsigned long long)v);
  }
  block_add_u128(ss, lo, hi);
}

template <typename W>
void modularity_parts(const int64_t* off, const int32_t* col, const W* wt, int64_t n, int64_t nnz,
                      const int32_t* memb, const long long* sig, unsigned long long* acc, int32_t* crow,
                      cudaStream_t s) {
  if (n <= 0) return;
  if (nnz > 0) {
    const int64_t nchunks = (n + nnz + kRelabelChunk - 1) / kRelabelChunk;
    (count_launch(), chunk_rows_k<<<grid1d(nchunks + 1), kT, 0, s>>>(off, n, nchunks, crow));
    int64_t blocks = (nchunks + 7) / 8;
    if (blocks > 152 * 8) blocks = 152 * 8;
    (count_launch(), intra_weight_k<W><<<(unsigned)blocks, 256, 0, s>>>(off, col, wt, n, nnz, memb, crow, nchunks,
                                                                       acc));
  }
  (count_launch(), sum_squares_k<<<grid1d(n), kT, 0, s>>>(sig, n, acc + 1, acc + 2));
}
template void modularity_parts<int32_t>(const int64_t*, const int32_t*, const int32_t*, int64_t, int64_t,
                                        const int32_t*, const long long*, unsigned long long*, int32_t*,
                                        cudaStream_t);
template void modularity_parts<int64_t>(const int64_t*, const int32_t*, const int64_t*, int64_t, int64_t,
                                        const int32_t*, const long long*, unsigned long long*, int32_t*,
                                        cudaStream_t);

__global__ void community_totals_k(const long long* K, const int32_t* memb, int64_t n, long long* sig) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd((unsigned long long*)(sig + memb[i]), (unsigned long long)K[i]);
}
void sum_squares(const long long* v, int64_t n, unsigned long long* acc, cudaStream_t s) {
  if (n > 0) (count_launch(), sum_squares_k<<<grid1d(n), kT, 0, s>>>(v, n, acc, acc + 1));
}

void community_totals(const long long* K, const int32_t* memb, int64_t n, long long* sig, cudaStream_t s) {
  if (n <= 0) return;
  cudaMemsetAsync(sig, 0, n * sizeof(long long), s);
  (count_launch(), community_totals_k<<<grid1d(n), kT, 0, s>>>(K, memb, n, sig));
}

// ------------------------------------------------------------ renumber

__global__ void mark_used_k(const int32_t* memb, int64_t n, int32_t* used) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    used[memb[i]] = 1;
}
void mark_used(const int32_t* memb, int64_t n, int32_t* used, cudaStream_t s) {
  if (n <= 0) return;
  cudaMemsetAsync(used, 0, n * sizeof(int32_t), s);
  (count_launch(), mark_used_k<<<grid1d(n), kT, 0, s>>>(memb, n, used));
}

__global__ void apply_level_k(const int32_t* memb, const int32_t* newid, int64_t n, int32_t* level) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    level[i] = newid[memb[i]];
}
void apply_level(const int32_t* memb, const int32_t* newid, int64_t n, int32_t* level, cudaStream_t s) {
  if (n > 0) (count_launch(), apply_level_k<<<grid1d(n), kT, 0, s>>>(memb, newid, n, level));
}

// top[v] = level[top[v]]; a negative entry (a vertex whose community left
// the pass graphs with the isolated vertices, see compact_rows) stays.
__global__ void compose_top_k(int32_t* top, int64_t n0, const int32_t* level) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n0; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = top[v];
    if (t >= 0) top[v] = level[t];
  }
}
void compose_top(int32_t* top, int64_t n0, const int32_t* level, cudaStream_t s) {
  if (n0 > 0) (count_launch(), compose_top_k<<<grid1d(n0), kT, 0, s>>>(top, n0, level));
}

__global__ void coarse_degrees_k(const int32_t* used, const int32_t* newid, const long long* sig, int64_t n,
                                 long long* Knext) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
    if (used[c]) Knext[newid[c]] = sig[c];
}
void coarse_degrees(const int32_t* used, const int32_t* newid, const long long* sig, int64_t n, long long* Knext,
                    cudaStream_t s) {
  if (n > 0) (count_launch(), coarse_degrees_k<<<grid1d(n), kT, 0, s>>>(used, newid, sig, n, Knext));
}

// ------------------------------------------- isolated communities leave
//
// After pass 0 the communities of isolated vertices (empty coarse rows) are
// singletons that can never move; the later pass graphs keep only the other
// vertices, in the same order (compact ids).  isob[j] counts the isolated
// vertices before compact vertex j in the full numbering, so that full id =
// j + isob[j]; a vertex of the input whose community is isolated keeps in
// top[] -1 - (its rank among the isolated ones) until finalize_top.

__global__ void nonempty_rows_k(const int64_t* __restrict__ off, int64_t k, int32_t* __restrict__ flag) {
  for (int64_t C = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; C < k; C += (int64_t)gridDim.x * blockDim.x)
    flag[C] = off[C + 1] > off[C] ? 1 : 0;
}
void nonempty_rows(const int64_t* off, int64_t k, int32_t* flag, cudaStream_t s) {
  if (k > 0) (count_launch(), nonempty_rows_k<<<grid1d(k), kT, 0, s>>>(off, k, flag));
}

__global__ void compact_rows_k(const int64_t* __restrict__ off, const int32_t* __restrict__ flag,
                               const int32_t* __restrict__ pos, int64_t k, const long long* __restrict__ Kin,
                               const int32_t* __restrict__ gid_in, int64_t* __restrict__ off_out,
                               long long* __restrict__ K_out, int32_t* __restrict__ gid_out,
                               int32_t* __restrict__ isob) {
  for (int64_t C = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; C < k; C += (int64_t)gridDim.x * blockDim.x)
    if (flag[C]) {
      const int32_t j = pos[C];
      off_out[j] = off[C];
      K_out[j] = Kin[C];
      if (gid_in) gid_out[j] = gid_in[C];
      isob[j] = (int32_t)(C - j);
    }
}
__global__ void compact_cols_k(int32_t* __restrict__ col, int64_t nnz, const int32_t* __restrict__ pos) {
  constexpr int U = 4;   // four gathers in flight per thread
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t x0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x0 < nnz; x0 += U * stride) {
    int32_t c[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t x = x0 + u * stride;
      c[u] = x < nnz ? col[x] : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) c[u] = pos[c[u]];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t x = x0 + u * stride;
      if (x < nnz) col[x] = c[u];
    }
  }
}
__global__ void compact_top_k(int32_t* __restrict__ top, int64_t n0, const int32_t* __restrict__ flag,
                              const int32_t* __restrict__ pos) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n0; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t y = top[v];
    top[v] = flag[y] ? pos[y] : -1 - (y - pos[y]);
  }
}
void compact_rows(const int64_t* off, int64_t k, int64_t nnz, const int32_t* flag, const int32_t* pos,
                  const long long* Kin, const int32_t* gid_in, int64_t* off_out, long long* K_out, int32_t* gid_out,
                  int32_t* isob, int32_t* col, int32_t* top, int64_t n0, cudaStream_t s) {
  if (k > 0)
    (count_launch(), compact_rows_k<<<grid1d(k), kT, 0, s>>>(off, flag, pos, k, Kin, gid_in, off_out, K_out, gid_out,
                                                              isob));
  if (nnz > 0) (count_launch(), compact_cols_k<<<grid1d(nnz), kT, 0, s>>>(col, nnz, pos));
  if (n0 > 0) (count_launch(), compact_top_k<<<grid1d(n0), kT, 0, s>>>(top, n0, flag, pos));
}

// After a pass's renumbering: the isolated count before each new community.
__global__ void carry_isob_k(const int32_t* __restrict__ used, const int32_t* __restrict__ newid,
                             const int32_t* __restrict__ isob, int64_t n, int32_t* __restrict__ isob_next) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
    if (used[c]) isob_next[newid[c]] = isob[c];
}
void carry_isob(const int32_t* used, const int32_t* newid, const int32_t* isob, int64_t n, int32_t* isob_next,
                cudaStream_t s) {
  if (n > 0) (count_launch(), carry_isob_k<<<grid1d(n), kT, 0, s>>>(used, newid, isob, n, isob_next));
}

// The top membership in the full numbering: a compact community j is
// j + isob[j]; the r-th isolated community follows the compact communities
// with at most r isolated ones before them (isob is non-decreasing).
__global__ void finalize_top_k(int32_t* __restrict__ top, int64_t n0, const int32_t* __restrict__ isob, int64_t kc) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n0; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = top[v];
    if (t >= 0) {
      top[v] = t + isob[t];
    } else {
      const int32_t r = -1 - t;
      int64_t lo = 0, hi = kc;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (isob[mid] <= r) lo = mid + 1; else hi = mid;
      }
      top[v] = (int32_t)(lo + r);
    }
  }
}
__global__ void shift_vo_k(int64_t* vo, const int64_t* __restrict__ zpre, int64_t m) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < m; g += (int64_t)gridDim.x * blockDim.x)
    vo[g] += zpre[g];
}
void finalize_top(int32_t* top, int64_t n0, const int32_t* isob, int64_t kc, int64_t* vo_top, const int64_t* zpre,
                  int64_t G, cudaStream_t s) {
  if (n0 > 0) (count_launch(), finalize_top_k<<<grid1d(n0), kT, 0, s>>>(top, n0, isob, kc));
  if (vo_top) (count_launch(), shift_vo_k<<<grid1d(G + 1), kT, 0, s>>>(vo_top, zpre, G + 1));
}

// Per-graph first compact vertex: vo_c[g] = pos[vo_full[g]] (kc at the end).
__global__ void compact_vo_k(const int64_t* __restrict__ vo_full, int64_t m, const int32_t* __restrict__ pos,
                             int64_t k, int64_t kc, int64_t* __restrict__ vo_c) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < m; g += (int64_t)gridDim.x * blockDim.x)
    vo_c[g] = vo_full[g] < k ? pos[vo_full[g]] : kc;
}
void compact_vo(const int64_t* vo_full, int64_t G, const int32_t* pos, int64_t k, int64_t kc, int64_t* vo_c,
                cudaStream_t s) {
  (count_launch(), compact_vo_k<<<grid1d(G + 1), kT, 0, s>>>(vo_full, G + 1, pos, k, kc, vo_c));
}

__global__ void count_empty_rows_k(const int64_t* __restrict__ off, int64_t n, unsigned long long* out) {
  unsigned c = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    c += off[v + 1] == off[v] ? 1u : 0u;
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, (unsigned long long)c);
}
void count_empty_rows(const int64_t* off, int64_t n, unsigned long long* out, cudaStream_t s) {
  if (n > 0) (count_launch(), count_empty_rows_k<<<grid1d(n), kT, 0, s>>>(off, n, out));
}

// ------------------------------------------------------------ aggregation

// Counting sort of the vertices by community.  The lanes of a warp that hold
// the same community share one atomic (a community of a million members
// would otherwise serialise a million atomics on one address).
__global__ void count_members_k(const int32_t* level, int64_t n, int64_t* cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); i0 < n; i0 += stride) {
    const int64_t i = i0 + (threadIdx.x & 31);
    const int32_t C = i < n ? level[i] : -1;
    const unsigned grp = __match_any_sync(0xffffffffu, C);
    if (C >= 0 && (int)(threadIdx.x & 31) == __ffs(grp) - 1)
      atomicAdd((unsigned long long*)(cnt + C), (unsigned long long)__popc(grp));
  }
}
__global__ void place_members_k(const int32_t* level, int64_t n, const int64_t* cstart, int64_t* fill,
                                int32_t* members, int32_t* inv) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); i0 < n; i0 += stride) {
    const int64_t i = i0 + lane;
    const int32_t C = i < n ? level[i] : -1;
    const unsigned grp = __match_any_sync(0xffffffffu, C);
    const int leader = __ffs(grp) - 1;
    unsigned long long base = 0;
    if (C >= 0 && lane == leader) base = atomicAdd((unsigned long long*)(fill + C), (unsigned long long)__popc(grp));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (C >= 0) {
      const int64_t pos = cstart[C] + (int64_t)base + __popc(grp & ((1u << lane) - 1u));
      members[pos] = (int32_t)i;
      inv[i] = (int32_t)pos;
    }
  }
}

void agg_group_members(const int32_t* level, int64_t n, int64_t k, int64_t* cnt, int64_t* cstart, int64_t* fill,
                       int32_t* members, int32_t* inv, void* tmp, cudaStream_t s) {
  cudaMemsetAsync(cnt, 0, (k + 1) * sizeof(int64_t), s);
  cudaMemsetAsync(fill, 0, (k + 1) * sizeof(int64_t), s);
  if (n > 0) (count_launch(), count_members_k<<<grid1d(n), kT, 0, s>>>(level, n, cnt));
  scan_i64(cnt, cstart, k, cstart + k, tmp, s);
  if (n > 0) (count_launch(), place_members_k<<<grid1d(n), kT, 0, s>>>(level, n, cstart, fill, members, inv));
}

__global__ void member_degrees_k(const int64_t* off, const int32_t* members, int64_t n, int64_t* mdeg) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    int32_t u = members[p];
    mdeg[p] = off[u + 1] - off[u];
  }
}
void agg_member_prefix(const int64_t* off, const int32_t* members, int64_t n, int64_t* mdeg, int64_t* mpre,
                       void* tmp, cudaStream_t s) {
  if (n > 0) (count_launch(), member_degrees_k<<<grid1d(n), kT, 0, s>>>(off, members, n, mdeg));
  scan_i64(mdeg, mpre, n, mpre + n, tmp, s);
}

__global__ void agg_keys_k(const int64_t* cstart, const int64_t* mpre, int64_t k, int32_t* key) {
  for (int64_t C = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; C < k; C += (int64_t)gridDim.x * blockDim.x) {
    int64_t dsum = mpre[cstart[C + 1]] - mpre[cstart[C]];
    int b = agg_bucket_of(dsum);
    key[C] = b < 0 ? kAggBuckets : b;
  }
}
void agg_keys(const int64_t* cstart, const int64_t* mpre, int64_t k, int32_t* key, cudaStream_t s) {
  if (k > 0) (count_launch(), agg_keys_k<<<grid1d(k), kT, 0, s>>>(cstart, mpre, k, key));
}

// A coarse self-loop's weight is L_C: summed per graph when several graphs
// run together, else into one total.
__device__ __forceinline__ void add_self_loop(const AggArgs& a, int32_t C, unsigned long long w) {
  if (a.cgid) atomic_add_u128(a.glsum + 2 * a.cgid[C], a.glsum + 2 * a.cgid[C] + 1, (u128)w);
  else atomicAdd(a.lsum, w);
}

// The same sums held by each thread while it walks many communities (one
// atomic per thread and graph run instead of one per community: a pass of
// millions of small communities would otherwise queue millions of atomics on
// one address).  Communities are visited in increasing id order per thread,
// and a graph's communities are a contiguous id range, so a thread flushes
// when its graph changes.
struct SelfLoops {
  int g;
  unsigned long long v;
  __device__ __forceinline__ SelfLoops() : g(-1), v(0) {}
  __device__ __forceinline__ void flush(const AggArgs& a) {
    if (v) {
      if (a.cgid) atomic_add_u128(a.glsum + 2 * g, a.glsum + 2 * g + 1, (u128)v);
      else atomicAdd(a.lsum, v);
    }
    v = 0;
  }
  __device__ __forceinline__ void add(const AggArgs& a, int32_t C, unsigned long long w) {
    if (a.cgid) {
      const int gc = a.cgid[C];
      if (gc != g) { flush(a); g = gc; }
    }
    v += w;
  }
};

// Adds a warp's self-loop sums (all 32 lanes call it): one atomic per warp
// with one graph, else one per lane and graph.
__device__ __forceinline__ void selfloops_finish(const AggArgs& a, SelfLoops& sl) {
  if (a.cgid) {
    sl.flush(a);
    return;
  }
  unsigned long long v = sl.v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(a.lsum, v);
}

// ---- relabel: every CSR entry x = (u, v, w) of the pass graph is written to
// the tmp rows, which hold the communities' member rows back to back:
// position mpre[inv[u]] + (x - off[u]) gets (level[v], w).  The hash kernels
// below then read each community's entries contiguously.

// Merge-path split of the rows and entries: chunk c starts at diagonal
// c * kRelabelChunk of the sequence "row r ends after entry off[r + 1] - 1",
// i.e. at row crow[c] = the last r in [0, n] with r + off[r] <= c * kRelabelChunk
// and entry c * kRelabelChunk - crow[c]; every chunk spans at most
// kRelabelChunk rows plus entries (crow has nchunks + 1 elements).
__global__ void chunk_rows_k(const int64_t* __restrict__ off, int64_t n, int64_t nchunks, int32_t* crow) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c <= nchunks;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t D = c * kRelabelChunk;
    int64_t lo = 0, hi = n + 1;
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) >> 1;
      if (mid + off[mid] <= D) lo = mid; else hi = mid;
    }
    crow[c] = (int32_t)lo;
  }
}

// One warp per merge-path chunk.  It walks the chunk's rows 32 at a time (lane l holds row r + l's offset and destination
// shift); each lane finds the row of its entry among the 32 by a shuffle
// search, and U entries per lane are loaded and gathered before any store.
template <typename W, typename W2>
__global__ void __launch_bounds__(256) agg_relabel_k(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                                                     const W* __restrict__ wt, int64_t n, int64_t nnz,
                                                     const int32_t* __restrict__ level, const int32_t* __restrict__ inv,
                                                     const int64_t* __restrict__ mpre, const int32_t* __restrict__ crow,
                                                     int64_t nchunks, int32_t* __restrict__ tcol, W2* __restrict__ tw) {
  constexpr int U = 4;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks; c += warps) {
    const int64_t X0 = c * kRelabelChunk - crow[c];
    const int64_t X1 = min(nnz, (c + 1) * kRelabelChunk - crow[c + 1]);
    for (int64_t r = crow[c];; r += kWarp) {
      const int64_t u = r + lane;
      const int64_t o = off[min(u, n)];
      const int64_t wend = __shfl_sync(0xffffffffu, off[min(r + kWarp, n)], 0);
      const int64_t shift = u < n ? mpre[inv[u]] - o : 0;
      const int64_t xs = max(X0, __shfl_sync(0xffffffffu, o, 0)), xe = min(X1, wend);
      for (int64_t x0 = xs; x0 < xe; x0 += U * kWarp) {
        int64_t x[U], dst[U];
        int32_t v[U];
        W w[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
          x[k] = x0 + k * kWarp + lane;
          int rr = 0;
#pragma unroll
          for (int step = 16; step >= 1; step >>= 1) {
            const int cand = rr + step;
            if (__shfl_sync(0xffffffffu, o, cand) <= x[k]) rr = cand;
          }
          dst[k] = x[k] + __shfl_sync(0xffffffffu, shift, rr);
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
          v[k] = x[k] < xe ? col[x[k]] : 0;
          w[k] = x[k] < xe ? wt[x[k]] : (W)0;
        }
#pragma unroll
        for (int k = 0; k < U; ++k) v[k] = x[k] < xe ? level[v[k]] : 0;
#pragma unroll
        for (int k = 0; k < U; ++k)
          if (x[k] < xe) {
            tcol[dst[k]] = v[k];
            tw[dst[k]] = (W2)w[k];
          }
      }
      if (wend >= X1) break;
    }
  }
}

template <typename W, typename W2>
void agg_relabel(const int64_t* off, const int32_t* col, const W* wt, int64_t n, int64_t nnz, const int32_t* level,
                 const int32_t* inv, const int64_t* mpre, int32_t* crow, int32_t* tcol, W2* tw, cudaStream_t s) {
  if (n <= 0 || nnz <= 0) return;
  const int64_t nchunks = (n + nnz + kRelabelChunk - 1) / kRelabelChunk;
  (count_launch(), chunk_rows_k<<<grid1d(nchunks + 1), kT, 0, s>>>(off, n, nchunks, crow));
  int64_t blocks = (nchunks + 7) / 8;
  if (blocks > 152 * 8) blocks = 152 * 8;
  (count_launch(), agg_relabel_k<W, W2><<<(unsigned)blocks, 256, 0, s>>>(off, col, wt, n, nnz, level, inv, mpre, crow,
                                                                         nchunks, tcol, tw));
}
template void agg_relabel<int32_t, int32_t>(const int64_t*, const int32_t*, const int32_t*, int64_t, int64_t,
                                            const int32_t*, const int32_t*, const int64_t*, int32_t*, int32_t*,
                                            int32_t*, cudaStream_t);
template void agg_relabel<int32_t, int64_t>(const int64_t*, const int32_t*, const int32_t*, int64_t, int64_t,
                                            const int32_t*, const int32_t*, const int64_t*, int32_t*, int32_t*,
                                            int64_t*, cudaStream_t);
template void agg_relabel<int64_t, int64_t>(const int64_t*, const int32_t*, const int64_t*, int64_t, int64_t,
                                            const int32_t*, const int32_t*, const int64_t*, int32_t*, int32_t*,
                                            int64_t*, cudaStream_t);

// Shared-table values of the aggregation: coarse weights of 32 bits (total
// weight below 2^31) fit 32-bit sums.
template <typename W2>
using AggVal = typename std::conditional<sizeof(W2) == 4, unsigned int, unsigned long long>::type;

// Load U consecutive relabelled entries per lane (stride `stride`) of
// [t0, t1): D = kEmpty past the end.
template <typename W2, int U>
__device__ __forceinline__ void load_entries(const AggArgs& a, int64_t t0, int64_t t1, int stride, int32_t* D,
                                             unsigned long long* w) {
#pragma unroll
  for (int k = 0; k < U; ++k) {
    const int64_t t = t0 + (int64_t)k * stride;
    D[k] = t < t1 ? a.tcol[t] : kEmpty;
    w[k] = t < t1 ? (unsigned long long)((const W2*)a.tw)[t] : 0ull;
  }
}

// Communities with at most D member entries, a thread each: the entries are
// loaded into registers together, sorted by neighbour community with a
// bitonic network (static indices, no shared memory) and each run of equal
// keys summed into one coarse entry, written back over the community's tmp
// entries.
template <typename W2, int D>
__global__ void __launch_bounds__(256) agg_thread_k(AggArgs a, const int32_t* __restrict__ comms, int ncomms) {
  typedef AggVal<W2> V;
  static_assert((D & (D - 1)) == 0, "power-of-two network");
  constexpr int32_t kPast = 0x7fffffff;   // sorts after every community id
  SelfLoops sl;
  for (int ci = blockIdx.x * blockDim.x + threadIdx.x; ci < ncomms; ci += gridDim.x * blockDim.x) {
    const int32_t C = comms[ci];
    const int64_t vs = a.mpre[a.cstart[C]], ve = a.mpre[a.cstart[C + 1]];
    int32_t k[D];
    V w[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const int64_t x = vs + j;
      k[j] = x < ve ? a.tcol[x] : kPast;
      w[j] = x < ve ? (V)((const W2*)a.tw)[x] : (V)0;
    }
#pragma unroll
    for (int kk = 2; kk <= D; kk <<= 1) {
#pragma unroll
      for (int jj = kk >> 1; jj > 0; jj >>= 1) {
#pragma unroll
        for (int i = 0; i < D; ++i) {
          const int l = i ^ jj;
          if (l > i) {
            const bool up = (i & kk) == 0;
            if ((k[i] > k[l]) == up) {
              const int32_t tk = k[i]; k[i] = k[l]; k[l] = tk;
              const V tw = w[i]; w[i] = w[l]; w[l] = tw;
            }
          }
        }
      }
    }
    int cnt = 0;
    int32_t ck = k[0];
    V cs = w[0];
#pragma unroll
    for (int j = 1; j <= D; ++j) {
      const int32_t kj = j < D ? k[j] : kPast;
      if (j < D && kj == ck) {
        cs += w[j];
      } else {
        if (ck != kPast) {
          a.tcol[vs + cnt] = ck;
          ((W2*)a.tw)[vs + cnt] = (W2)cs;
          if (ck == C) sl.add(a, C, cs);
          ++cnt;
        }
        if (j < D) {
          ck = kj;
          cs = w[j];
        }
      }
    }
    a.rlen[C] = cnt;
  }
  selfloops_finish(a, sl);
}

// Communities with at most CAP / 2 member entries: a warp each, table in
// shared memory; the coarse row is written back over the community's tmp
// entries (all of them are read before the first write).
template <typename W2, int CAP>
__global__ void __launch_bounds__(256) agg_warp_k(AggArgs a, const int32_t* __restrict__ comms, int ncomms) {
  typedef AggVal<W2> V;
  constexpr int WPB = 8;
  constexpr int U = CAP / 2 / kWarp > 0 ? CAP / 2 / kWarp : 1;
  __shared__ int32_t skeys[WPB][CAP];
  __shared__ V svals[WPB][CAP];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* keys = skeys[wib];
  V* vals = svals[wib];
  for (int t = lane; t < CAP; t += kWarp) { keys[t] = kEmpty; vals[t] = 0; }
  __syncwarp();
  bool ok = true;
  SelfLoops sl;
  // the next community's id and ranges are fetched while the current one is
  // summed (lanes 0 and 1 load the two bounds)
  const int stride = gridDim.x * WPB;
  int ci = blockIdx.x * WPB + wib;
  int32_t C = ci < ncomms ? comms[ci] : 0;
  int64_t bnd = 0;
  if (ci < ncomms && lane < 2) bnd = a.mpre[a.cstart[C + lane]];
  for (; ci < ncomms; ci += stride) {
    const int64_t vs = __shfl_sync(0xffffffffu, bnd, 0), ve = __shfl_sync(0xffffffffu, bnd, 1);
    const int ci2 = ci + stride;
    const bool more = ci2 < ncomms;
    const int32_t C2 = more ? comms[ci2] : 0;
    int64_t st2 = 0;
    bool got = false;   // st2 issued (after the first entries' loads)
    for (int64_t t0 = vs + lane; t0 < ve; t0 += U * kWarp) {
      int32_t D[U];
      unsigned long long w[U];
      load_entries<W2, U>(a, t0, ve, kWarp, D, w);
      if (!got) {
        if (more && lane < 2) st2 = a.cstart[C2 + lane];
        got = true;
      }
#pragma unroll
      for (int k = 0; k < U; ++k)
        if (D[k] != kEmpty) ok &= table_add_pow2<CAP, V>(keys, vals, D[k], w[k]);
    }
    if (!got && more && lane < 2) st2 = a.cstart[C2 + lane];
    const int64_t b2 = more && lane < 2 ? a.mpre[st2] : 0;
    __syncwarp();
    int64_t base = 0;
    for (int t = lane; t < CAP; t += kWarp) {
      int32_t key = keys[t];
      bool occ = key != kEmpty;
      unsigned m = __ballot_sync(0xffffffffu, occ);
      if (occ) {
        int64_t pos = vs + base + __popc(m & lanemask_lt());
        a.tcol[pos] = key;
        ((W2*)a.tw)[pos] = (W2)vals[t];
        if (key == C) sl.add(a, C, vals[t]);
        keys[t] = kEmpty;
        vals[t] = 0;
      }
      base += __popc(m);
    }
    if (lane == 0) a.rlen[C] = base;
    __syncwarp();
    C = C2;
    bnd = b2;
  }
  selfloops_finish(a, sl);
  if (!__all_sync(0xffffffffu, ok) && lane == 0) atomicOr(a.error, kErrProbe);
}

// Communities with at most CAP / 2 member entries, a block each.  Each key
// seen for the first time appends its slot to a fill list (one shared atomic
// per warp), so writing the row costs its distinct keys, not the table's
// CAP slots; the row comes out in first-insert order.
template <typename W2, int CAP, int THREADS>
__global__ void __launch_bounds__(THREADS) agg_block_k(AggArgs a, const int32_t* __restrict__ comms, int ncomms) {
  typedef AggVal<W2> V;
  static_assert(CAP <= 65536, "slot ids fit 16 bits");
  constexpr int U = 4;
  // dynamic shared memory: values (CAP V), keys (CAP i32), fill list (CAP / 2 u16)
  extern __shared__ unsigned long long adyn[];
  V* vals = (V*)adyn;
  int32_t* keys = (int32_t*)(vals + CAP);
  uint16_t* fill = (uint16_t*)(keys + CAP);
  __shared__ int scnt;
  const int lane = threadIdx.x & 31;
  for (int t = threadIdx.x; t < CAP; t += THREADS) { keys[t] = kEmpty; vals[t] = 0; }
  if (threadIdx.x == 0) scnt = 0;
  __syncthreads();
  bool ok = true;
  SelfLoops sl;
  for (int ci = blockIdx.x; ci < ncomms; ci += gridDim.x) {
    int32_t C = comms[ci];
    const int64_t vs = a.mpre[a.cstart[C]], ve = a.mpre[a.cstart[C + 1]];
    for (int64_t r0 = vs; r0 < ve; r0 += U * THREADS) {   // same trip count for every thread
      int32_t D[U];
      unsigned long long w[U];
      load_entries<W2, U>(a, r0 + threadIdx.x, ve, THREADS, D, w);
#pragma unroll
      for (int k = 0; k < U; ++k) {
        bool fresh = false;
        int h = -1;
        if (D[k] != kEmpty) {
          h = table_add_pow2_slot<CAP, V>(keys, vals, D[k], w[k], &fresh);
          if (h < 0) ok = false;
        }
        const unsigned m = __ballot_sync(0xffffffffu, fresh);
        int base = 0;
        if (lane == 0 && m) base = atomicAdd(&scnt, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (fresh) fill[base + __popc(m & lanemask_lt())] = (uint16_t)h;
      }
    }
    __syncthreads();
    const int cnt = scnt;
    for (int j = threadIdx.x; j < cnt; j += THREADS) {
      const int h = fill[j];
      const int32_t key = keys[h];
      const V v = vals[h];
      a.tcol[vs + j] = key;
      ((W2*)a.tw)[vs + j] = (W2)v;
      if (key == C) sl.add(a, C, v);
      keys[h] = kEmpty;
      vals[h] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      a.rlen[C] = cnt;
      scnt = 0;
    }
    __syncthreads();
  }
  selfloops_finish(a, sl);
  if (!ok) atomicOr(a.error, kErrProbe);
}

// Large communities: blocks are (community, kAggChunkEntries-entry chunk)
// pairs; each sums its chunk per neighbour community in shared memory, then
// adds each distinct one to the community's global table (hashed, 2 x its
// entries slots, or direct-indexed by community id).
constexpr int kAggItemCache = 2048;   // community prefix entries a block copies to shared memory

template <typename W2>
__global__ void __launch_bounds__(256) agg_global_insert_k(AggArgs a, const int32_t* __restrict__ comms, int ncomms,
                                                           const int64_t* __restrict__ gbase,
                                                           const int64_t* __restrict__ chunk_pre) {
  typedef AggVal<W2> V;
  constexpr int CAP = 2 * (int)kAggChunkEntries;
  constexpr int U = (int)kAggChunkEntries / 256;
  // dynamic shared memory: values (CAP V), keys (CAP i32)
  extern __shared__ unsigned long long gdyn[];
  V* svals = (V*)gdyn;
  int32_t* skeys = (int32_t*)(svals + CAP);
  __shared__ int64_t s_pre[kAggItemCache + 1];
  const int h = block_item<kAggItemCache>(chunk_pre, ncomms, blockIdx.x, s_pre);
  const int32_t C = comms[h];
  const int64_t vs = a.mpre[a.cstart[C]], ve = a.mpre[a.cstart[C + 1]];
  const int64_t q = (int64_t)blockIdx.x - chunk_pre[h];
  const int64_t base = gbase[h];
  const uint32_t cap = (uint32_t)(gbase[h + 1] - base);
  for (int t = threadIdx.x; t < CAP; t += blockDim.x) { skeys[t] = kEmpty; svals[t] = 0; }
  const int64_t t0 = vs + q * kAggChunkEntries, t1 = min(ve, t0 + kAggChunkEntries);
  int32_t D[U];
  unsigned long long w[U];
  load_entries<W2, U>(a, t0 + threadIdx.x, t1, 256, D, w);
  __syncthreads();
  bool ok = true;
#pragma unroll
  for (int k = 0; k < U; ++k)
    if (D[k] != kEmpty) ok &= table_add_pow2<CAP, V>(skeys, svals, D[k], w[k]);
  __syncthreads();
  int32_t* keys = a.gkeys + base;
  unsigned long long* vals = a.gvals + base;
  const int64_t lo = a.glo[h];
  if (lo >= 0) {   // direct table: slot Dk - lo (same-value key stores may race)
    // the key is stored without reading the slot first: no load waits, so a
    // thread's slots go out back to back
    for (int t = threadIdx.x; t < CAP; t += blockDim.x) {
      const int32_t Dk = skeys[t];
      if (Dk == kEmpty) continue;
      const int64_t y = (int64_t)Dk - lo;
      if (y < 0 || y >= (int64_t)cap) { ok = false; continue; }
      keys[y] = Dk;
      atomicAdd(&vals[y], (unsigned long long)svals[t]);
    }
  } else {
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
  }
  if (!ok) atomicOr(a.error, kErrProbe);
}

// Blocks are (community, 4096-slot chunk) pairs: every occupied slot is
// appended to the community's tmp row and cleared.  A thread holds its
// kSlotChunk / 256 keys in registers; the block counts them, claims its
// positions with one atomic on the row length and writes (one round trip
// per block instead of one per warp and 256 slots).
template <typename W2>
__global__ void __launch_bounds__(256) agg_global_write_k(AggArgs a, const int32_t* __restrict__ comms, int ncomms,
                                                          const int64_t* __restrict__ gbase,
                                                          const int64_t* __restrict__ spre) {
  constexpr int J = (int)kSlotChunk / 256;
  constexpr int NW = 256 / kWarp;
  __shared__ int wsum[NW];
  __shared__ long long sbase;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __shared__ int64_t s_pre[kAggItemCache + 1];
  const int h = block_item<kAggItemCache>(spre, ncomms, blockIdx.x, s_pre);
  const int32_t C = comms[h];
  const int64_t base = gbase[h];
  const int64_t cap = gbase[h + 1] - base;
  const int64_t q = (int64_t)blockIdx.x - spre[h];
  const int64_t t0 = q * kSlotChunk, t1 = min(cap, t0 + kSlotChunk);
  int32_t D[J];
  int mine = 0;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int64_t t = t0 + j * 256 + threadIdx.x;
    D[j] = t < t1 ? a.gkeys[base + t] : kEmpty;
    mine += D[j] != kEmpty ? 1 : 0;
  }
  // exclusive prefix of the threads' counts over the block
  int incl = mine;
#pragma unroll
  for (int o = 1; o < kWarp; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == kWarp - 1) wsum[wid] = incl;
  __syncthreads();
  int before = 0, total = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    before += w < wid ? wsum[w] : 0;
    total += wsum[w];
  }
  if (threadIdx.x == 0)
    sbase = total ? (long long)atomicAdd((unsigned long long*)(a.rlen + C), (unsigned long long)total) : 0;
  __syncthreads();
  if (!mine) return;
  int64_t pos = a.mpre[a.cstart[C]] + sbase + before + (incl - mine);
#pragma unroll
  for (int j = 0; j < J; ++j) {
    if (D[j] == kEmpty) continue;
    const int64_t t = base + t0 + j * 256 + threadIdx.x;
    const unsigned long long v = a.gvals[t];
    a.tcol[pos] = D[j];
    ((W2*)a.tw)[pos] = (W2)v;
    if (D[j] == C) add_self_loop(a, C, v);
    a.gkeys[t] = kEmpty;
    a.gvals[t] = 0;
    ++pos;
  }
}

namespace {
template <typename K>
int agrid(K kernel, int threads, size_t smem, int work) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  int per = 0;
  per = blocks_per_sm(kernel, threads, smem);
  int g = sms * per;
  if (work < g) g = work;
  return g < 1 ? 1 : g;
}
}  // namespace

template <typename W, typename W2>
void agg_launch_bucket(const AggArgs& a, int bucket, const int32_t* comms, int ncomms, cudaStream_t s) {
  if (ncomms <= 0) return;
  switch (bucket) {
    case 0: {
      auto k = agg_thread_k<W2, kAggThreadEntries>;
      (count_launch(), k<<<agrid(k, 256, 0, (ncomms + 255) / 256), 256, 0, s>>>(a, comms, ncomms));
      break;
    }
    case 1: {
      auto k = agg_thread_k<W2, 32>;
      (count_launch(), k<<<agrid(k, 256, 0, (ncomms + 255) / 256), 256, 0, s>>>(a, comms, ncomms));
      break;
    }
    case 2: {
      auto k = agg_warp_k<W2, 256>;
      (count_launch(), k<<<agrid(k, 256, 0, (ncomms + 7) / 8), 256, 0, s>>>(a, comms, ncomms));
      break;
    }
    case 3: {
      constexpr int CAP = 2048;
      size_t smem = (size_t)CAP * (4 + sizeof(AggVal<W2>) + 1);
      auto k = agg_block_k<W2, CAP, 128>;
      (count_launch(), k<<<agrid(k, 128, smem, ncomms), 128, smem, s>>>(a, comms, ncomms));
      break;
    }
    case 4: {
      constexpr int CAP = 8192;
      size_t smem = (size_t)CAP * (4 + sizeof(AggVal<W2>) + 1);
      auto k = agg_block_k<W2, CAP, 256>;
      static std::atomic<unsigned long long> attr{0};
      smem_limit_once(attr, k, smem);
      (count_launch(), k<<<agrid(k, 256, smem, ncomms), 256, smem, s>>>(a, comms, ncomms));
      break;
    }
    default: break;
  }
}

template <typename W, typename W2>
void agg_launch_global(const AggArgs& a, const int32_t* comms, int ncomms, const int64_t* gbase,
                       const int64_t* chunk_pre, int64_t nchunks, const int64_t* spre, int64_t nslotchunks,
                       cudaStream_t s) {
  if (ncomms <= 0 || nchunks <= 0) return;
  const size_t smem = (size_t)(2 * kAggChunkEntries) * (4 + sizeof(AggVal<W2>));
  static std::atomic<unsigned long long> attr{0};
  smem_limit_once(attr, agg_global_insert_k<W2>, smem);
  (count_launch(), agg_global_insert_k<W2><<<(unsigned)nchunks, 256, smem, s>>>(a, comms, ncomms, gbase, chunk_pre));
  (count_launch(), agg_global_write_k<W2><<<(unsigned)nslotchunks, 256, 0, s>>>(a, comms, ncomms, gbase, spre));
}

#define AGG_INST(W, W2)                                                                                        \
  template void agg_launch_bucket<W, W2>(const AggArgs&, int, const int32_t*, int, cudaStream_t);            \
  template void agg_launch_global<W, W2>(const AggArgs&, const int32_t*, int, const int64_t*, const int64_t*, \
                                         int64_t, const int64_t*, int64_t, cudaStream_t);
AGG_INST(int32_t, int32_t)
AGG_INST(int32_t, int64_t)
AGG_INST(int64_t, int64_t)

__global__ void agg_global_sizes_k(const int64_t* cstart, const int64_t* mpre, const int32_t* comms, int64_t ncomms,
                                   int64_t k, const int32_t* cgid, const int64_t* cvo, int64_t* cap, int64_t* chunks,
                                   int64_t* schunks, int64_t* glo) {
  for (int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; h < ncomms; h += (int64_t)gridDim.x * blockDim.x) {
    int32_t C = comms[h];
    int64_t dsum = mpre[cstart[C + 1]] - mpre[cstart[C]];
    int64_t lo = 0, range = k;
    if (cgid) {
      const int g = cgid[C];
      lo = cvo[g];
      range = cvo[g + 1] - lo;
    }
    const bool direct = 2 * dsum >= range;
    cap[h] = direct ? range : 2 * dsum;
    glo[h] = direct ? lo : -1;
    chunks[h] = (dsum + kAggChunkEntries - 1) / kAggChunkEntries;
    schunks[h] = (cap[h] + kSlotChunk - 1) / kSlotChunk;
  }
}

void agg_global_layout(const int64_t* cstart, const int64_t* mpre, const int32_t* comms, int64_t ncomms, int64_t k,
                       const int32_t* cgid, const int64_t* cvo, int64_t* gbase, int64_t* chunk_pre, int64_t* spre,
                       int64_t* glo, void* tmp, cudaStream_t s) {
  if (ncomms <= 0) {
    cudaMemsetAsync(gbase, 0, sizeof(int64_t), s);
    cudaMemsetAsync(chunk_pre, 0, sizeof(int64_t), s);
    cudaMemsetAsync(spre, 0, sizeof(int64_t), s);
    return;
  }
  int64_t* cap = (int64_t*)tmp;
  int64_t* chunks = cap + ncomms;
  int64_t* schunks = chunks + ncomms;
  void* stmp = (void*)(schunks + ncomms);
  (count_launch(), agg_global_sizes_k<<<grid1d(ncomms), kT, 0, s>>>(cstart, mpre, comms, ncomms, k, cgid, cvo, cap,
                                                                       chunks, schunks, glo));
  scan_i64(cap, gbase, ncomms, gbase + ncomms, stmp, s);
  scan_i64(chunks, chunk_pre, ncomms, chunk_pre + ncomms, stmp, s);
  scan_i64(schunks, spre, ncomms, spre + ncomms, stmp, s);
}

// Copy each community's coarse row from its tmp position mpre[cstart[C]] to
// coff[C] (coff: k + 1 offsets).  Merge-path chunks of the rows and output
// entries (chunk_rows_k over coff) give every warp the same amount of work
// however skewed the rows are; within a chunk a warp walks the rows 32 at a
// time and each lane finds its entry's row by a shuffle search, as in the
// relabel kernel.
template <typename W2>
__global__ void __launch_bounds__(256) agg_compact_k(const int64_t* __restrict__ coff, int64_t k, int64_t nnz2,
                                                     const int64_t* __restrict__ cstart,
                                                     const int64_t* __restrict__ mpre, const int32_t* __restrict__ crow,
                                                     int64_t nchunks, const int32_t* __restrict__ tcol,
                                                     const W2* __restrict__ tw, int32_t* __restrict__ ocol,
                                                     W2* __restrict__ ow) {
  constexpr int U = 4;
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks; c += warps) {
    const int64_t X0 = c * kRelabelChunk - crow[c];
    const int64_t X1 = min(nnz2, (c + 1) * kRelabelChunk - crow[c + 1]);
    for (int64_t r = crow[c];; r += kWarp) {
      const int64_t C = r + lane;
      const int64_t o = coff[min(C, k)];
      const int64_t wend = __shfl_sync(0xffffffffu, coff[min(r + kWarp, k)], 0);
      const int64_t shift = C < k ? mpre[cstart[C]] - o : 0;
      const int64_t xs = max(X0, __shfl_sync(0xffffffffu, o, 0)), xe = min(X1, wend);
      for (int64_t x0 = xs; x0 < xe; x0 += U * kWarp) {
        int64_t x[U], src[U];
        int32_t cv[U];
        W2 wv[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
          x[q] = x0 + q * kWarp + lane;
          int rr = 0;
#pragma unroll
          for (int step = 16; step >= 1; step >>= 1) {
            const int cand = rr + step;
            if (__shfl_sync(0xffffffffu, o, cand) <= x[q]) rr = cand;
          }
          src[q] = x[q] + __shfl_sync(0xffffffffu, shift, rr);
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
          cv[q] = x[q] < xe ? tcol[src[q]] : 0;
          wv[q] = x[q] < xe ? tw[src[q]] : (W2)0;
        }
#pragma unroll
        for (int q = 0; q < U; ++q)
          if (x[q] < xe) {
            ocol[x[q]] = cv[q];
            ow[x[q]] = wv[q];
          }
      }
      if (wend >= X1) break;
    }
  }
}

template <typename W2>
void agg_compact(const int64_t* cstart, const int64_t* mpre, const int64_t* coff, int64_t k, int64_t nnz2,
                 int32_t* crow, const int32_t* tcol, const W2* tw, int32_t* ocol, W2* ow, cudaStream_t s) {
  if (k <= 0 || nnz2 <= 0) return;
  const int64_t nchunks = (k + nnz2 + kRelabelChunk - 1) / kRelabelChunk;
  (count_launch(), chunk_rows_k<<<grid1d(nchunks + 1), kT, 0, s>>>(coff, k, nchunks, crow));
  int64_t blocks = (nchunks + 7) / 8;
  if (blocks > 152 * 8) blocks = 152 * 8;
  (count_launch(), agg_compact_k<W2><<<(unsigned)blocks, 256, 0, s>>>(coff, k, nnz2, cstart, mpre, crow, nchunks, tcol,
                                                                       tw, ocol, ow));
}
template void agg_compact<int32_t>(const int64_t*, const int64_t*, const int64_t*, int64_t, int64_t, int32_t*,
                                   const int32_t*, const int32_t*, int32_t*, int32_t*, cudaStream_t);
template void agg_compact<int64_t>(const int64_t*, const int64_t*, const int64_t*, int64_t, int64_t, int32_t*,
                                   const int32_t*, const int64_t*, int32_t*, int64_t*, cudaStream_t);

// ----------------------------------------------------------- several graphs
//
// Vertices of one graph are contiguous, so the kT rows (or communities) of a
// block span a contiguous range of graph ids: sums are gathered per graph in
// shared memory (slot = graph - first graph of the block) and flushed with
// one atomic per graph and block.

__device__ __forceinline__ void flush_graph_sums(const unsigned long long* lo, const unsigned long long* hi, int g0,
                                                 int ng, unsigned long long* out /* 2 per graph */) {
  for (int t = threadIdx.x; t < ng; t += blockDim.x) {
    u128 v = ((u128)hi[t] << 64) | (u128)lo[t];
    if (v) atomic_add_u128(out + 2 * (g0 + t), out + 2 * (g0 + t) + 1, v);
  }
}

// M of every graph: Mg[g] (lo, hi) += K[u] for u in g.
__global__ void __launch_bounds__(kT) graph_totals_k(const long long* __restrict__ K, const int32_t* __restrict__ gid,
                                                     int64_t n, unsigned long long* Mg) {
  __shared__ unsigned long long lo[kT], hi[kT];
  const int64_t v0 = (int64_t)blockIdx.x * kT;
  if (v0 >= n) return;
  const int64_t v1 = min(n, v0 + kT);
  const int g0 = gid[v0], ng = gid[v1 - 1] - g0 + 1;
  lo[threadIdx.x] = 0;
  hi[threadIdx.x] = 0;
  __syncthreads();
  const int64_t u = v0 + threadIdx.x;
  if (u < n) atomic_add_u128(&lo[gid[u] - g0], &hi[gid[u] - g0], (u128)(unsigned long long)K[u]);
  __syncthreads();
  flush_graph_sums(lo, hi, g0, ng, Mg);
}

void graph_totals(const long long* K, const int32_t* gid, int64_t n, unsigned long long* Mg, cudaStream_t s) {
  if (n > 0) (count_launch(), graph_totals_k<<<(unsigned)((n + kT - 1) / kT), kT, 0, s>>>(K, gid, n, Mg));
}

// Per-graph modularity parts: L_g (lo, hi) over intra-community entries of
// the graph's rows (merge-path chunks as in intra_weight_k; a lane's entries
// come in increasing row order, so it sums a run of one graph in registers
// and adds it when the graph changes) and SS_g (lo, hi) over its
// communities' Sigma^2.
template <typename W>
__global__ void __launch_bounds__(256) graph_intra_k(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                                                    const W* __restrict__ wt, int64_t n, int64_t nnz,
                                                    const int32_t* __restrict__ memb, const int32_t* __restrict__ gid,
                                                    const int32_t* __restrict__ crow, int64_t nchunks,
                                                    unsigned long long* Lg) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  int g = -1;
  u128 L = 0;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks; c += warps) {
    const int64_t X0 = c * kRelabelChunk - crow[c];
    const int64_t X1 = min(nnz, (c + 1) * kRelabelChunk - crow[c + 1]);
    for (int64_t r = crow[c];; r += kWarp) {
      const int64_t o = off[min(r + lane, n)];
      const int32_t mr = r + lane < n ? memb[r + lane] : -1;
      const int32_t gr = r + lane < n ? gid[r + lane] : -1;
      const int64_t wend = __shfl_sync(0xffffffffu, off[min(r + kWarp, n)], 0);
      const int64_t xs = max(X0, __shfl_sync(0xffffffffu, o, 0)), xe = min(X1, wend);
      for (int64_t x = xs + lane; x - lane < xe; x += kWarp) {
        int q = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
          const int cand = q + step;
          if (__shfl_sync(0xffffffffu, o, cand) <= x) q = cand;
        }
        const int32_t cm = __shfl_sync(0xffffffffu, mr, q), cg = __shfl_sync(0xffffffffu, gr, q);
        if (x < xe && memb[col[x]] == cm) {
          if (cg != g) {
            if (L) atomic_add_u128(Lg + 2 * g, Lg + 2 * g + 1, L);
            g = cg;
            L = 0;
          }
          L += (unsigned long long)wt[x];
        }
      }
      if (wend >= X1) break;
    }
  }
  if (L) atomic_add_u128(Lg + 2 * g, Lg + 2 * g + 1, L);
}

__global__ void __launch_bounds__(kT) graph_squares_k(const long long* __restrict__ sig, const int32_t* __restrict__ gid,
                                                      int64_t n, unsigned long long* SSg) {
  __shared__ unsigned long long lo[kT], hi[kT];
  const int64_t c0 = (int64_t)blockIdx.x * kT;
  if (c0 >= n) return;
  const int64_t c1 = min(n, c0 + kT);
  const int g0 = gid[c0], ng = gid[c1 - 1] - g0 + 1;
  lo[threadIdx.x] = 0;
  hi[threadIdx.x] = 0;
  __syncthreads();
  const int64_t c = c0 + threadIdx.x;
  if (c < n && sig[c]) {
    const unsigned long long v = (unsigned long long)sig[c];
    atomic_add_u128(&lo[gid[c] - g0], &hi[gid[c] - g0], (u128)v * (u128)v);
  }
  __syncthreads();
  flush_graph_sums(lo, hi, g0, ng, SSg);
}

template <typename W>
void graph_modularity_parts(const int64_t* off, const int32_t* col, const W* wt, int64_t n, int64_t nnz,
                            const int32_t* memb, const long long* sig, const int32_t* gid, unsigned long long* Lg,
                            unsigned long long* SSg, int32_t* crow, cudaStream_t s) {
  if (n <= 0) return;
  if (nnz > 0) {
    const int64_t nchunks = (n + nnz + kRelabelChunk - 1) / kRelabelChunk;
    (count_launch(), chunk_rows_k<<<grid1d(nchunks + 1), kT, 0, s>>>(off, n, nchunks, crow));
    int64_t blocks = (nchunks + 7) / 8;
    if (blocks > 152 * 8) blocks = 152 * 8;
    (count_launch(), graph_intra_k<W><<<(unsigned)blocks, 256, 0, s>>>(off, col, wt, n, nnz, memb, gid, crow, nchunks,
                                                                      Lg));
  }
  const unsigned nb = (unsigned)((n + kT - 1) / kT);
  (count_launch(), graph_squares_k<<<nb, kT, 0, s>>>(sig, gid, n, SSg));
}
template void graph_modularity_parts<int32_t>(const int64_t*, const int32_t*, const int32_t*, int64_t, int64_t,
                                              const int32_t*, const long long*, const int32_t*, unsigned long long*,
                                              unsigned long long*, int32_t*, cudaStream_t);
template void graph_modularity_parts<int64_t>(const int64_t*, const int32_t*, const int64_t*, int64_t, int64_t,
                                              const int32_t*, const long long*, const int32_t*, unsigned long long*,
                                              unsigned long long*, int32_t*, cudaStream_t);

void graph_squares(const long long* sig, const int32_t* gid, int64_t n, unsigned long long* SSg, cudaStream_t s) {
  if (n > 0) (count_launch(), graph_squares_k<<<(unsigned)((n + kT - 1) / kT), kT, 0, s>>>(sig, gid, n, SSg));
}

// After renumbering: communities per graph (kcount[g] += used[c]) and the
// graph of every coarse vertex (gid_next[newid[c]] = gid[c]).
__global__ void graph_renumber_k(const int32_t* __restrict__ used, const int32_t* __restrict__ newid,
                                 const int32_t* __restrict__ gid, int64_t n, int64_t* kcount, int32_t* gid_next) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
    if (used[c]) {
      atomicAdd((unsigned long long*)(kcount + gid[c]), 1ull);
      gid_next[newid[c]] = gid[c];
    }
}
void graph_renumber(const int32_t* used, const int32_t* newid, const int32_t* gid, int64_t n, int64_t* kcount,
                    int32_t* gid_next, cudaStream_t s) {
  if (n > 0) (count_launch(), graph_renumber_k<<<grid1d(n), kT, 0, s>>>(used, newid, gid, n, kcount, gid_next));
}

// Final memberships as ids local to each graph.
__global__ void localize_k(const int32_t* __restrict__ top, const int32_t* __restrict__ gid0,
                           const int64_t* __restrict__ vo, int64_t n0, int32_t* out) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n0; v += (int64_t)gridDim.x * blockDim.x)
    out[v] = (int32_t)(top[v] - vo[gid0[v]]);
}
void localize_membership(const int32_t* top, const int32_t* gid0, const int64_t* vo, int64_t n0, int32_t* out,
                         cudaStream_t s) {
  if (n0 > 0) (count_launch(), localize_k<<<grid1d(n0), kT, 0, s>>>(top, gid0, vo, n0, out));
}

// Graph of every input vertex from the graph vertex offsets, and a check that
// no entry leaves its row's graph (flags |= 8).
__global__ void graph_ids_k(const int64_t* __restrict__ vo, int G, int64_t n, int32_t* gid) {
  for (int g = blockIdx.x; g < G; g += gridDim.x)
    for (int64_t v = vo[g] + threadIdx.x; v < vo[g + 1]; v += blockDim.x) gid[v] = g;
}
__global__ void __launch_bounds__(256) graph_check_k(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                                                    const int32_t* __restrict__ gid, int64_t n, int64_t nnz,
                                                    const int32_t* __restrict__ crow, int64_t nchunks, int* flags) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  int f = 0;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks; c += warps) {
    const int64_t X0 = c * kRelabelChunk - crow[c];
    const int64_t X1 = min(nnz, (c + 1) * kRelabelChunk - crow[c + 1]);
    for (int64_t r = crow[c];; r += kWarp) {
      const int64_t o = off[min(r + lane, n)];
      const int32_t gr = r + lane < n ? gid[r + lane] : -1;
      const int64_t wend = __shfl_sync(0xffffffffu, off[min(r + kWarp, n)], 0);
      const int64_t xs = max(X0, __shfl_sync(0xffffffffu, o, 0)), xe = min(X1, wend);
      for (int64_t x = xs + lane; x - lane < xe; x += kWarp) {
        int q = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
          const int cand = q + step;
          if (__shfl_sync(0xffffffffu, o, cand) <= x) q = cand;
        }
        const int32_t cg = __shfl_sync(0xffffffffu, gr, q);
        if (x < xe) {
          const int32_t v = col[x];
          if (v < 0 || v >= n || gid[v] != cg) f = 8;
        }
      }
      if (wend >= X1) break;
    }
  }
  if (f) atomicOr(flags, f);
}
void graph_ids(const int64_t* vo, int G, int64_t n, int64_t nnz, int32_t* gid, const int64_t* off, const int32_t* col,
               int32_t* crow, int* flags, cudaStream_t s) {
  if (G <= 0 || n <= 0) return;
  (count_launch(), graph_ids_k<<<G < 65535 ? G : 65535, 256, 0, s>>>(vo, G, n, gid));
  if (nnz <= 0) return;
  const int64_t nchunks = (n + nnz + kRelabelChunk - 1) / kRelabelChunk;
  (count_launch(), chunk_rows_k<<<grid1d(nchunks + 1), kT, 0, s>>>(off, n, nchunks, crow));
  int64_t blocks = (nchunks + 7) / 8;
  if (blocks > 152 * 8) blocks = 152 * 8;
  (count_launch(), graph_check_k<<<(unsigned)blocks, 256, 0, s>>>(off, col, gid, n, nnz, crow, nchunks, flags));
}

// Entries of every graph of a batch: off[vo[q + 1]] - off[vo[q]].
__global__ void graph_entries_k(const int64_t* __restrict__ off, const int64_t* __restrict__ vo, int64_t G,
                                int64_t* __restrict__ out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < G) out[q] = off[vo[q + 1]] - off[vo[q]];
}
void graph_entries(const int64_t* off, const int64_t* vo, int64_t G, int64_t* out, cudaStream_t s) {
  if (G > 0) (count_launch(), graph_entries_k<<<(unsigned)((G + kT - 1) / kT), kT, 0, s>>>(off, vo, G, out));
}

// ------------------------------------------------------ colour classes
//
// A capped greedy colouring of the pass graph (the class schedule of the
// colour_classes option): a vertex's priority is hash32(local id ^ salt)
// (lowbias32), salt = 0x9E3779B9 * (pass + 1); a vertex precedes its
// neighbour when its priority is higher (ties: the lower id).  In priority
// order each vertex takes the smallest class in 0..62 that no preceding
// neighbour holds, else 63 - computed in rounds: a vertex whose preceding
// neighbours all have their class takes its own (Jones-Plassmann order), then
// counts itself off its succeeding neighbours.  Every edge is read twice.
// Edges never join two graphs of a batch, so global ids order ties as local
// ones do.

__device__ __forceinline__ uint32_t colour_pri(int64_t v, const int32_t* gid, const int64_t* vo, const int32_t* isob,
                                               const int64_t* zpre, uint32_t salt) {
  int64_t local = gid ? v - vo[gid[v]] : v;
  if (isob) local += isob[v] - (gid ? zpre[gid[v]] : 0);   // the full numbering's id
  return hash32((uint32_t)local ^ salt);
}

// Frontier lists of the colouring: a vertex of degree above kColourHubDeg
// (a hub) goes to the hub frontier, whose rows are split over many blocks.
constexpr int64_t kColourHubDeg = kColourHubDegree;
constexpr int64_t kColourChunk = 4096;   // entries of a hub row per block item
constexpr int kColourHubBlocks = 152 * 4;

__device__ __forceinline__ void colour_push(const int64_t* __restrict__ off, int32_t u, int32_t* front,
                                            unsigned long long* nfront, int32_t* hfront,
                                            unsigned long long* nhfront) {
  if (off[u + 1] - off[u] > kColourHubDeg) hfront[atomicAdd(nhfront, 1ull)] = u;
  else front[atomicAdd(nfront, 1ull)] = u;
}

// Warp per vertex: cnt[v] = its preceding neighbours; those with none start.
__global__ void colour_init_k(const int64_t* __restrict__ off, const int32_t* __restrict__ col, int64_t n,
                              const int32_t* __restrict__ gid, const int64_t* __restrict__ vo,
                              const int32_t* __restrict__ isob, const int64_t* __restrict__ zpre, uint32_t salt,
                              int32_t* __restrict__ cnt, int32_t* __restrict__ cls, int32_t* __restrict__ front,
                              unsigned long long* __restrict__ nfront, int32_t* __restrict__ hfront,
                              unsigned long long* __restrict__ nhfront) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t ws = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = w0; v < n; v += ws) {   // uniform across the warp
    const uint32_t pv = colour_pri(v, gid, vo, isob, zpre, salt);
    unsigned c = 0;
    for (int64_t x = off[v] + lane; x < off[v + 1]; x += kWarp) {
      const int32_t u = col[x];
      if (u == v) continue;
      const uint32_t pu = colour_pri(u, gid, vo, isob, zpre, salt);
      if (pu > pv || (pu == pv && u < v)) ++c;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) {
      cnt[v] = (int32_t)c;
      cls[v] = -1;
      if (c == 0) colour_push(off, (int32_t)v, front, nfront, hfront, nhfront);
    }
  }
}

// One Jones-Plassmann round.  Blocks below gridDim.x - kColourHubBlocks:
// a warp per frontier vertex takes its class from its preceding neighbours'
// classes, then counts itself off its succeeding neighbours; those left with
// no predecessor form the next frontier (hubs apart).  The last
// kColourHubBlocks blocks do the same for the hub frontier with each hub row
// split into kColourChunk-entry items: an item ORs its preceding neighbours'
// classes into the hub's mask (hmask) and counts itself off its succeeding
// neighbours; the block that finishes a hub's last item (hdone, after a
// fence) takes the class from the complete mask and clears the mask and
// counter for the next round.  No block waits for another.  Frontier
// vertices are never neighbours, so the items of one round are independent.
// A class outside 0..63 (a preceding neighbour without one) sets flags bit 1
// and is not used.
__global__ void colour_round_k(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                               const int32_t* __restrict__ gid, const int64_t* __restrict__ vo,
                               const int32_t* __restrict__ isob, const int64_t* __restrict__ zpre, uint32_t salt,
                               const int32_t* __restrict__ front, const unsigned long long* __restrict__ nfront,
                               const int32_t* __restrict__ hfront, const unsigned long long* __restrict__ nhfront,
                               int32_t* __restrict__ cnt, int32_t* __restrict__ cls, int32_t* __restrict__ next,
                               unsigned long long* __restrict__ nnext, int32_t* __restrict__ hnext,
                               unsigned long long* __restrict__ nhnext, unsigned long long* __restrict__ total,
                               unsigned long long* __restrict__ hmask, int32_t* __restrict__ hdone,
                               int* __restrict__ flags) {
  const int lane = threadIdx.x & 31;
  const int64_t nf = (int64_t)*nfront, nh = (int64_t)*nhfront;
  if (blockIdx.x == 0 && threadIdx.x == 0) *total += (unsigned long long)(nf + nh);
  const int64_t wblocks = (int64_t)gridDim.x - kColourHubBlocks;
  if ((int64_t)blockIdx.x < wblocks) {
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t ws = (wblocks * blockDim.x) >> 5;
    for (int64_t t = w0; t < nf; t += ws) {   // uniform across the warp
      const int32_t v = front[t];
      const uint32_t pv = colour_pri(v, gid, vo, isob, zpre, salt);
      unsigned long long used = 0;
      bool bad = false;
      for (int64_t x = off[v] + lane; x < off[v + 1]; x += kWarp) {
        const int32_t u = col[x];
        if (u == v) continue;
        const uint32_t pu = colour_pri(u, gid, vo, isob, zpre, salt);
        if (pu > pv || (pu == pv && u < v)) {
          const int32_t cu = cls[u];
          if (cu >= 0 && cu < 64) used |= 1ull << cu;
          else bad = true;
        }
      }
      const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)used);
      const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(used >> 32));
      const unsigned long long free_cls = ~(((unsigned long long)hi << 32) | lo) & 0x7fffffffffffffffull;
      if (lane == 0) cls[v] = free_cls ? __ffsll((long long)free_cls) - 1 : 63;
      if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flags, 2);
      for (int64_t x = off[v] + lane; x < off[v + 1]; x += kWarp) {
        const int32_t u = col[x];
        if (u == v) continue;
        const uint32_t pu = colour_pri(u, gid, vo, isob, zpre, salt);
        if (pv > pu || (pv == pu && v < u))
          if (atomicSub(cnt + u, 1) == 1) colour_push(off, u, next, nnext, hnext, nhnext);
      }
    }
    return;
  }
  // hub items: (hub slot, chunk) in hub-frontier order
  __shared__ unsigned long long s_mask[8];
  __shared__ int s_bad;
  const int64_t hb = (int64_t)blockIdx.x - wblocks;
  int64_t h = 0, h_first = 0;   // hub slot h owns items [h_first, h_first + chunks(h))
  for (int64_t item = hb;; item += kColourHubBlocks) {
    int64_t nc = 0;
    while (h < nh) {
      const int32_t v = hfront[h];
      nc = (off[v + 1] - off[v] + kColourChunk - 1) / kColourChunk;
      if (item < h_first + nc) break;
      h_first += nc;
      ++h;
    }
    if (h >= nh) break;   // uniform across the block
    const int32_t v = hfront[h];
    const uint32_t pv = colour_pri(v, gid, vo, isob, zpre, salt);
    const int64_t x0 = off[v] + (item - h_first) * kColourChunk, x1 = min(off[v + 1], x0 + kColourChunk);
    unsigned long long used = 0;
    bool bad = false;
    for (int64_t x = x0 + threadIdx.x; x < x1; x += blockDim.x) {
      const int32_t u = col[x];
      if (u == v) continue;
      const uint32_t pu = colour_pri(u, gid, vo, isob, zpre, salt);
      if (pu > pv || (pu == pv && u < v)) {
        const int32_t cu = cls[u];
        if (cu >= 0 && cu < 64) used |= 1ull << cu;
        else bad = true;
      } else if (atomicSub(cnt + u, 1) == 1) {
        colour_push(off, u, next, nnext, hnext, nhnext);
      }
    }
    const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)used);
    const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(used >> 32));
    const bool wbad = __any_sync(0xffffffffu, bad);
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    if (lane == 0) {
      s_mask[threadIdx.x >> 5] = ((unsigned long long)hi << 32) | lo;
      if (wbad) s_bad = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long m = 0;
      for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m |= s_mask[k];
      if (s_bad) atomicOr(flags, 2);
      if (m) atomicOr(hmask + h, m);
      __threadfence();
      if (atomicAdd(hdone + h, 1) == (int)nc - 1) {   // this hub's last item: its mask is complete
        __threadfence();
        const unsigned long long full = atomicOr(hmask + h, 0ull);
        const unsigned long long free_cls = ~full & 0x7fffffffffffffffull;
        cls[v] = free_cls ? __ffsll((long long)free_cls) - 1 : 63;
        hmask[h] = 0;
        hdone[h] = 0;
      }
    }
    __syncthreads();   // s_mask and s_bad are reused by the next item
  }
}

__global__ void class_max_k(const int32_t* __restrict__ cls, int64_t n, int* __restrict__ out) {
  int m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, cls[i]);
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

static unsigned warp_grid(int64_t items) {
  const int64_t b = (items + 7) / 8;   // 8 warps per block of 256
  return (unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

void colour_init(const int64_t* off, const int32_t* col, int64_t n, const int32_t* gid, const int64_t* vo,
                 const int32_t* isob, const int64_t* zpre, uint32_t salt, int32_t* cnt, int32_t* cls, int32_t* front,
                 unsigned long long* nfront, int32_t* hfront, unsigned long long* nhfront, cudaStream_t s) {
  if (n > 0) (count_launch(), colour_init_k<<<warp_grid(n), 256, 0, s>>>(off, col, n, gid, vo, isob, zpre, salt, cnt,
                                                                         cls, front, nfront, hfront, nhfront));
}
void colour_round(const int64_t* off, const int32_t* col, int64_t n, const int32_t* gid, const int64_t* vo,
                  const int32_t* isob, const int64_t* zpre, uint32_t salt, const int32_t* front,
                  const unsigned long long* nfront, const int32_t* hfront,
                  const unsigned long long* nhfront, int32_t* cnt, int32_t* cls, int32_t* next,
                  unsigned long long* nnext, int32_t* hnext, unsigned long long* nhnext, unsigned long long* total,
                  unsigned long long* hmask, int32_t* hdone, int* flags, cudaStream_t s) {
  (count_launch(), colour_round_k<<<warp_grid(n) + kColourHubBlocks, 256, 0, s>>>(
                       off, col, gid, vo, isob, zpre, salt, front, nfront, hfront, nhfront, cnt, cls, next, nnext,
                       hnext, nhnext, total, hmask, hdone, flags));
}
void class_max(const int32_t* cls, int64_t n, int* out, cudaStream_t s) {
  if (n > 0) (count_launch(), class_max_k<<<grid1d(n), kT, 0, s>>>(cls, n, out));
}

// -------------------------------------------------------------- validation

__global__ void validate_off_k(const int64_t* off, int64_t n, int64_t nnz, int* flags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (off[i] > off[i + 1]) atomicOr(flags, 1);
  if (blockIdx.x == 0 && threadIdx.x == 0 && (off[0] != 0 || off[n] != nnz)) atomicOr(flags, 1);
}

// Offsets monotone with the right ends (flag 1); the entries are checked by
// row_sums with its check on, which needs monotone offsets for its chunks.
void validate_offsets(const int64_t* off, int64_t n, int64_t nnz, int* flags, cudaStream_t s) {
  cudaMemsetAsync(flags, 0, sizeof(int), s);
  if (n <= 0) return;
  (count_launch(), validate_off_k<<<grid1d(n), kT, 0, s>>>(off, n, nnz, flags));
}

// ------------------------------------------------------------ conversions

__global__ void widen_k(const int32_t* in, int64_t* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}
void widen_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  if (n > 0) (count_launch(), widen_k<<<grid1d(n), kT, 0, s>>>(in, out, n));
}
__global__ void fill_k(int32_t* p, int32_t v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}
void fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t s) {
  if (n > 0) (count_launch(), fill_k<<<grid1d(n), kT, 0, s>>>(p, v, n));
}
__global__ void iota_k(int32_t* p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (int32_t)i;
}
void iota_i32(int32_t* p, int64_t n, cudaStream_t s) {
  if (n > 0) (count_launch(), iota_k<<<grid1d(n), kT, 0, s>>>(p, n));
}

}  // namespace gbl
