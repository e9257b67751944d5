// noalloc.cu — exact modularity of a membership with no device allocation.
//
// Some callers cannot allocate device memory: an application whose allocator
// (PyTorch's caching allocator, for one) already owns the free memory and
// gives none back, a service that plans its whole memory budget up front and
// forbids allocations once it runs, or a pipeline that cannot afford the
// device-wide synchronisation a cudaMalloc or cudaFree implies while other
// streams are busy.  For them louvain_modularity_static computes what
// louvain_modularity computes, with its scratch (vertex degrees, community
// totals, sums) in the file-scope array below instead of context memory.
// The paper has no counterpart to this entry point.
//
// The array is part of the library image: every GPU that loads the library
// holds kStaticScratchBytes of it until the process exits.  Host code cannot
// use the array's name as a device address (in host code it names a
// host-side stand-in), so the first call on each device looks up the array's
// device address with cudaGetSymbolAddress, with that device current, and
// keeps it; that first call should come before any stream capture.  Every
// call shares the one array and leaves its contents behind: each call clears
// what must start at zero, and calls whose work overlaps on the GPU (on
// different streams, or from different threads) race on it.
#include <mutex>
#include "common.cuh"
#include "../../include/louvain.h"

namespace gbl {
namespace {

constexpr int64_t kMaxV = LOUVAIN_STATIC_MAX_VERTICES;
constexpr size_t kAccWords = 8;                              // M, L, sum Sigma^2 (lo/hi each), flags
constexpr size_t kStaticScratchBytes = 256 + 2 * sizeof(long long) * (size_t)kMaxV;

// [0, 256): accumulators; [256, 256 + 8 kMaxV): degrees K; then totals Sigma.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LOUVAIN_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return LOUVAIN_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return 0;
}

// One warp per row: K[u] = row sum; M += K[u].  A row whose offsets are
// negative or decreasing sets a flag and is not read.
template <typename W>
__global__ void static_row_sums_k(const int64_t* __restrict__ off, const W* __restrict__ wt, int64_t n,
                                  long long* K, unsigned long long* acc) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < n; u += warps) {
    const int64_t x0 = off[u], x1 = off[u + 1];
    if (x0 < 0 || x1 < x0) {   // not a CSR: flag it, read nothing of the row
      if (lane == 0) atomicOr(&acc[6], 2ull);
      continue;
    }
    unsigned long long s = 0;
    for (int64_t x = x0 + lane; x < x1; x += 32) s += (unsigned long long)wt[x];
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    if (lane == 0) {
      K[u] = (long long)s;
      atomic_add_u128(&acc[0], &acc[1], (u128)s);
    }
  }
}

// Sigma[memb[u]] += K[u]; a membership outside [0, n) sets the flag.
__global__ void static_totals_k(const long long* K, const int32_t* __restrict__ memb, int64_t n, long long* sig,
                                unsigned long long* acc) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = memb[u];
    if (c < 0 || c >= n) { atomicOr(&acc[6], 1ull); continue; }
    atomicAdd((unsigned long long*)(sig + c), (unsigned long long)K[u]);
  }
}

// L += weights of entries whose ends share a community (one warp per row);
// a column outside [0, n) sets a flag instead.
template <typename W>
__global__ void static_intra_k(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                               const W* __restrict__ wt, int64_t n, const int32_t* __restrict__ memb,
                               unsigned long long* acc) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned long long L = 0;
  for (int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < n; u += warps) {
    const int32_t cu = memb[u];
    const int64_t x0 = off[u], x1 = off[u + 1];
    if (x0 < 0 || x1 < x0) continue;   // flagged by static_row_sums_k
    for (int64_t x = x0 + lane; x < x1; x += 32) {
      const int32_t v = col[x];
      if (v < 0 || v >= n) {   // a column outside [0, n): flag it, do not index memb with it
        atomicOr(&acc[6], 4ull);
        continue;
      }
      if (memb[v] == cu) L += (unsigned long long)wt[x];
    }
  }
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) L += __shfl_xor_sync(0xffffffffu, L, m);
  if (lane == 0 && L) atomic_add_u128(&acc[2], &acc[3], (u128)L);
}

__global__ void static_squares_k(const long long* __restrict__ sig, int64_t n, unsigned long long* acc) {
  u128 ss = 0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long v = (unsigned long long)sig[c];
    ss += (u128)v * (u128)v;
  }
  if (ss) atomic_add_u128(&acc[4], &acc[5], ss);
}

unsigned grid_of(int64_t work, int per) {
  int64_t b = (work + per - 1) / per;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace
}  // namespace gbl

using namespace gbl;

extern "C" int louvain_modularity_static(int64_t n, const int64_t* offsets, const int32_t* cols,
                                         const int32_t* weights, const int32_t* memb, void* cuda_stream, double* q,
                                         int64_t* num_hi, uint64_t* num_lo, int64_t* M_out) {
  if (n > kMaxV) return LOUVAIN_ERR_CAPACITY;
  if (n < 0 || !q || (n > 0 && (!offsets || !cols || !weights || !memb))) return LOUVAIN_ERR_INVALID_ARG;
  if (n == 0) {
    *q = 0.0;
    if (num_hi) *num_hi = 0;
    if (num_lo) *num_lo = 0;
    if (M_out) *M_out = 0;
    return 0;
  }
  void* base = nullptr;
  if (int r = scratch_address(&base)) return r;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned long long* acc = (unsigned long long*)base;
  long long* K = (long long*)((unsigned char*)base + 256);
  long long* sig = K + kMaxV;
  // clear what must start at zero: the sums and the community totals
  if (cudaMemsetAsync(acc, 0, kAccWords * sizeof(unsigned long long), s) != cudaSuccess ||
      cudaMemsetAsync(sig, 0, (size_t)n * sizeof(long long), s) != cudaSuccess)
    return LOUVAIN_ERR_CUDA;
  (count_launch(), static_row_sums_k<int32_t><<<grid_of(n, 8), 256, 0, s>>>(offsets, weights, n, K, acc));
  (count_launch(), static_totals_k<<<grid_of(n, 256), 256, 0, s>>>(K, memb, n, sig, acc));
  (count_launch(), static_intra_k<int32_t><<<grid_of(n, 8), 256, 0, s>>>(offsets, cols, weights, n, memb, acc));
  (count_launch(), static_squares_k<<<grid_of(n, 256), 256, 0, s>>>(sig, n, acc));
  unsigned long long h[kAccWords];
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return LOUVAIN_ERR_CUDA;
  if (h[6] & 1) return LOUVAIN_ERR_INVALID_ARG;   // a membership outside [0, n)
  if (h[6] & 6) return LOUVAIN_ERR_BAD_CSR;       // decreasing offsets or a column outside [0, n)
  if (h[1] != 0 || h[0] >= (1ull << 62)) return LOUVAIN_ERR_OVERFLOW;
  const int64_t M = (int64_t)h[0];
  const u128 L = ((u128)h[3] << 64) | (u128)h[2];
  const u128 SS = ((u128)h[5] << 64) | (u128)h[4];
  const i128 N = (i128)M * (i128)L - (i128)SS;
  *q = M == 0 ? 0.0 : (double)N / (double)((i128)M * M);
  if (num_hi) *num_hi = (int64_t)(N >> 64);
  if (num_lo) *num_lo = (uint64_t)N;
  if (M_out) *M_out = M;
  return 0;
}
