// engine.h — host-side declarations shared by the engine's translation units.
#pragma once
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>
#include <cuda_runtime.h>
#include "common.cuh"

namespace gbl {

// Degree classes of the local-moving phase (see local_move.cu).
constexpr int kBuckets = 6;          // 0 thread, 1 warp/64, 2 warp/256, 3 block/2k, 4 block/8k, 5 hub
constexpr int kHubBucket = 5;
// Degree thresholds of the local-moving mapping: bucket b < 5 takes the
// degrees in (t[b - 1], t[b]], degrees above t[4] are hubs.  Each t[b] stays
// within its kernel's capacity kLMCap[b] (register table of 8 entries; shared
// tables of 64, 256, 2048 and 8192 slots at most half full), so lowering one
// moves vertices to a wider mapping with a sparser table.  The defaults are
// the capacities; louvain_autotune picks others by timing.
struct LMThresholds {
  int32_t t[5];
};
constexpr int32_t kLMCap[5] = {8, 32, 128, 1024, 4096};
__host__ __device__ inline int lm_bucket_of(int64_t deg, const LMThresholds& th) {
  if (deg <= 0) return -1;
#pragma unroll
  for (int b = 0; b < 5; ++b)
    if (deg <= th.t[b]) return b;
  return 5;
}
constexpr int64_t kHubChunkEntries = 1024;   // entries per insert block of a hub
constexpr int64_t kSlotChunk = 4096;         // table slots per scan block (hubs and large communities)

// Community classes of the aggregation phase by total member degree.
constexpr int kAggBuckets = 6;   // 0 thread/16, 1 thread/32, 2 warp/256, 3 block/2k, 4 block/8k, 5 global
constexpr int kAggGlobal = 5;
constexpr int kAggThreadEntries = 16;   // bucket 0: a thread sorts up to this many entries in registers
__host__ __device__ inline int agg_bucket_of(int64_t dsum) {
  return dsum <= 0 ? -1
         : dsum <= kAggThreadEntries ? 0
         : dsum <= 32 ? 1 : dsum <= 128 ? 2 : dsum <= 1024 ? 3 : dsum <= 4096 ? 4 : 5;
}
constexpr int64_t kAggChunkEntries = 2048;
constexpr int64_t kRelabelChunk = 1024;     // CSR entries per warp of the relabel kernel

// Vertex classes of one iteration.  Every graph has a schedule category
// (per-graph gcat, or single_cat with one graph): kCatSmall takes class
// (local id mod Ps, or with mode_s != 0 hash32(local id ^ salt) mod Ps),
// kCatLarge the same with Pb and mode_b, kCatSparse with Pl and mode_b.
// Mode 1 salts by (pass, iteration), mode 2 by pass only; the iteration is
// read on the device, so an iteration's launches do not depend on it.
constexpr int32_t kCatLarge = 0, kCatSmall = 1, kCatSparse = 2;
struct ClassSpec {
  int32_t Ps, Pb, Pl;
  int32_t mode_s, mode_b;
  int32_t pass;
  int32_t single_cat;
  const int32_t* colour;   // colour classes of the pass graph's vertices, or null
  // a compact pass graph (isolated communities left out): the isolated count
  // before each vertex and, per graph, before the graph's first vertex, so
  // that classes follow the full numbering (null: the ids are full)
  const int32_t* isob;
  const int64_t* zpre;
};
// splitmix64 finaliser of (pass, iteration), folded to 32 bits, never 0.
__host__ __device__ inline uint32_t class_salt(int pass, int iter) {
  uint64_t z = ((uint64_t)(uint32_t)pass << 32 | (uint32_t)iter) + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const uint32_t v = (uint32_t)(z ^ (z >> 32));
  return v ? v : 1u;
}
// The class of vertex i in iteration iter (gid, vo, gcat null: one graph).
__device__ __forceinline__ int vertex_class(int64_t i, const int32_t* gid, const int64_t* vo, const int32_t* gcat,
                                            const ClassSpec& cs, int iter) {
  if (cs.colour) return cs.colour[i];
  int64_t local = i;
  int cat = cs.single_cat;
  if (gid) {
    const int g = gid[i];
    local = i - vo[g];
    cat = gcat[g];
    if (cs.isob) local += cs.isob[i] - cs.zpre[g];
  } else if (cs.isob) {
    local += cs.isob[i];
  }
  const uint32_t Pg = (uint32_t)(cat == kCatSmall ? cs.Ps : (cat == kCatSparse ? cs.Pl : cs.Pb));
  const int mode = cat == kCatSmall ? cs.mode_s : cs.mode_b;
  if (!mode) return (int)(local % Pg);
  return (int)(hash32((uint32_t)local ^ class_salt(cs.pass, mode == 1 ? iter : 0)) % Pg);
}

// ------------------------------------------------------ local_move.cu
template <typename W>
void lm_launch_bucket(const LMArgs<W>& a, bool wide, bool async, int bucket, const int32_t* verts, int nverts,
                      cudaStream_t s);
template <typename W>
void lm_launch_hubs(const LMArgs<W>& a, bool wide, bool async, const int32_t* hubs, int nhubs,
                    const int64_t* chunk_pre, int64_t nchunks, const int64_t* spre, int64_t nslotchunks,
                    cudaStream_t s);
// Class ch of a small pass graph with no vertex above degree 128 in one
// launch (buckets 0-2, nverts vertices); ko = the bucket offsets (device).
template <typename W>
void lm_launch_class(const LMArgs<W>& a, bool wide, bool async, const int32_t* list, const int64_t* ko, int P,
                     int ch, int64_t nverts, cudaStream_t s);
constexpr int64_t kSmallPassEntries = 1 << 21;   // CSR entries up to which a pass takes one launch per class
// Pruning marks of every hub of the pass's hub list that moved in this iteration.
template <typename W>
void lm_launch_hub_mark(const LMArgs<W>& a, const int32_t* hubs, int nhubs, const int64_t* chunk_pre, int64_t nchunks,
                        cudaStream_t s);
template <typename W>
void lm_launch_commit(const LMArgs<W>& a, int64_t max_moves, cudaStream_t s);

// ------------------------------------------------------- graph_ops.cu

// Exclusive scan of n values into out (out may alias in); if total != nullptr
// the sum of all values is stored there (device).  tmp needs scan_tmp_bytes(n).
size_t scan_tmp_bytes(int64_t n);
void scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, int64_t* total, void* tmp, cudaStream_t s);
void scan_i64(const int64_t* in, int64_t* out, int64_t n, int64_t* total, void* tmp, cudaStream_t s);
void scan_i32(const int32_t* in, int32_t* out, int64_t n, int64_t* total, void* tmp, cudaStream_t s);

// Stable partition of [0, n) by key[i] in [0, nkeys): out lists the ids in key
// order, ascending within a key; key_off[nkeys + 1] (device) gets the offsets.
size_t partition_tmp_bytes(int64_t n, int nkeys);
void stable_partition(const int32_t* key, int64_t n, int nkeys, int32_t* out, int64_t* key_off, void* tmp,
                      cudaStream_t s);

// Keys for the local-moving lists, bucket-major: key[i] = bucket * P + class
// of vertex i (P >= Ps, Pb); vertices of degree 0 get the trailing key
// kBuckets * P.
// active (may be null): the stamps of this iteration; with it, vertices not
// active in it, or of a stopped graph (g_on), get the trailing key.
void lm_keys(const int64_t* off, int64_t n, int P, int32_t* key, const int32_t* gid, const int64_t* vo,
             const int32_t* gcat, ClassSpec cs, const int* d_iter, LMThresholds th, const int32_t* active,
             const int32_t* g_on, cudaStream_t s);
// lm_keys for the m vertices sub[0..m) (with `active`, as lm_keys);
// gather_ids: out[j] = sub[idx[j]].
void lm_keys_sub(const int64_t* off, const int32_t* sub, int64_t m, int P, int32_t* key, const int32_t* gid,
                 const int64_t* vo, const int32_t* gcat, ClassSpec cs, const int* d_iter, LMThresholds th,
                 const int32_t* active, const int32_t* g_on, cudaStream_t s);
void gather_ids(const int32_t* idx, const int32_t* sub, int64_t m, int32_t* out, cudaStream_t s);
// For the hub list: per hub its table base (2 * degree slots), the prefix of
// its insert chunks and the prefix of its slot chunks (each nhubs + 1 long).
void hub_layout(const int64_t* off, const int32_t* hubs, int64_t nhubs, int64_t* hbase, int64_t* chunk_pre,
                int64_t* spre, void* tmp, cudaStream_t s);

// Row sums K (int64) of a CSR, the total M (u128 lo/hi) and the self-loop
// total (u128 at acc[2..3]); crow: (n + nnz) / kRelabelChunk + 2 ints of
// scratch for the merge-path chunks.  With flags non-null the same pass
// checks the entries: flags |= 2 column out of range, 4 weight <= 0;
// hashes[0..1] += sums of mix(u,v,w) and mix(v,u,w) (the offsets must have
// passed validate_offsets).
template <typename W>
void row_sums(const int64_t* off, const int32_t* col, const W* wt, int64_t n, int64_t nnz, int32_t* crow,
              long long* K, unsigned long long* acc /* [0..1] M lo/hi, [2..3] self-loop total */, int* flags,
              unsigned long long* hashes, cudaStream_t s);

// Pass set-up: memb = identity, Sigma = K, sizes 1, stamps -1.
void pass_init(int64_t n, const long long* K, int32_t* memb, long long* sig, int32_t* csize, int32_t* stampA,
               int32_t* stampB, cudaStream_t s);
// Partition, then merge: vertex u in part floor(u * parts / n) (part p's
// first vertex ceil(p * n / parts)); induced_parts writes the induced
// subgraphs' block-diagonal CSR (flags, pos: nnz scratch; total: 1 device
// int64); part_base turns part-local community ids into global ones.
void induced_parts(const int64_t* off, const int32_t* col, const int32_t* w, int64_t n, int64_t nnz, int64_t parts,
                   int64_t* flags, int64_t* pos, int64_t* total, int64_t* off_sub, int32_t* col_sub, int32_t* w_sub,
                   void* tmp, cudaStream_t s);
void part_base(int32_t* memb, int64_t n, int64_t parts, cudaStream_t s);
// Shift the offsets and columns of graphs copied side by side (see louvain_load_parts).
void rebase_parts(int64_t* off, int32_t* col, int64_t n, int64_t nnz, const int64_t* vo, const int64_t* eo, int G,
                  cudaStream_t s);
// *flag |= 1 if some memb[i] lies outside vertex i's graph's range (gid and
// vo null: outside [0, n)).
void check_membership(int64_t n, const int32_t* memb, const int32_t* gid, const int64_t* vo, int* flag,
                      cudaStream_t s);
// Pass 0 from the membership already in memb (validated per graph; *flag set
// on a bad id): Sigma and sizes summed over the communities' members.
void pass_init_from(int64_t n, const long long* K, int32_t* memb, long long* sig, int32_t* csize, int32_t* stampA,
                    int32_t* stampB, const int32_t* gid, const int64_t* vo, int* flag, cudaStream_t s);

// Modularity numerator parts: sumL (u64) += weights inside communities,
// ss (u128 lo/hi) += sum over c < n of sig[c]^2.
// crow: merge-path scratch ((n + nnz) / kRelabelChunk + 2 ints).
template <typename W>
void modularity_parts(const int64_t* off, const int32_t* col, const W* wt, int64_t n, int64_t nnz,
                      const int32_t* memb, const long long* sig,
                      unsigned long long* acc /* [0], [3] L lo/hi, [1..2] ss lo/hi */, int32_t* crow, cudaStream_t s);
// ss (u128 lo/hi at acc[0..1]) += sum over i < n of v[i]^2.
void sum_squares(const long long* v, int64_t n, unsigned long long* acc, cudaStream_t s);
// Community totals for an arbitrary membership (Sigma_c = sum K_i over c).
void community_totals(const long long* K, const int32_t* memb, int64_t n, long long* sig, cudaStream_t s);

// Renumbering: used flags, dense ids by ascending old id, level = newid[memb],
// top = level[top].
void mark_used(const int32_t* memb, int64_t n, int32_t* used, cudaStream_t s);
void apply_level(const int32_t* memb, const int32_t* newid, int64_t n, int32_t* level, cudaStream_t s);
void compose_top(int32_t* top, int64_t n0, const int32_t* level, cudaStream_t s);
void coarse_degrees(const int32_t* used, const int32_t* newid, const long long* sig, int64_t n, long long* Knext,
                    cudaStream_t s);

// Aggregation.  members grouped by community (counting sort), mpre = prefix
// of member degrees, then per community the (D, w) sums into tmp rows at
// mpre[cstart[C]], row lengths into rlen; finally compaction into the coarse CSR.
struct AggArgs {
  const int64_t* off;
  const int32_t* col;
  const void* wt;          // W
  const int32_t* level;    // community of each vertex, in [0, k)
  int64_t n, k;
  const int64_t* cstart;   // k + 1
  const int32_t* members;  // n
  const int64_t* mpre;     // n + 1
  int32_t* tcol;           // nnz (tmp rows)
  void* tw;                // nnz (W2)
  int64_t* rlen;           // k
  int32_t* gkeys;          // global tables
  unsigned long long* gvals;
  unsigned long long* lsum;  // += weight of every coarse self-loop (sum of L_C)
  const int32_t* cgid;       // several graphs: graph of each coarse vertex (else nullptr)
  unsigned long long* glsum; // several graphs: per-graph sum of L_C (lo, hi)
  const int64_t* glo;        // global-table communities: first key of a direct table, or -1 (hashed)
  int* error;
};
// Members grouped by community (members[cstart[C] ..]), inv[u] = position of u.
void agg_group_members(const int32_t* level, int64_t n, int64_t k, int64_t* cnt /* k+1 */, int64_t* cstart,
                       int64_t* fill, int32_t* members, int32_t* inv, void* tmp, cudaStream_t s);
void agg_member_prefix(const int64_t* off, const int32_t* members, int64_t n, int64_t* mdeg, int64_t* mpre,
                       void* tmp, cudaStream_t s);
void agg_keys(const int64_t* cstart, const int64_t* mpre, int64_t k, int32_t* key, cudaStream_t s);
// Relabelled member rows: tmp entry mpre[inv[u]] + (x - off[u]) = (level[col[x]],
// w[x]) for every CSR entry x of row u (crow: nnz / kRelabelChunk + 1 ints).
template <typename W, typename W2>
void agg_relabel(const int64_t* off, const int32_t* col, const W* wt, int64_t n, int64_t nnz, const int32_t* level,
                 const int32_t* inv, const int64_t* mpre, int32_t* crow, int32_t* tcol, W2* tw, cudaStream_t s);
template <typename W, typename W2>
void agg_launch_bucket(const AggArgs& a, int bucket, const int32_t* comms, int ncomms, cudaStream_t s);
template <typename W, typename W2>
void agg_launch_global(const AggArgs& a, const int32_t* comms, int ncomms, const int64_t* gbase,
                       const int64_t* chunk_pre, int64_t nchunks, const int64_t* spre, int64_t nslotchunks,
                       cudaStream_t s);
// Table of each global-bucket community: hashed with 2 x its member entries
// slots, or, when that is at least the number of communities of its graph,
// direct-indexed by community id (glo[h] = the graph's first community id).
void agg_global_layout(const int64_t* cstart, const int64_t* mpre, const int32_t* comms, int64_t ncomms, int64_t k,
                       const int32_t* cgid, const int64_t* cvo, int64_t* gbase, int64_t* chunk_pre, int64_t* spre,
                       int64_t* glo, void* tmp, cudaStream_t s);
// Coarse rows from their tmp positions to the coarse CSR (coff = its
// offsets, k rows, nnz2 entries; crow: merge-path scratch of
// (k + nnz2) / kRelabelChunk + 2 ints).
template <typename W2>
void agg_compact(const int64_t* cstart, const int64_t* mpre, const int64_t* coff, int64_t k, int64_t nnz2,
                 int32_t* crow, const int32_t* tcol, const W2* tw, int32_t* ocol, W2* ow, cudaStream_t s);

// Several graphs in one CSR (contiguous vertex ranges per graph).
void graph_totals(const long long* K, const int32_t* gid, int64_t n, unsigned long long* Mg, cudaStream_t s);
template <typename W>
void graph_modularity_parts(const int64_t* off, const int32_t* col, const W* wt, int64_t n, int64_t nnz,
                            const int32_t* memb, const long long* sig, const int32_t* gid, unsigned long long* Lg,
                            unsigned long long* SSg, int32_t* crow /* merge-path scratch */, cudaStream_t s);
void graph_squares(const long long* sig, const int32_t* gid, int64_t n, unsigned long long* SSg, cudaStream_t s);
void graph_renumber(const int32_t* used, const int32_t* newid, const int32_t* gid, int64_t n, int64_t* kcount,
                    int32_t* gid_next, cudaStream_t s);
void localize_membership(const int32_t* top, const int32_t* gid0, const int64_t* vo, int64_t n0, int32_t* out,
                         cudaStream_t s);
void graph_entries(const int64_t* off, const int64_t* vo, int64_t G, int64_t* out, cudaStream_t s);
// Colour classes: capped greedy colouring of a pass graph (graph_ops.cu).
// Isolated communities leave the pass graphs after pass 0 (graph_ops.cu):
// flags of non-empty rows; the compacted offsets, degrees, graph ids and
// isolated counts (isob), columns renumbered in place and top[] rewritten;
// the counts carried through a pass's renumbering; top[] back in the full
// numbering at the end (and the per-graph offsets vo_top shifted by zpre).
void nonempty_rows(const int64_t* off, int64_t k, int32_t* flag, cudaStream_t s);
void compact_rows(const int64_t* off, int64_t k, int64_t nnz, const int32_t* flag, const int32_t* pos,
                  const long long* Kin, const int32_t* gid_in, int64_t* off_out, long long* K_out, int32_t* gid_out,
                  int32_t* isob, int32_t* col, int32_t* top, int64_t n0, cudaStream_t s);
void carry_isob(const int32_t* used, const int32_t* newid, const int32_t* isob, int64_t n, int32_t* isob_next,
                cudaStream_t s);
void finalize_top(int32_t* top, int64_t n0, const int32_t* isob, int64_t kc, int64_t* vo_top, const int64_t* zpre,
                  int64_t G, cudaStream_t s);
void count_empty_rows(const int64_t* off, int64_t n, unsigned long long* out, cudaStream_t s);
void compact_vo(const int64_t* vo_full, int64_t G, const int32_t* pos, int64_t k, int64_t kc, int64_t* vo_c,
                cudaStream_t s);

// Colouring frontiers: vertices of degree above kColourHubDegree go to the
// hub frontier (hfront / hnext), whose rows many blocks share; hmask / hdone
// hold a zeroed mask and item counter per hub-frontier slot (at most
// nnz / kColourHubDegree + 1 slots), left zeroed after every round.
constexpr int64_t kColourHubDegree = 2048;
// isob / zpre: as in ClassSpec (priorities follow the full numbering).
void colour_init(const int64_t* off, const int32_t* col, int64_t n, const int32_t* gid, const int64_t* vo,
                 const int32_t* isob, const int64_t* zpre, uint32_t salt, int32_t* cnt, int32_t* cls, int32_t* front,
                 unsigned long long* nfront, int32_t* hfront, unsigned long long* nhfront, cudaStream_t s);
void colour_round(const int64_t* off, const int32_t* col, int64_t n, const int32_t* gid, const int64_t* vo,
                  const int32_t* isob, const int64_t* zpre, uint32_t salt, const int32_t* front,
                  const unsigned long long* nfront, const int32_t* hfront,
                  const unsigned long long* nhfront, int32_t* cnt, int32_t* cls, int32_t* next,
                  unsigned long long* nnext, int32_t* hnext, unsigned long long* nhnext, unsigned long long* total,
                  unsigned long long* hmask, int32_t* hdone, int* flags, cudaStream_t s);
void class_max(const int32_t* cls, int64_t n, int* out, cudaStream_t s);
void graph_ids(const int64_t* vo, int G, int64_t n, int64_t nnz, int32_t* gid, const int64_t* off, const int32_t* col,
               int32_t* crow /* merge-path scratch */, int* flags, cudaStream_t s);

// Input checks: flags |= 1 offsets not monotone / bad ends, 2 col out of
// range, 4 weight <= 0; hashes[0..1] = sums of mix(u,v,w) and mix(v,u,w).
// flags = 1 if the offsets decrease or have the wrong ends (else 0).
void validate_offsets(const int64_t* off, int64_t n, int64_t nnz, int* flags, cudaStream_t s);

// Copies with conversion.
void widen_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);
void fill_i32(int32_t* p, int32_t v, int64_t n, cudaStream_t s);
void iota_i32(int32_t* p, int64_t n, cudaStream_t s);

// Resident blocks per SM of a kernel at a block size and dynamic shared
// memory size, asked of the runtime once per combination (the query costs
// several microseconds of host time, and launches are on the host's critical
// path when kernels are short).
template <typename K>
int blocks_per_sm(K kernel, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t>, int> cache;
  const auto key = std::make_tuple((const void*)kernel, threads, smem);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess || per < 1) {
    cudaGetLastError();
    per = 1;
  }
  cache.emplace(key, per);
  return per;
}

}  // namespace gbl
