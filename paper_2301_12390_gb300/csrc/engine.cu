// engine.cu — the pass driver and the C ABI (include/louvain.h).
//
// A run follows Section 3.2 of the paper: passes of a local-moving phase
// (iterations until the iteration gain is <= tolerance, at most
// max_iterations) and an aggregation phase; tolerance divided by the decline
// factor after every pass; the run ends after a pass with no move, a pass
// whose modularity gain is <= pass_tolerance, or max_passes.  Every decision
// that a floating-point value takes is made on exact integers converted
// once: the iteration test is (2.0 * dbl(S)) / dbl(M^2) <= tolerance and the
// pass test dbl(N_after - N_before) / dbl(M^2) <= pass_tolerance, dbl() the
// correctly rounded int128 -> double conversion.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <initializer_list>
#include <vector>
#include "engine.h"
#include "../../include/louvain.h"

using namespace gbl;

#include <atomic>
namespace gbl {
static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace gbl

namespace {

// Vertex classes per asynchronous iteration when the options leave it to the
// engine, per graph: with every vertex deciding at once, stale neighbour
// memberships make pairs and groups swap and modularity can collapse; classes
// run in sequence keep the result near the sequential order's.  Small graphs
// (few thousand vertices, few dense communities) need small classes: at 16
// some planted-partition graphs ended more than 0.01 below the sequential
// order, at 32 none did.  A large graph of fewer than kSparseEntries entries
// per vertex (a vertex rarely shares its class with a neighbour) takes 8: the
// road grid ran 13% faster than at 16 with the same Q.  A denser one takes
// 16: 24 raised R-MAT s22's Q from 0.076 to 0.077 (the sequential order's is
// 0.075) but took the serving pool's large graphs 9% more run time.
constexpr int kAsyncSubroundsLarge = 16;
constexpr int kAsyncSubroundsSparse = 8;
constexpr int kAsyncSubroundsSmall = 32;
constexpr int64_t kSparseEntries = 8;
// Asynchronous bucket streams: the hubs of an iteration run in this many
// groups of consecutive classes (one class per group up to this many classes).
constexpr int kHubGroups = 16;
constexpr int64_t kSmallGraph = 65536;
// Active-list filtering (local_moving): measured on the 4,096-graph SBM batch
// (pass 0, most graphs stopped after a few iterations: 150 -> 96 ms) and the
// road grid and R-MAT (no gain; a quarter as the threshold cost the road grid 9%).
constexpr int64_t kFilterMinList = 2000000;
constexpr double kFilterFraction = 0.1;
// A pass with at least this many vertices per vertex with edges classifies
// its later iterations over the vertices with edges only.
constexpr int64_t kEdgeListRatio = 4;

struct IterRec {
  int pass;
  int64_t moves;
  u128 S;
};

// One graph of a run (a plain load is one graph; a batch load, several).
struct GraphState {
  int64_t M = 0;          // its total weight
  i128 qnum = 0;          // exact Q numerator of its current partition
  bool stopped = false;   // has left the run
  int64_t k = 0;          // communities after its last pass
  int passes = 0;         // passes whose local-moving it took part in
  int64_t pass_moves = 0; // moves in the current pass
  int pass_iters = 0;     // iterations in the current pass
  std::vector<IterRec> iters;   // every iteration it took part in (several graphs only)
};

struct PassRec {
  louvain_pass_info info;
  std::vector<int32_t> level;
  std::vector<int64_t> coff;
  std::vector<int32_t> ccol;
  std::vector<int64_t> cw;
};

}  // namespace

struct louvain_ctx {
  louvain_options opt;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;

  // graph
  bool loaded = false, ran = false;
  int64_t n0 = 0, nnz0 = 0;
  int64_t bytes = 0;
  std::vector<void*> allocs;

  // device buffers
  int64_t* off0 = nullptr;
  int32_t* col0 = nullptr;
  int32_t* w0 = nullptr;
  int64_t* offX[2] = {nullptr, nullptr};
  int32_t* colX[2] = {nullptr, nullptr};
  unsigned char* wX[2] = {nullptr, nullptr};   // int64-sized storage, used as int32 when M < 2^31
  long long* K0 = nullptr;            // input row sums (for louvain_modularity)
  long long* K = nullptr;
  long long* Knext = nullptr;
  int32_t* memb = nullptr;
  long long* sig = nullptr;
  int32_t* csize = nullptr;
  int32_t* stamp[2] = {nullptr, nullptr};
  int32_t* key = nullptr;
  int32_t* list = nullptr;
  int32_t* used = nullptr;
  int32_t* newid = nullptr;
  int32_t* level = nullptr;
  int32_t* top = nullptr;
  int2* moves = nullptr;
  int64_t* key_off = nullptr;
  int64_t* cnt = nullptr;
  int64_t* cstart = nullptr;
  int64_t* fill = nullptr;
  int32_t* members = nullptr;
  int64_t* mdeg = nullptr;
  int64_t* mpre = nullptr;
  int64_t* rlen = nullptr;
  int32_t* tcol = nullptr;
  unsigned char* tw = nullptr;
  int32_t* gkeys = nullptr;
  unsigned long long* gvals = nullptr;
  int64_t* gbase = nullptr;
  int64_t* chunk_pre = nullptr;
  int64_t* spre = nullptr;
  int64_t* glo = nullptr;
  int32_t* inv = nullptr;      // aggregation: member position of each vertex
  int32_t* hmoved = nullptr;   // local moving: iteration + 1 of a hub's last move (by hub-list position)
  int32_t* d_gcat = nullptr;   // per graph: its class-schedule category (kCatSmall, kCatLarge, kCatSparse)
  std::vector<int32_t> hgcat;   // the same on the host
  LMThresholds thr = {{kLMCap[0], kLMCap[1], kLMCap[2], kLMCap[3], kLMCap[4]}};   // degree mapping
  bool warm = false;           // this run's pass 0 starts from the membership in memb
  int64_t lm_cands = 0;        // candidate communities evaluated by this run's local moving
  louvain_ctx* sub = nullptr;  // louvain_run_partitioned: the parts' context (same device and stream)
  int32_t* crow = nullptr;     // aggregation: first row of each relabel chunk      // aggregation: direct-table first key per global community, or -1
  unsigned long long* hkid = nullptr;
  int32_t* hdone = nullptr;            // local moving: finished scan chunks per hub (zero between uses)
  long long* hpart = nullptr;
  int32_t* hpart_c = nullptr;
  int64_t npart = 0;
  unsigned char* tmp = nullptr;
  size_t tmp_bytes = 0;
  int64_t M0 = 0;                      // total weight of the loaded graph
  int64_t cap_n = 0, cap_nnz = 0;      // arena capacity
  bool dry_run = false;                // alloc_arena only adds up the bytes
  bool tables_dirty = true;            // global tables need clearing (new arena or a failed run)
  i128 qnum0 = 0;                      // exact Q numerator of the singleton partition of the loaded graph
  DevCounters* ctr = nullptr;
  unsigned long long* acc = nullptr;   // 8 words of reduction scratch
  int* flags = nullptr;
  int* d_iter = nullptr;               // current local-moving iteration (device)
  int* h_iter = nullptr;               // pinned staging for it
  int64_t* scal = nullptr;             // small device scalars
  // pinned host mirror
  DevCounters* h_ctr = nullptr;
  unsigned long long* h_acc = nullptr;
  int64_t* h_scal = nullptr;
  void* h_pair = nullptr;   // pinned staging of fetch_pair (grown on demand)
  size_t h_pair_cap = 0;

  // several graphs (block-diagonal CSR): G graphs, vertex ranges vo0
  int64_t G = 1;
  std::vector<GraphState> gst;
  std::vector<int64_t> gM0, gn0;       // per graph: M and vertices of the loaded graph
  std::vector<i128> gqnum0;            // per graph: singleton Q numerator of the loaded graph
  int32_t* gid0 = nullptr;             // graph of every input vertex
  int32_t* gid_a = nullptr;
  int32_t* gid_b = nullptr;
  int32_t* gid = nullptr;              // graph of every vertex of the pass graph
  int32_t* gid_next = nullptr;         // ... of the coarse graph being built
  int64_t* vo0 = nullptr;              // first input vertex of each graph (G + 1)
  int64_t* vo_a = nullptr;
  int64_t* vo_b = nullptr;
  int64_t* vo = nullptr;               // first pass-graph vertex of each graph
  int64_t* vo_next = nullptr;
  int64_t* vo_top = nullptr;           // first community id of each graph in the top membership
  // Isolated communities leave the pass graphs after pass 0 (communities of
  // vertices without edges: singletons that never move); later passes run on
  // the other vertices only, in the same order (compact ids).
  int64_t iso0 = 0;                    // empty rows of the loaded graph
  bool compacted = false;              // this run's pass graphs are compact
  int64_t iso_z = 0;                   // isolated communities left out (all graphs)
  std::vector<int64_t> h_zg;           // ... per graph
  int32_t* isob[2] = {nullptr, nullptr};   // per compact vertex: isolated communities before it
  int isob_cur = 0;                    // isob[isob_cur] belongs to the current pass graph
  int64_t kc_top = 0;                  // the compact ids in top[] lie below this
  int64_t* d_zpre = nullptr;           // per graph: isolated communities of the graphs before it
  int64_t* kcount = nullptr;
  long long* d_Mg = nullptr;
  int32_t* d_gon = nullptr;
  unsigned long long* d_gmoves = nullptr;
  unsigned long long* d_gs = nullptr;
  unsigned long long* d_gL = nullptr;
  unsigned long long* d_gSS = nullptr;
  int64_t hcap = 0;                    // pinned per-graph host buffers below hold hcap graphs
  int32_t* h_gon = nullptr;
  unsigned long long* h_gmoves = nullptr;
  unsigned long long* h_gs = nullptr;
  unsigned long long* h_gL = nullptr;
  unsigned long long* h_gSS = nullptr;

  // results
  int64_t M = 0;
  i128 qnum = 0;
  double Q = 0.0;
  int64_t k_final = 0;
  i128 agg_nafter = 0;                 // Q numerator found by the last aggregation
  std::vector<IterRec> iters;
  std::vector<PassRec> passes;
  louvain_stats stats;
  cudaEvent_t ev[8] = {};
  // the degree buckets of a vertex class run concurrently, one stream each
  static constexpr int kAux = kBuckets;
  cudaStream_t aux[kAux] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kAux] = {};
};

namespace {

int fail(louvain_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CK(call)                                                                                    \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return fail(c, e_ == cudaErrorMemoryAllocation ? LOUVAIN_ERR_OOM : LOUVAIN_ERR_CUDA,          \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                             \
  } while (0)

#define CKLAUNCH() CK(cudaGetLastError())

double dbl(i128 x) { return (double)x; }

void free_all(louvain_ctx* c) {
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  c->bytes = 0;
  c->loaded = false;
  c->ran = false;
  c->cap_n = 0;
  c->cap_nnz = 0;
}

template <typename T>
int dalloc(louvain_ctx* c, T** p, int64_t count) {
  size_t b = (size_t)(count > 0 ? count : 1) * sizeof(T);
  b = (b + 255) & ~(size_t)255;
  if (c->dry_run) {   // size the arena only
    c->bytes += (int64_t)b;
    *p = nullptr;
    return 0;
  }
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, b);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, LOUVAIN_ERR_OOM, "cudaMalloc of " + std::to_string(b) + " bytes failed");
  }
  c->allocs.push_back(q);
  c->bytes += (int64_t)b;
  *p = (T*)q;
  return 0;
}

#define ALLOC(ptr, count)                          \
  do {                                             \
    int r_ = dalloc(c, &(ptr), (int64_t)(count));  \
    if (r_) { free_all(c); return r_; }            \
  } while (0)

int check_options(const louvain_options* o) {
  if (o->mode != LOUVAIN_SYNC && o->mode != LOUVAIN_ASYNC) return 1;
  if (!(o->tolerance >= 0) || !(o->tolerance_decline > 0) || !(o->pass_tolerance == o->pass_tolerance)) return 1;
  if (o->max_iterations < 1 || o->max_passes < 0 || o->max_passes > 64) return 1;
  if (o->subrounds < 0 || o->subrounds > 64) return 1;
  if (o->reclass < 0 || o->reclass > 3) return 1;
  if (o->bucket_streams < 0 || o->bucket_streams > 1) return 1;
  if (o->colour_classes < 0 || o->colour_classes > 1) return 1;
  if (o->stop_rule < 0 || o->stop_rule > 1) return 1;
  return 0;
}

// Copy a small device array to host (synchronises the stream).
int fetch(louvain_ctx* c, void* host, const void* dev, size_t bytes) {
  CK(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return 0;
}

// Several small device arrays to host with one synchronisation (through
// pinned staging, so all copies are queued before the stream is waited for).
struct FetchPiece {
  void* host;
  const void* dev;
  size_t bytes;
};
int fetch_many(louvain_ctx* c, std::initializer_list<FetchPiece> pieces) {
  size_t need = 0;
  for (const FetchPiece& f : pieces) need = ((need + 15) & ~(size_t)15) + f.bytes;
  if (need > c->h_pair_cap) {
    if (c->h_pair) cudaFreeHost(c->h_pair);
    c->h_pair = nullptr;
    c->h_pair_cap = 0;
    const size_t cap = need < 4096 ? 4096 : 2 * need;
    CK(cudaMallocHost(&c->h_pair, cap));
    c->h_pair_cap = cap;
  }
  char* p = (char*)c->h_pair;
  size_t o = 0;
  for (const FetchPiece& f : pieces) {
    o = (o + 15) & ~(size_t)15;
    if (f.bytes) CK(cudaMemcpyAsync(p + o, f.dev, f.bytes, cudaMemcpyDeviceToHost, c->stream));
    o += f.bytes;
  }
  CK(cudaStreamSynchronize(c->stream));
  o = 0;
  for (const FetchPiece& f : pieces) {
    o = (o + 15) & ~(size_t)15;
    if (f.bytes) memcpy(f.host, p + o, f.bytes);
    o += f.bytes;
  }
  return 0;
}

int fetch_pair(louvain_ctx* c, void* h1, const void* d1, size_t b1, void* h2, const void* d2, size_t b2) {
  return fetch_many(c, {{h1, d1, b1}, {h2, d2, b2}});
}

// --------------------------------------------------------------- a pass

struct PassState {
  int64_t n, nnz;
  int64_t* off;
  int32_t* col;
  void* w;
  int widx;   // which coarse buffer holds this graph (-1 = input)
};


// Colour classes of the pass graph (option colour_classes) into c->members,
// the aggregation's member list, which is free until the pass aggregates;
// c->inv (predecessor counts) and c->mdeg / c->fill (the two frontiers) are
// free too, and so are the aggregation's c->tcol (the two hub frontiers) and
// local moving's hub partials c->hpart / c->hpart_c (the hubs' masks and item
// counters; nothing keeps state in them from one iteration to the next; the
// global tables c->gkeys / c->gvals must stay cleared, so they are not
// borrowed).  Rounds run
// kColourRoundsPerCheck at a time between host checks of the frontiers (a
// round with empty frontiers does nothing).  *ncls = the number of classes
// (largest class + 1).
constexpr int kColourRoundsPerCheck = 8;
int colour_pass(louvain_ctx* c, const PassState& g, int pass, int* ncls) {
  cudaStream_t s = c->stream;
  const bool multi = c->G > 1;
  const int32_t* gid = multi ? c->gid : nullptr;
  const int64_t* vo = multi ? c->vo : nullptr;
  const uint32_t salt = 0x9E3779B9u * (uint32_t)(pass + 1);
  int32_t* cls = c->members;
  int32_t* cnt = c->inv;
  int32_t* front[2] = {(int32_t*)c->mdeg, (int32_t*)c->fill};
  const int64_t hslots = g.nnz / kColourHubDegree + 1;
  int32_t* hfront[2] = {c->tcol, c->tcol + hslots};
  unsigned long long* hmask = (unsigned long long*)c->hpart;
  int32_t* hdone = c->hpart_c;
  if (hslots > c->npart) return fail(c, LOUVAIN_ERR_INTERNAL, "colouring: hub slots exceed the partial buffer");
  // [0], [1]: frontier sizes; [2]: coloured; [3], [4]: hub frontier sizes (c->scal + 8)
  unsigned long long* sz = (unsigned long long*)(c->scal + 4);
  unsigned long long* hsz = (unsigned long long*)(c->scal + 8);
  int* cmax = (int*)(c->scal + 7);
  CK(cudaMemsetAsync(sz, 0, 3 * sizeof(unsigned long long), s));
  CK(cudaMemsetAsync(hsz, 0, 2 * sizeof(unsigned long long), s));
  CK(cudaMemsetAsync(hmask, 0, hslots * sizeof(unsigned long long), s));
  CK(cudaMemsetAsync(hdone, 0, hslots * sizeof(int32_t), s));
  CK(cudaMemsetAsync(c->flags, 0, sizeof(int), s));
  const int32_t* isob = c->compacted ? c->isob[c->isob_cur] : nullptr;
  const int64_t* zpre = c->compacted ? c->d_zpre : nullptr;
  colour_init(g.off, g.col, g.n, gid, vo, isob, zpre, salt, cnt, cls, front[0], sz, hfront[0], hsz, s);
  int64_t r = 0;
  for (;;) {
    for (int k = 0; k < kColourRoundsPerCheck; ++k, ++r) {
      const int a = (int)(r & 1), b = a ^ 1;
      CK(cudaMemsetAsync(sz + b, 0, sizeof(unsigned long long), s));
      CK(cudaMemsetAsync(hsz + b, 0, sizeof(unsigned long long), s));
      colour_round(g.off, g.col, g.n, gid, vo, isob, zpre, salt, front[a], sz + a, hfront[a], hsz + a, cnt, cls,
                   front[b],
                   sz + b, hfront[b], hsz + b, sz + 2, hmask, hdone, c->flags, s);
    }
    CKLAUNCH();
    unsigned long long left[2] = {0, 0};
    if (int e = fetch(c, &left[0], sz + (r & 1), sizeof(unsigned long long))) return e;
    if (int e = fetch(c, &left[1], hsz + (r & 1), sizeof(unsigned long long))) return e;
    if (left[0] + left[1] == 0) break;
    if (r > g.n + kColourRoundsPerCheck) return fail(c, LOUVAIN_ERR_INTERNAL, "colouring did not end");
  }
  unsigned long long coloured = 0;
  int flags = 0;
  if (int e = fetch(c, &coloured, sz + 2, sizeof(coloured))) return e;
  if (int e = fetch(c, &flags, c->flags, sizeof(flags))) return e;
  if ((int64_t)coloured != g.n || (flags & 2))
    return fail(c, LOUVAIN_ERR_INTERNAL, "colouring left a vertex without a class (asymmetric CSR?)");
  CK(cudaMemsetAsync(cmax, 0, sizeof(int), s));
  class_max(cls, g.n, cmax, s);
  CKLAUNCH();
  int m = 0;
  if (int e = fetch(c, &m, cmax, sizeof(m))) return e;
  *ncls = m + 1;
  return 0;
}

template <typename W>
int q_numerators(louvain_ctx* c, const PassState& g, std::vector<i128>& out);

template <typename W>
int local_moving(louvain_ctx* c, const PassState& g, int pass, double tol, bool wide, int* iters_out,
                 int64_t* edges_out, int64_t* visited_out) {
  const bool async = c->opt.mode == LOUVAIN_ASYNC;
  // Colour classes (option): the classes are a greedy colouring of the pass
  // graph, the same for every iteration of the pass.
  const bool colour = c->opt.colour_classes != 0;
  int ncls = 1;
  if (colour)
    if (int r = colour_pass(c, g, pass, &ncls)) return r;
  // Classes, per graph (its category, set at load): a graph below
  // kSmallGraph vertices takes kAsyncSubroundsSmall classes drawn once per
  // pass, a larger one kAsyncSubroundsLarge (or, sparse, kAsyncSubroundsSparse)
  // classes drawn anew every iteration (automatic settings), so a graph gets
  // the same schedule alone and in a batch.  Synchronous classes are id mod P.
  bool any_cat[3] = {false, false, false};
  for (int64_t q = 0; q < c->G; ++q) any_cat[c->hgcat[q]] = true;
  const bool any_small = any_cat[kCatSmall], any_big = any_cat[kCatLarge] || any_cat[kCatSparse];
  ClassSpec cs{1, 1, 1, 0, 0, pass, c->G == 1 ? c->hgcat[0] : kCatLarge, nullptr,
               c->compacted ? c->isob[c->isob_cur] : nullptr, c->compacted ? c->d_zpre : nullptr};
  if (colour) {
    cs.Ps = cs.Pb = cs.Pl = ncls;
    cs.colour = c->members;
  } else if (c->opt.subrounds > 0) {
    cs.Ps = cs.Pb = cs.Pl = c->opt.subrounds;
  } else if (async) {
    cs.Ps = kAsyncSubroundsSmall;
    cs.Pb = kAsyncSubroundsLarge;
    cs.Pl = kAsyncSubroundsSparse;
  }
  const int P = colour ? ncls
                       : std::max({any_small ? cs.Ps : 1, any_cat[kCatLarge] ? cs.Pb : 1, any_cat[kCatSparse] ? cs.Pl : 1});
  const int nkeys = kBuckets * P + 1;
  const bool multi = c->G > 1;
  const int64_t G = c->G;
  cudaStream_t s = c->stream;
  // reclass: 1 = hashed classes drawn anew every iteration, 2 = once per pass
  const int mode_s = (!colour && async && cs.Ps > 1) ? (c->opt.reclass == 3 ? 2 : c->opt.reclass) : 0;
  const int mode_b = (!colour && async && (cs.Pb > 1 || cs.Pl > 1)) ? (c->opt.reclass == 3 ? 1 : c->opt.reclass) : 0;
  const bool reclass = (any_small && mode_s == 1) || (any_big && mode_b == 1);   // every iteration
  cs.mode_s = mode_s;
  cs.mode_b = mode_b;
  // Bucket lists: key = bucket * P + class, hubs of all classes contiguous,
  // and the hubs' table layout.
  std::vector<int64_t> ko(nkeys + 1);
  int64_t hub0 = 0, hub1 = 0, nhubs = 0;
  std::vector<int64_t> hchunks, hschunks;
  // sub_m > 0: the classes are drawn anew over the sub_m vertices with edges
  // kept in c->level (a small pass; its other vertices are isolated)
  int64_t sub_m = 0;
  // the class lists of the vertices with edges only, all on the device (a
  // small pass whose classes are drawn anew: part of its iteration)
  auto reclassify_small = [&]() {
    int32_t* idx = (int32_t*)c->moves;   // free in asynchronous mode
    lm_keys_sub(g.off, c->level, sub_m, P, c->key, multi ? c->gid : nullptr, multi ? c->vo : nullptr, c->d_gcat,
                cs, c->d_iter, c->thr, nullptr, nullptr, s);
    stable_partition(c->key, sub_m, nkeys, idx, c->key_off, c->tmp, s);
    gather_ids(idx, c->level, sub_m, c->list, s);
  };
  // With pruning, once few vertices of a large pass are active (the last
  // iteration visited less than kFilterFraction of at least kFilterMinList
  // vertices with edges; below that, partitioning again costs more than the
  // launches over inactive vertices), the
  // lists keep only the vertices the iteration visits (active, graph still
  // iterating): the late iterations of a pass, and batches whose graphs have
  // mostly stopped, launch over those alone.  A filtered list is never reused.
  // A pass whose vertices are mostly isolated (the later passes of a
  // heavy-tailed graph: every isolated vertex stays a community of its own)
  // classifies again only its vertices with edges, kept in c->level (free
  // until renumbering) after the first classification; c->newid (free too)
  // takes the partition's positions.
  int64_t edge_m = 0;
  auto classify = [&](int iter, bool filter) -> int {
    if (edge_m > 0) {
      lm_keys_sub(g.off, c->level, edge_m, P, c->key, multi ? c->gid : nullptr, multi ? c->vo : nullptr, c->d_gcat,
                  cs, c->d_iter, c->thr, filter ? c->stamp[iter & 1] : nullptr, multi ? c->d_gon : nullptr, s);
      stable_partition(c->key, edge_m, nkeys, c->newid, c->key_off, c->tmp, s);
      gather_ids(c->newid, c->level, edge_m, c->list, s);
    } else {
      lm_keys(g.off, g.n, P, c->key, multi ? c->gid : nullptr, multi ? c->vo : nullptr, c->d_gcat, cs, c->d_iter,
              c->thr, filter ? c->stamp[iter & 1] : nullptr, multi ? c->d_gon : nullptr, s);
      stable_partition(c->key, g.n, nkeys, c->list, c->key_off, c->tmp, s);
    }
    CKLAUNCH();
    if (int r = fetch(c, ko.data(), c->key_off, ko.size() * sizeof(int64_t))) return r;
    hub0 = ko[kHubBucket * P];
    hub1 = ko[kHubBucket * P + P];
    nhubs = hub1 - hub0;
    if (nhubs > 0) {
      hub_layout(g.off, c->list + hub0, nhubs, c->gbase, c->chunk_pre, c->spre, c->tmp, s);
      CKLAUNCH();
      hchunks.resize(nhubs + 1);
      hschunks.resize(nhubs + 1);
      if (int r = fetch_pair(c, hchunks.data(), c->chunk_pre, hchunks.size() * sizeof(int64_t), hschunks.data(),
                             c->spre, hschunks.size() * sizeof(int64_t)))
        return r;
      if (hschunks[nhubs] > c->npart) return fail(c, LOUVAIN_ERR_INTERNAL, "hub partial buffer too small");
    }
    return 0;
  };
  // the first classification draws iteration 0's classes
  *c->h_iter = 0;
  CK(cudaMemcpyAsync(c->d_iter, c->h_iter, sizeof(int), cudaMemcpyHostToDevice, s));
  if (int r = classify(0, false)) return r;
  const int64_t full_len = ko[kBuckets * P];   // vertices with edges
  // A small pass graph without vertices above degree 128 takes one launch per
  // class; when its classes are drawn anew every iteration, only its vertices
  // with edges are partitioned again (on R-MAT most vertices of the late
  // passes are isolated).
  const bool small_pass = g.nnz <= kSmallPassEntries && ko[3 * P] == ko[kBuckets * P];
  if (small_pass && reclass) {
    // later classifications partition only the vertices with edges
    sub_m = ko[3 * P];
    CK(cudaMemcpyAsync(c->level, c->list, sub_m * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  } else if (!small_pass && !colour && full_len > 0 && full_len * kEdgeListRatio <= g.n &&
             (reclass || c->opt.prune)) {
    edge_m = full_len;
    CK(cudaMemcpyAsync(c->level, c->list, edge_m * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  }
  // a class kernel of a small pass loops over its class, however large: one
  // grid for the pass, so its iteration's launches do not depend on the draw
  const int64_t class_grid_verts = (ko[3 * P] + P - 1) / P + 1;
  // hub move stamps are iteration numbers of this pass (by position in the
  // first hub list; later lists are subsets of it)
  if (nhubs > 0) CK(cudaMemsetAsync(c->hmoved, 0, (size_t)nhubs * sizeof(int32_t), s));
  LMArgs<W> a;
  memset(&a, 0, sizeof(a));
  a.off = g.off;
  a.col = g.col;
  a.wt = (const W*)g.w;
  a.K = c->K;
  a.memb = c->memb;
  a.sig = c->sig;
  a.csize = c->csize;
  a.moves = c->moves;
  a.ctr = c->ctr;
  a.M = c->M;
  a.prune = c->opt.prune;
  a.guard = c->opt.singleton_guard;
  a.hkeys = c->gkeys;
  a.hvals = c->gvals;
  a.hpart = c->hpart;
  a.hpart_c = c->hpart_c;
  a.hdone = c->hdone;
  a.d_iter = c->d_iter;
  a.stamps[0] = c->stamp[0];
  a.stamps[1] = c->stamp[1];
  if (multi) {
    a.gid = c->gid;
    a.Mg = c->d_Mg;
    a.g_on = c->d_gon;
    a.g_moves = c->d_gmoves;
    a.g_s = c->d_gs;
  }
  // the graphs that iterate in this pass
  for (int64_t q = 0; q < G; ++q) {
    c->gst[q].pass_moves = 0;
    c->gst[q].pass_iters = 0;
    c->h_gon[q] = c->gst[q].stopped ? 0 : 1;
  }
  if (multi) CK(cudaMemcpyAsync(c->d_gon, c->h_gon, G * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  int64_t edges_total = 0, visited_total = 0, cands_total = 0;

  // One iteration's launch sequence: counters cleared, every class's buckets
  // forked onto their streams and joined (synchronous: then committed), and
  // the counters copied to pinned host memory.  The sequence depends on the
  // iteration only through *d_iter (and, for several graphs, the device copy
  // of which graphs still iterate), so a pass can capture it once into a CUDA
  // graph and replay that (a small pass from its second iteration, others
  // with the cuda_graphs option from the third).  A small pass whose classes
  // are drawn anew every iteration draws them inside the sequence, except in
  // iteration 0, whose classes the first classification drew.
  bool drawn = true;
  auto iteration = [&]() -> int {
    CK(cudaMemsetAsync(c->ctr, 0, sizeof(DevCounters), s));
    if (multi) {
      CK(cudaMemsetAsync(c->d_gmoves, 0, G * sizeof(unsigned long long), s));
      CK(cudaMemsetAsync(c->d_gs, 0, 2 * G * sizeof(unsigned long long), s));
    }
    // a small pass graph without vertices above degree 128: one launch per
    // class on the main stream (and the new draw of its classes first)
    if (small_pass && sub_m > 0 && !drawn) reclassify_small();
    drawn = false;
    for (int ch = 0; ch < P && small_pass; ++ch) {
      lm_launch_class<W>(a, wide, async, c->list, c->key_off, P, ch, class_grid_verts, s);
      if (!async) lm_launch_commit<W>(a, ko[3 * P], s);
      CKLAUNCH();
    }
    // Asynchronous, with bucket_streams: every degree bucket runs the classes
    // in order on its own stream without waiting for the other buckets'
    // previous class; the streams join at the end of the iteration.
    const bool streams = async && c->opt.bucket_streams && !small_pass;
    bool sused[kBuckets] = {};
    if (streams) {
      CK(cudaEventRecord(c->ev_fork, s));
      for (int b = 0; b < kBuckets; ++b) CK(cudaStreamWaitEvent(c->aux[b], c->ev_fork, 0));
      for (int ch = 0; ch < P; ++ch) {
        for (int b = 0; b < kHubBucket; ++b) {
          int64_t s0 = ko[b * P + ch], s1 = ko[b * P + ch + 1];
          if (s1 <= s0) continue;
          sused[b] = true;
          lm_launch_bucket<W>(a, wide, async, b, c->list + s0, (int)(s1 - s0), c->aux[b]);
        }
        // hubs go in groups of consecutive classes (one launch sequence each)
        const int hstep = P / kHubGroups > 1 ? P / kHubGroups : 1;
        if (ch % hstep != 0) continue;
        const int chend = ch + hstep < P ? ch + hstep : P;
        int64_t h0 = ko[kHubBucket * P + ch] - hub0, h1 = ko[kHubBucket * P + chend] - hub0;
        if (h1 > h0) {
          sused[kHubBucket] = true;
          LMArgs<W> ah = a;
          ah.hbase = c->gbase + h0;
          ah.spre = c->spre + h0;
          ah.hkid = c->hkid + h0;
          ah.hdone = c->hdone + h0;
          ah.hmoved = c->hmoved + h0;
          lm_launch_hubs<W>(ah, wide, async, c->list + hub0 + h0, (int)(h1 - h0), c->chunk_pre + h0,
                            hchunks[h1] - hchunks[h0], c->spre + h0, hschunks[h1] - hschunks[h0], c->aux[kHubBucket]);
        }
        CKLAUNCH();
      }
      for (int b = 0; b < kBuckets; ++b) {
        if (!sused[b]) continue;
        CK(cudaEventRecord(c->ev_join[b], c->aux[b]));
        CK(cudaStreamWaitEvent(s, c->ev_join[b], 0));
      }
    }
    for (int ch = 0; ch < P && !small_pass && !streams; ++ch) {
      // fork: every non-empty bucket of the class on its own stream
      bool used[kBuckets] = {};
      CK(cudaEventRecord(c->ev_fork, s));
      for (int b = 0; b < kHubBucket; ++b) {
        int64_t s0 = ko[b * P + ch], s1 = ko[b * P + ch + 1];
        if (s1 <= s0) continue;
        used[b] = true;
        CK(cudaStreamWaitEvent(c->aux[b], c->ev_fork, 0));
        lm_launch_bucket<W>(a, wide, async, b, c->list + s0, (int)(s1 - s0), c->aux[b]);
      }
      int64_t h0 = ko[kHubBucket * P + ch] - hub0, h1 = ko[kHubBucket * P + ch + 1] - hub0;
      if (h1 > h0) {
        used[kHubBucket] = true;
        CK(cudaStreamWaitEvent(c->aux[kHubBucket], c->ev_fork, 0));
        LMArgs<W> ah = a;
        ah.hbase = c->gbase + h0;
        ah.spre = c->spre + h0;
        ah.hkid = c->hkid + h0;
        ah.hdone = c->hdone + h0;
        ah.hmoved = c->hmoved + h0;
        lm_launch_hubs<W>(ah, wide, async, c->list + hub0 + h0, (int)(h1 - h0), c->chunk_pre + h0,
                          hchunks[h1] - hchunks[h0], c->spre + h0, hschunks[h1] - hschunks[h0], c->aux[kHubBucket]);
      }
      // join
      for (int b = 0; b < kBuckets; ++b) {
        if (!used[b]) continue;
        CK(cudaEventRecord(c->ev_join[b], c->aux[b]));
        CK(cudaStreamWaitEvent(s, c->ev_join[b], 0));
      }
      if (!async) {
        int64_t cls = 0;
        for (int b = 0; b <= kHubBucket; ++b) cls += ko[b * P + ch + 1] - ko[b * P + ch];
        lm_launch_commit<W>(a, cls, s);
      }
      CKLAUNCH();
    }
    if (nhubs > 0 && a.prune) {
      LMArgs<W> am = a;
      am.hmoved = c->hmoved;
      lm_launch_hub_mark<W>(am, c->list + hub0, (int)nhubs, c->chunk_pre, hchunks[nhubs], s);
    }
    CK(cudaMemcpyAsync(c->h_ctr, c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
    if (multi) {
      CK(cudaMemcpyAsync(c->h_gmoves, c->d_gmoves, G * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
      CK(cudaMemcpyAsync(c->h_gs, c->d_gs, 2 * G * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    }
    return 0;
  };

  // stop_rule 1: each graph's Q numerator before the current iteration
  const bool recompute = c->opt.stop_rule == 1;
  std::vector<i128> nprev, nnow;
  if (recompute) {
    nprev.resize(G);
    nnow.resize(G);
    for (int64_t q = 0; q < G; ++q) nprev[q] = c->gst[q].qnum;
  }
  bool filtered = false;     // the lists hold only the last iteration's visits
  int64_t last_visited = 0;  // vertices the last iteration visited (all graphs)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  long long graph_launches = 0;   // kernels in the captured graph
  int it = 0;
  int rc = 0;
  for (; it < c->opt.max_iterations; ++it) {
    *c->h_iter = it;
    if ((rc = [&]() -> int {
           CK(cudaMemcpyAsync(c->d_iter, c->h_iter, sizeof(int), cudaMemcpyHostToDevice, s));
           return 0;
         }()))
      break;
    if (it > 0 && !small_pass) {
      const bool filter_now =
          c->opt.prune && full_len >= kFilterMinList && (double)last_visited < kFilterFraction * (double)full_len;
      if (reclass || filtered || filter_now) {
        if ((rc = classify(it, filter_now))) break;
        filtered = filter_now;
      }
    }
    // A small pass replays its iteration as a captured CUDA graph from the
    // second iteration on (all its launches are fixed for the pass); others
    // only with the cuda_graphs option and fixed classes.
    if ((small_pass && it >= 1) || (c->opt.cuda_graphs && !reclass && !c->opt.prune && it >= 2)) {
      if (!gexec) {
        if ((rc = [&]() -> int {
               CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
               return 0;
             }()))
          break;
        const long long l0 = launches_so_far();
        int r1 = iteration();
        cudaError_t e = cudaStreamEndCapture(s, &graph);
        graph_launches = launches_so_far() - l0;
        if (r1 || e != cudaSuccess) {
          cudaGetLastError();
          rc = r1 ? r1 : fail(c, LOUVAIN_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
          break;
        }
        if ((rc = [&]() -> int {
               CK(cudaGraphInstantiate(&gexec, graph, 0));
               return 0;
             }()))
          break;
      } else {
        add_launches(graph_launches);   // a replay runs the captured kernels again
      }
      if ((rc = [&]() -> int {
             CK(cudaGraphLaunch(gexec, s));
             return 0;
           }()))
        break;
    } else {
      if ((rc = iteration())) break;
    }
    if ((rc = [&]() -> int {
           CK(cudaStreamSynchronize(s));
           return 0;
         }()))
      break;
    if (c->h_ctr->error) {
      rc = fail(c, LOUVAIN_ERR_INTERNAL, "local-moving: hash table overflow");
      break;
    }
    edges_total += (int64_t)c->h_ctr->edges;
    visited_total += (int64_t)c->h_ctr->visited;
    last_visited = (int64_t)c->h_ctr->visited;
    cands_total += (int64_t)c->h_ctr->cands;
    bool any_on = false;
    if (recompute)
      if ((rc = q_numerators<W>(c, g, nnow))) break;
    if (!multi) {
      const u128 S = ((u128)c->h_ctr->s_hi << 64) | (u128)c->h_ctr->s_lo;
      const int64_t mv = (int64_t)c->h_ctr->moves;
      c->iters.push_back(IterRec{pass, mv, S});
      c->gst[0].pass_moves += mv;
      c->gst[0].pass_iters++;
      if (recompute) {
        any_on = !(dbl(nnow[0] - nprev[0]) / dbl((i128)c->M * c->M) <= tol);
        nprev[0] = nnow[0];
      } else {
        any_on = !((2.0 * (double)S) / dbl((i128)c->M * c->M) <= tol);
      }
    } else {
      u128 Stot = 0;
      int64_t mvtot = 0;
      for (int64_t q = 0; q < G; ++q) {
        if (!c->h_gon[q]) continue;
        GraphState& st = c->gst[q];
        const u128 S = ((u128)c->h_gs[2 * q + 1] << 64) | (u128)c->h_gs[2 * q];
        const int64_t mv = (int64_t)c->h_gmoves[q];
        st.iters.push_back(IterRec{pass, mv, S});
        st.pass_moves += mv;
        st.pass_iters++;
        Stot += S;
        mvtot += mv;
        bool settled;
        if (recompute) {
          settled = dbl(nnow[q] - nprev[q]) / dbl((i128)st.M * st.M) <= tol;
          nprev[q] = nnow[q];
        } else {
          settled = (2.0 * (double)S) / dbl((i128)st.M * st.M) <= tol;
        }
        if (settled) c->h_gon[q] = 0;
        else any_on = true;
      }
      c->iters.push_back(IterRec{pass, mvtot, Stot});

      if (any_on)
        if ((rc = [&]() -> int {
               CK(cudaMemcpyAsync(c->d_gon, c->h_gon, G * sizeof(int32_t), cudaMemcpyHostToDevice, s));
               return 0;
             }()))
          break;
    }
    if (!any_on) {
      ++it;
      break;
    }
  }
  if (gexec) cudaGraphExecDestroy(gexec);
  if (graph) cudaGraphDestroy(graph);
  if (rc) return rc;
  *iters_out = it;
  *edges_out = edges_total;
  *visited_out = visited_total;
  c->lm_cands += cands_total;
  return 0;
}

// Exact Q numerator of every graph's current membership on the pass graph.
template <typename W>
int q_numerators(louvain_ctx* c, const PassState& g, std::vector<i128>& out) {
  cudaStream_t s = c->stream;
  if (c->G == 1) {
    CK(cudaMemsetAsync(c->acc, 0, 4 * sizeof(unsigned long long), s));
    modularity_parts<W>(g.off, g.col, (const W*)g.w, g.n, g.nnz, c->memb, c->sig, c->acc, c->crow, s);
    CKLAUNCH();
    if (int r = fetch(c, c->h_acc, c->acc, 4 * sizeof(unsigned long long))) return r;
    u128 L = ((u128)c->h_acc[3] << 64) | (u128)c->h_acc[0];
    u128 SS = ((u128)c->h_acc[2] << 64) | (u128)c->h_acc[1];
    out[0] = (i128)c->M * (i128)L - (i128)SS;
    return 0;
  }
  const int64_t G = c->G;
  CK(cudaMemsetAsync(c->d_gL, 0, 2 * G * sizeof(unsigned long long), s));
  CK(cudaMemsetAsync(c->d_gSS, 0, 2 * G * sizeof(unsigned long long), s));
  graph_modularity_parts<W>(g.off, g.col, (const W*)g.w, g.n, g.nnz, c->memb, c->sig, c->gid, c->d_gL, c->d_gSS,
                            c->crow, s);
  CKLAUNCH();
  if (int r = fetch_pair(c, c->h_gL, c->d_gL, 2 * G * sizeof(unsigned long long), c->h_gSS, c->d_gSS,
                         2 * G * sizeof(unsigned long long)))
    return r;
  for (int64_t q = 0; q < G; ++q) {
    u128 L = ((u128)c->h_gL[2 * q + 1] << 64) | (u128)c->h_gL[2 * q];
    u128 SS = ((u128)c->h_gSS[2 * q + 1] << 64) | (u128)c->h_gSS[2 * q];
    out[q] = (i128)c->gst[q].M * (i128)L - (i128)SS;
  }
  return 0;
}

template <typename W, typename W2>
int aggregate(louvain_ctx* c, const PassState& g, int64_t k, PassState* next, std::vector<i128>& nafter) {
  cudaStream_t s = c->stream;
  const bool multi = c->G > 1;
  const int64_t G = c->G;
  const int dst = g.widx == 0 ? 1 : 0;
  coarse_degrees(c->used, c->newid, c->sig, g.n, c->Knext, s);
  agg_group_members(c->level, g.n, k, c->cnt, c->cstart, c->fill, c->members, c->inv, c->tmp, s);
  agg_member_prefix(g.off, c->members, g.n, c->mdeg, c->mpre, c->tmp, s);
  agg_relabel<W, W2>(g.off, g.col, (const W*)g.w, g.n, g.nnz, c->level, c->inv, c->mpre, c->crow, c->tcol,
                     (W2*)c->tw, s);
  agg_keys(c->cstart, c->mpre, k, c->key, s);
  stable_partition(c->key, k, kAggBuckets + 1, c->list, c->key_off, c->tmp, s);
  CKLAUNCH();
  int64_t ko[kAggBuckets + 2];
  if (int r = fetch(c, ko, c->key_off, sizeof(ko))) return r;
  CK(cudaMemsetAsync(c->flags, 0, sizeof(int), s));
  AggArgs a;
  memset(&a, 0, sizeof(a));
  a.off = g.off;
  a.col = g.col;
  a.wt = g.w;
  a.level = c->level;
  a.n = g.n;
  a.k = k;
  a.cstart = c->cstart;
  a.members = c->members;
  a.mpre = c->mpre;
  a.tcol = c->tcol;
  a.tw = c->tw;
  a.rlen = c->rlen;
  a.gkeys = c->gkeys;
  a.gvals = c->gvals;
  a.lsum = c->acc + 6;
  a.glo = c->glo;
  a.error = c->flags;
  // communities whose members have no edge get empty rows
  CK(cudaMemsetAsync(c->rlen, 0, (k + 1) * sizeof(int64_t), s));
  CK(cudaMemsetAsync(c->acc, 0, 8 * sizeof(unsigned long long), s));
  if (multi) {
    a.cgid = c->gid_next;
    a.glsum = c->d_gL;
    CK(cudaMemsetAsync(c->d_gL, 0, 2 * G * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(c->d_gSS, 0, 2 * G * sizeof(unsigned long long), s));
    graph_squares(c->sig, c->gid, g.n, c->d_gSS, s);
  } else {
    sum_squares(c->sig, g.n, c->acc + 4, s);   // sum of Sigma_c^2 for the pass's Q numerator
  }
  for (int b = 0; b < kAggGlobal; ++b)
    agg_launch_bucket<W, W2>(a, b, c->list + ko[b], (int)(ko[b + 1] - ko[b]), s);
  const int64_t ng = ko[kAggGlobal + 1] - ko[kAggGlobal];
  if (ng > 0) {
    agg_global_layout(c->cstart, c->mpre, c->list + ko[kAggGlobal], ng, k, multi ? c->gid_next : nullptr,
                      multi ? c->vo_next : nullptr, c->gbase, c->chunk_pre, c->spre, c->glo, c->tmp, s);
    int64_t nchunks = 0, nschunks = 0;
    CKLAUNCH();
    if (int r = fetch_pair(c, &nchunks, c->chunk_pre + ng, sizeof(int64_t), &nschunks, c->spre + ng, sizeof(int64_t)))
      return r;
    agg_launch_global<W, W2>(a, c->list + ko[kAggGlobal], (int)ng, c->gbase, c->chunk_pre, nchunks, c->spre,
                             nschunks, s);
  }
  CKLAUNCH();
  // coarse offsets = scan of row lengths, written straight into the next graph
  scan_i64(c->rlen, c->offX[dst], k, c->offX[dst] + k, c->tmp, s);
  CKLAUNCH();
  // the coarse row count, the overflow flag and the Q numerator's parts
  // (complete: the kernels that sum them ran before the scan) in one read
  int64_t nnz2 = 0;
  int flag = 0;
  if (!multi) {
    if (int r = fetch_many(c, {{&nnz2, c->offX[dst] + k, sizeof(int64_t)}, {&flag, c->flags, sizeof(int)},
                               {c->h_acc, c->acc, 8 * sizeof(unsigned long long)}}))
      return r;
  } else {
    if (int r = fetch_many(c, {{&nnz2, c->offX[dst] + k, sizeof(int64_t)}, {&flag, c->flags, sizeof(int)},
                               {c->h_gL, c->d_gL, 2 * G * sizeof(unsigned long long)},
                               {c->h_gSS, c->d_gSS, 2 * G * sizeof(unsigned long long)}}))
      return r;
  }
  if (flag) return fail(c, LOUVAIN_ERR_INTERNAL, "aggregation: hash table overflow");
  agg_compact<W2>(c->cstart, c->mpre, c->offX[dst], k, nnz2, c->crow, c->tcol, (const W2*)c->tw, c->colX[dst],
                  (W2*)c->wX[dst], s);
  CKLAUNCH();
  // Q numerator after the pass: M * sum_C L_C (coarse self-loops) - sum_c Sigma_c^2
  if (!multi) {
    u128 SS = ((u128)c->h_acc[5] << 64) | (u128)c->h_acc[4];
    nafter[0] = (i128)c->M * (i128)c->h_acc[6] - (i128)SS;
  } else {
    for (int64_t q = 0; q < G; ++q) {
      u128 L = ((u128)c->h_gL[2 * q + 1] << 64) | (u128)c->h_gL[2 * q];
      u128 SS = ((u128)c->h_gSS[2 * q + 1] << 64) | (u128)c->h_gSS[2 * q];
      nafter[q] = (i128)c->gst[q].M * (i128)L - (i128)SS;
    }
  }
  next->n = k;
  next->nnz = nnz2;
  next->off = c->offX[dst];
  next->col = c->colX[dst];
  next->w = (void*)c->wX[dst];
  next->widx = dst;
  return 0;
}

template <typename W2>
int record_coarse(louvain_ctx* c, PassRec& pr, const PassState& h) {
  pr.coff.resize(h.n + 1);
  pr.ccol.resize(h.nnz);
  pr.cw.resize(h.nnz);
  std::vector<W2> w(h.nnz);
  CK(cudaMemcpyAsync(pr.coff.data(), h.off, (h.n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  if (h.nnz) {
    CK(cudaMemcpyAsync(pr.ccol.data(), h.col, h.nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(w.data(), h.w, h.nnz * sizeof(W2), cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  for (int64_t i = 0; i < h.nnz; ++i) pr.cw[i] = (int64_t)w[i];
  return 0;
}

// After pass 0: if enough communities of the coarse graph are isolated
// (empty rows: communities of vertices without entries, which never move),
// the later pass graphs leave them out.  Every other coarse vertex keeps its
// order (compact id = rank among the non-empty rows); the columns are
// renumbered in place, the offsets, degrees (c->Knext) and graph ids (batch)
// compacted, top[] takes compact ids (an isolated community: -1 - its rank
// among the isolated ones) and isob the isolated count before each compact
// vertex.  finalize_top puts top[] back in the full numbering at the end.
constexpr int64_t kCompactMinIsolated = 1024;   // and at least 1/16 of the coarse vertices
int compact_coarse(louvain_ctx* c, PassState* next, int64_t k, const std::vector<int64_t>& vo_full) {
  cudaStream_t s = c->stream;
  const bool multi = c->G > 1;
  const int64_t G = c->G;
  int32_t* flag = c->used;    // free: the renumbering and the coarse degrees are done
  int32_t* pos = c->newid;
  nonempty_rows(next->off, k, flag, s);
  scan_i32(flag, pos, k, c->scal, c->tmp, s);
  CKLAUNCH();
  int64_t kc = 0;
  if (int r = fetch(c, &kc, c->scal, sizeof(int64_t))) return r;
  const int64_t z = k - kc;
  if (z < kCompactMinIsolated || z * 16 < k) return 0;
  compact_rows(next->off, k, next->nnz, flag, pos, c->Knext, multi ? c->gid_next : nullptr, c->cnt, c->K,
               multi ? c->gid : nullptr, c->isob[0], next->col, c->top, c->n0, s);
  c->h_scal[0] = next->nnz;
  CK(cudaMemcpyAsync(c->cnt + kc, c->h_scal, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(next->off, c->cnt, (kc + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  std::swap(c->K, c->Knext);   // the run swaps them back: the next pass's degrees are the compact ones
  c->h_zg.assign(G, 0);
  if (multi) {
    std::swap(c->gid, c->gid_next);   // the pass swaps them back: gid_next holds the compact graph ids
    compact_vo(c->vo_next, G, pos, k, kc, c->vo, s);
    CKLAUNCH();
    std::vector<int64_t> vo_c(G + 1), zpre(G + 1);
    if (int r = fetch(c, vo_c.data(), c->vo, (G + 1) * sizeof(int64_t))) return r;
    for (int64_t q = 0; q <= G; ++q) zpre[q] = vo_full[q] - vo_c[q];
    for (int64_t q = 0; q < G; ++q) c->h_zg[q] = zpre[q + 1] - zpre[q];
    CK(cudaMemcpyAsync(c->d_zpre, zpre.data(), (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->vo_next, c->vo, (G + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c->vo_top, c->vo, (G + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
  } else {
    c->h_zg[0] = z;
  }
  CKLAUNCH();
  next->n = kc;
  c->compacted = true;
  c->iso_z = z;
  c->isob_cur = 0;
  c->kc_top = kc;
  return 0;
}

// A compact pass's recorded level and coarse graph in the full numbering
// (parity dumps only): the pass graph had n compact vertices, its level k
// compact communities; isob[isob_cur ^ 1] and isob[isob_cur] hold the
// isolated counts before them.
int record_full_numbering(louvain_ctx* c, PassRec& pr, int64_t n, int64_t k) {
  const int64_t z = c->iso_z;
  std::vector<int32_t> before(n), after(k);
  if (n) CK(cudaMemcpyAsync(before.data(), c->isob[c->isob_cur ^ 1], n * sizeof(int32_t), cudaMemcpyDeviceToHost,
                            c->stream));
  if (k) CK(cudaMemcpyAsync(after.data(), c->isob[c->isob_cur], k * sizeof(int32_t), cudaMemcpyDeviceToHost,
                            c->stream));
  CK(cudaStreamSynchronize(c->stream));
  // full id of the r-th isolated community after the renumbering
  auto iso_id = [&](int64_t r) -> int32_t {
    const int64_t j = std::upper_bound(after.begin(), after.end(), (int32_t)r) - after.begin();
    return (int32_t)(j + r);
  };
  if (!pr.level.empty()) {
    std::vector<int32_t> full(n + z);
    int64_t j = 0;
    for (int64_t x = 0; x < n + z; ++x) {
      if (j < n && j + before[j] == x) {
        const int32_t L = pr.level[j++];
        full[x] = L + after[L];
      } else {
        full[x] = iso_id(x - j);
      }
    }
    pr.level.swap(full);
  }
  if (pr.info.coarse_built) {
    std::vector<int64_t> off(k + z + 1, 0);
    std::vector<int32_t> col(pr.ccol.size());
    int64_t j = 0;
    for (int64_t R = 0; R < k + z; ++R) {
      int64_t len = 0;
      if (j < k && j + after[j] == R) {
        len = pr.coff[j + 1] - pr.coff[j];
        for (int64_t x = pr.coff[j]; x < pr.coff[j + 1]; ++x) col[x] = pr.ccol[x] + after[pr.ccol[x]];
        ++j;
      }
      off[R + 1] = off[R] + len;
    }
    pr.coff.swap(off);
    pr.ccol.swap(col);
  }
  return 0;
}

// One pass on graph g (weights W), coarse graphs use W2.  Every graph that
// has not stopped takes part; a graph stops after a pass with no move, a
// pass whose gain is <= pass_tolerance, or the last pass.  Returns 0 and sets
// *stop when every graph has stopped; otherwise *next holds the coarse graph.
template <typename W, typename W2>
int run_pass(louvain_ctx* c, const PassState& g, int pass, double* tol, bool wide, bool* stop, PassState* next) {
  cudaStream_t s = c->stream;
  const bool multi = c->G > 1;
  const int64_t G = c->G;
  PassRec pr;
  memset(&pr.info, 0, sizeof(pr.info));
  const int64_t iso = c->compacted ? c->iso_z : 0;   // isolated communities outside the pass graph
  pr.info.n = g.n + iso;
  pr.info.nnz = g.nnz;
  CK(cudaEventRecord(c->ev[0], s));
  // pass 0 of louvain_run_from starts from the caller's membership (in memb)
  const bool warm = pass == 0 && c->warm;
  if (warm) {
    CK(cudaMemsetAsync(c->flags, 0, sizeof(int), s));
    pass_init_from(g.n, c->K, c->memb, c->sig, c->csize, c->stamp[0], c->stamp[1], multi ? c->gid : nullptr,
                   multi ? c->vo : nullptr, c->flags, s);
    CKLAUNCH();
    int flag = 0;
    if (int r = fetch(c, &flag, c->flags, sizeof(int))) return r;
    if (flag) return fail(c, LOUVAIN_ERR_INVALID_ARG, "initial membership: an id outside its graph's vertex range");
    std::vector<i128> n0(G, 0);
    if (int r = q_numerators<W>(c, g, n0)) return r;
    for (int64_t q = 0; q < G; ++q) c->gst[q].qnum = n0[q];
  } else {
    pass_init(g.n, c->K, c->memb, c->sig, c->csize, c->stamp[0], c->stamp[1], s);
  }
  CKLAUNCH();
  const i128 nbefore = c->gst[0].qnum;
  int64_t edges = 0, visited = 0;
  int iters = 0;
  CK(cudaEventRecord(c->ev[1], s));
  if (int r = local_moving<W>(c, g, pass, *tol, wide, &iters, &edges, &visited)) return r;
  CK(cudaEventRecord(c->ev[2], s));
  int64_t pmoves = 0;
  for (int64_t q = 0; q < G; ++q) pmoves += c->gst[q].pass_moves;
  pr.info.moves = pmoves;
  pr.info.iterations = iters;
  pr.info.n_before_hi = (int64_t)(nbefore >> 64);
  pr.info.n_before_lo = (uint64_t)nbefore;
  c->stats.lm_edges += edges;
  // algorithmic bytes of local-moving: per scanned entry its column, weight
  // and neighbour membership; per visited vertex two offsets, its membership,
  // degree, own community total and activity stamp (32 B)
  c->stats.lm_vertices += visited;
  // + per distinct candidate community its total Sigma_c (8), per move the two
  // totals it updates (16)
  const int64_t cands = c->lm_cands - c->stats.lm_candidates;
  c->stats.lm_candidates = c->lm_cands;
  c->stats.lm_bytes += edges * (int64_t)(4 + sizeof(W) + 4) + visited * 32 + cands * 8 + pmoves * 16;
  c->stats.moves += pmoves;
  c->stats.iterations += iters;
  c->stats.passes = pass + 1;
  for (int64_t q = 0; q < G; ++q)
    if (!c->gst[q].stopped) c->gst[q].passes++;
  float ms_init = 0, ms_lm = 0;
  if (pmoves == 0 && !warm) {
    // no graph moved: every graph stops, nothing to renumber
    CK(cudaEventSynchronize(c->ev[2]));
    cudaEventElapsedTime(&ms_init, c->ev[0], c->ev[1]);
    cudaEventElapsedTime(&ms_lm, c->ev[1], c->ev[2]);
    pr.info.k = g.n + iso;
    pr.info.n_after_hi = pr.info.n_before_hi;
    pr.info.n_after_lo = pr.info.n_before_lo;
    pr.info.lm_ms = ms_lm;
    c->stats.lm_ms += ms_lm;
    c->stats.other_ms += ms_init;
    c->passes.push_back(std::move(pr));
    for (int64_t q = 0; q < G; ++q) c->gst[q].stopped = true;
    *stop = true;
    return 0;
  }
  // renumber by ascending old id and compose the top level; with several
  // graphs each graph's communities stay contiguous and in order
  mark_used(c->memb, g.n, c->used, s);
  scan_i32(c->used, c->newid, g.n, c->scal, c->tmp, s);
  apply_level(c->memb, c->newid, g.n, c->level, s);
  compose_top(c->top, c->n0, c->level, s);
  if (multi) {
    CK(cudaMemsetAsync(c->kcount, 0, (G + 1) * sizeof(int64_t), s));
    graph_renumber(c->used, c->newid, c->gid, g.n, c->kcount, c->gid_next, s);
    scan_i64(c->kcount, c->vo_next, G, c->vo_next + G, c->tmp, s);
    CK(cudaMemcpyAsync(c->vo_top, c->vo_next, (G + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  }
  if (c->compacted) {
    carry_isob(c->used, c->newid, c->isob[c->isob_cur], g.n, c->isob[c->isob_cur ^ 1], s);
    c->isob_cur ^= 1;
  }
  CKLAUNCH();
  int64_t k = 0;
  std::vector<int64_t> vo_next;
  if (multi) {
    vo_next.resize(G + 1);
    if (int r = fetch_pair(c, &k, c->scal, sizeof(int64_t), vo_next.data(), c->vo_next, (G + 1) * sizeof(int64_t)))
      return r;
  } else {
    if (int r = fetch(c, &k, c->scal, sizeof(int64_t))) return r;
  }
  if (c->compacted) c->kc_top = k;
  // If another pass may follow, aggregate first: the coarse self-loops give
  // sum_C L_C, so the pass's Q numerators cost no extra scan of the graph; a
  // coarse graph built for a pass after which every graph stops is dropped.
  std::vector<i128> nafter(G, 0);
  bool built = false;
  if (pass + 1 < c->opt.max_passes) {
    if (int r = aggregate<W, W2>(c, g, k, next, nafter)) return r;
    built = true;
  } else {
    if (int r = q_numerators<W>(c, g, nafter)) return r;
  }
  CK(cudaEventRecord(c->ev[3], s));
  bool all_stopped = true;
  for (int64_t q = 0; q < G; ++q) {
    GraphState& st = c->gst[q];
    if (st.stopped) continue;
    if (st.pass_moves == 0 && !warm) {
      st.stopped = true;   // its level is the identity: nothing changes
    } else {
      const i128 gain = nafter[q] - st.qnum;
      st.qnum = nafter[q];
      st.k = (multi ? vo_next[q + 1] - vo_next[q] : k) + (c->compacted ? c->h_zg[q] : 0);
      st.stopped = dbl(gain) / dbl((i128)st.M * st.M) <= c->opt.pass_tolerance || pass + 1 == c->opt.max_passes;
    }
    all_stopped = all_stopped && st.stopped;
  }
  pr.info.k = k + iso;
  pr.info.n_after_hi = (int64_t)(c->gst[0].qnum >> 64);
  pr.info.n_after_lo = (uint64_t)c->gst[0].qnum;
  pr.info.level_recorded = c->opt.record_levels ? 1 : 0;
  if (c->opt.record_levels) {
    pr.level.resize(g.n);
    CK(cudaMemcpyAsync(pr.level.data(), c->level, g.n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  }
  *stop = all_stopped;
  float ms_agg = 0;
  CK(cudaEventSynchronize(c->ev[3]));
  cudaEventElapsedTime(&ms_agg, c->ev[2], c->ev[3]);
  if (!*stop && built) {
    pr.info.coarse_built = 1;
    pr.info.coarse_nnz = next->nnz;
    if (c->opt.record_levels)
      if (int r = record_coarse<W2>(c, pr, *next)) return r;
    *tol = *tol / c->opt.tolerance_decline;
    if (pass == 0 && !c->compacted && c->iso0 >= kCompactMinIsolated)
      if (int r = compact_coarse(c, next, k, vo_next)) return r;
    if (multi) {
      std::swap(c->gid, c->gid_next);
      std::swap(c->vo, c->vo_next);
    }
  }
  if (c->opt.record_levels && iso > 0)
    if (int r = record_full_numbering(c, pr, g.n, k)) return r;
  cudaEventElapsedTime(&ms_init, c->ev[0], c->ev[1]);
  cudaEventElapsedTime(&ms_lm, c->ev[1], c->ev[2]);
  pr.info.lm_ms = ms_lm;
  pr.info.agg_ms = ms_agg;
  c->stats.lm_ms += ms_lm;
  c->stats.agg_ms += ms_agg;
  c->stats.other_ms += ms_init;
  c->passes.push_back(std::move(pr));
  return 0;
}

// Per-run state of pass 0: degrees, M and the singleton numerators were
// found when the graph was loaded.
int init_run_state(louvain_ctx* c) {
  cudaStream_t s = c->stream;
  const int64_t G = c->G;
  c->iters.clear();
  c->passes.clear();
  CK(cudaMemcpyAsync(c->K, c->K0, c->n0 * sizeof(long long), cudaMemcpyDeviceToDevice, s));
  c->M = c->M0;
  for (int64_t q = 0; q < G; ++q) {
    GraphState& st = c->gst[q];
    st.M = c->gM0[q];
    st.qnum = c->gqnum0[q];
    st.stopped = st.M == 0;      // a graph without edges never moves
    st.k = c->gn0[q];
    st.passes = 0;
    st.iters.clear();
  }
  if (G > 1) {
    c->gid = c->gid_a;
    c->gid_next = c->gid_b;
    c->vo = c->vo_a;
    c->vo_next = c->vo_b;
    CK(cudaMemcpyAsync(c->gid, c->gid0, c->n0 * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c->vo, c->vo0, (G + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c->vo_top, c->vo0, (G + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
  }
  return 0;
}

int run_all(louvain_ctx* c) {
  cudaStream_t s = c->stream;
  const int64_t G = c->G;
  memset(&c->stats, 0, sizeof(c->stats));
  c->lm_cands = 0;
  c->Q = 0;
  const long long launches0 = launches_so_far();
  CK(cudaEventRecord(c->ev[6], s));
  iota_i32(c->top, c->n0, s);
  if (int r = init_run_state(c)) return r;
  c->compacted = false;
  c->iso_z = 0;
  c->isob_cur = 0;
  c->kc_top = 0;
  c->h_zg.assign(G, 0);
  const bool wide = c->M >= (1ll << 31);           // M^2 >= 2^62: 128-bit gains
  const bool coarse64 = c->M >= (1ll << 31) - 1;   // coarse weights can exceed int32
  PassState g{c->n0, c->nnz0, c->off0, c->col0, (void*)c->w0, -1};
  double tol = c->opt.tolerance;
  auto any_running = [&]() {
    for (int64_t q = 0; q < G; ++q)
      if (!c->gst[q].stopped) return true;
    return false;
  };
  for (int p = 0; p < c->opt.max_passes && any_running(); ++p) {
    bool stop = false;
    PassState next{};
    int r;
    if (g.widx < 0)
      r = coarse64 ? run_pass<int32_t, int64_t>(c, g, p, &tol, wide, &stop, &next)
                   : run_pass<int32_t, int32_t>(c, g, p, &tol, wide, &stop, &next);
    else
      r = coarse64 ? run_pass<int64_t, int64_t>(c, g, p, &tol, wide, &stop, &next)
                   : run_pass<int32_t, int32_t>(c, g, p, &tol, wide, &stop, &next);
    if (r) return r;
    if (stop) break;
    std::swap(c->K, c->Knext);
    g = next;
  }
  if (c->compacted) {   // top[] back in the full numbering
    finalize_top(c->top, c->n0, c->isob[c->isob_cur], c->kc_top, G > 1 ? c->vo_top : nullptr, c->d_zpre, G, s);
    CKLAUNCH();
  }
  CK(cudaEventRecord(c->ev[7], s));
  CK(cudaEventSynchronize(c->ev[7]));
  float tot = 0;
  cudaEventElapsedTime(&tot, c->ev[6], c->ev[7]);
  c->stats.total_ms = tot;
  int64_t comms = 0;
  for (int64_t q = 0; q < G; ++q) comms += c->gst[q].k;
  c->qnum = c->gst[0].qnum;
  c->Q = c->M == 0 ? 0.0 : dbl(c->qnum) / dbl((i128)c->M * c->M);
  c->stats.q = G == 1 ? c->Q : 0.0;
  c->stats.communities = comms;
  c->stats.kernel_launches = launches_so_far() - launches0;
  return 0;
}

// Device time of the first local-moving iteration of pass 0 under mapping th
// (the run's own mode, classes and options; the state is reset by the next run).
int tune_trial(louvain_ctx* c, const LMThresholds& th, float* ms) {
  cudaStream_t s = c->stream;
  if (int r = init_run_state(c)) return r;
  c->thr = th;
  PassState g{c->n0, c->nnz0, c->off0, c->col0, (void*)c->w0, -1};
  const bool wide = c->M >= (1ll << 31);
  pass_init(g.n, c->K, c->memb, c->sig, c->csize, c->stamp[0], c->stamp[1], s);
  CKLAUNCH();
  int iters = 0;
  int64_t edges = 0, visited = 0;
  CK(cudaEventRecord(c->ev[0], s));
  if (int r = local_moving<int32_t>(c, g, 0, c->opt.tolerance, wide, &iters, &edges, &visited)) return r;
  CK(cudaEventRecord(c->ev[1], s));
  CK(cudaEventSynchronize(c->ev[1]));
  cudaEventElapsedTime(ms, c->ev[0], c->ev[1]);
  return 0;
}

// Coordinate descent over the local-moving degree thresholds, from the
// current mapping: each threshold in turn takes each of its candidate values
// (within its kernel's capacity and between its neighbours) and keeps the
// fastest first iteration (best of two trials, at least 2% faster to change).
int autotune(louvain_ctx* c, float* best_ms) {
  static const int32_t cand[5][3] = {{4, 8, 0}, {16, 32, 0}, {64, 128, 0}, {256, 512, 1024}, {2048, 4096, 0}};
  const louvain_options saved = c->opt;
  c->opt.max_iterations = 1;
  LMThresholds best = c->thr;
  auto timed = [&](const LMThresholds& th, float* out) -> int {
    float t0 = 0, t1 = 0;
    if (int r = tune_trial(c, th, &t0)) return r;
    if (int r = tune_trial(c, th, &t1)) return r;
    *out = std::min(t0, t1);
    return 0;
  };
  float bms = 0;
  int rc = timed(best, &bms);
  for (int b = 0; b < 5 && !rc; ++b) {
    for (int k = 0; k < 3 && !rc; ++k) {
      const int32_t v = cand[b][k];
      if (v <= 0 || v == best.t[b] || v > kLMCap[b]) continue;
      if ((b > 0 && v <= best.t[b - 1]) || (b < 4 && v >= best.t[b + 1])) continue;
      LMThresholds th = best;
      th.t[b] = v;
      float ms = 0;
      rc = timed(th, &ms);
      if (!rc && ms < 0.98f * bms) {
        best = th;
        bms = ms;
      }
    }
  }
  c->opt = saved;
  c->thr = best;
  c->ran = false;
  if (best_ms) *best_ms = bms;
  return rc;
}

}  // namespace

// Device arena for graphs of up to n vertices and nnz entries (every buffer
// is sized by one of the two); reused by later loads that fit.
int alloc_arena(louvain_ctx* c, int64_t n, int64_t nnz) {
  free_all(c);
  const int64_t N1 = n + 1;
  ALLOC(c->off0, N1);
  ALLOC(c->col0, nnz);
  ALLOC(c->w0, nnz);
  for (int i = 0; i < 2; ++i) {
    ALLOC(c->offX[i], N1);
    ALLOC(c->colX[i], nnz);
    ALLOC(c->wX[i], nnz * 8);   // bytes
  }
  ALLOC(c->K0, n);
  ALLOC(c->K, n);
  ALLOC(c->Knext, n);
  ALLOC(c->memb, n);
  ALLOC(c->sig, n);
  ALLOC(c->csize, n);
  ALLOC(c->stamp[0], n);
  ALLOC(c->stamp[1], n);
  ALLOC(c->key, n);
  ALLOC(c->list, n);
  ALLOC(c->used, n);
  ALLOC(c->newid, n);
  ALLOC(c->level, n);
  ALLOC(c->top, n);
  ALLOC(c->moves, n);
  ALLOC(c->key_off, kBuckets * 64 + 8);
  ALLOC(c->cnt, N1);
  ALLOC(c->cstart, N1);
  ALLOC(c->fill, N1);
  ALLOC(c->members, n);
  ALLOC(c->inv, n);
  ALLOC(c->crow, (n + nnz) / kRelabelChunk + 3);
  ALLOC(c->mdeg, n);
  ALLOC(c->mpre, N1);
  ALLOC(c->rlen, N1);
  ALLOC(c->tcol, nnz);
  ALLOC(c->tw, nnz * 8);
  ALLOC(c->gkeys, 2 * nnz);
  ALLOC(c->gvals, 2 * nnz);
  ALLOC(c->gbase, N1);
  ALLOC(c->chunk_pre, N1);
  ALLOC(c->spre, N1);
  ALLOC(c->glo, N1);
  ALLOC(c->hkid, N1);
  ALLOC(c->hdone, N1);
  ALLOC(c->hmoved, N1);
  // slot chunks of all hubs: sum of ceil(2 deg / kSlotChunk) <= 2 nnz / kSlotChunk + #hubs
  c->npart = 2 * nnz / kSlotChunk + n + 16;   // every hub has at least one slot chunk
  ALLOC(c->hpart, 2 * c->npart);
  ALLOC(c->hpart_c, c->npart);
  {
    size_t t1 = partition_tmp_bytes(n, kBuckets * 64 + 1);
    size_t t2 = (size_t)N1 * 24 + scan_tmp_bytes(N1);
    size_t t3 = scan_tmp_bytes(nnz + 1);
    c->tmp_bytes = std::max(t1, std::max(t2, t3));
    ALLOC(c->tmp, (int64_t)c->tmp_bytes);
  }
  ALLOC(c->ctr, 1);
  ALLOC(c->acc, 8);
  ALLOC(c->flags, 4);
  ALLOC(c->d_iter, 4);
  ALLOC(c->scal, 16);
  ALLOC(c->isob[0], n);
  ALLOC(c->isob[1], n);
  ALLOC(c->d_zpre, N1 + 1);
  ALLOC(c->gid0, n);
  ALLOC(c->gid_a, n);
  ALLOC(c->gid_b, n);
  ALLOC(c->vo0, N1 + 1);
  ALLOC(c->vo_a, N1 + 1);
  ALLOC(c->vo_b, N1 + 1);
  ALLOC(c->vo_top, N1 + 1);
  ALLOC(c->kcount, N1 + 1);
  ALLOC(c->d_Mg, N1);
  ALLOC(c->d_gon, N1);
  ALLOC(c->d_gcat, N1);
  ALLOC(c->d_gmoves, N1);
  ALLOC(c->d_gs, 2 * N1);
  ALLOC(c->d_gL, 2 * N1);
  ALLOC(c->d_gSS, 2 * N1);
  c->cap_n = n;
  c->cap_nnz = nnz;
  c->tables_dirty = true;
  return 0;
}

void free_host_graph_buffers(louvain_ctx* c) {
  if (c->h_gon) cudaFreeHost(c->h_gon);
  if (c->h_gmoves) cudaFreeHost(c->h_gmoves);
  if (c->h_gs) cudaFreeHost(c->h_gs);
  if (c->h_gL) cudaFreeHost(c->h_gL);
  if (c->h_gSS) cudaFreeHost(c->h_gSS);
  c->h_gon = nullptr;
  c->h_gmoves = c->h_gs = c->h_gL = c->h_gSS = nullptr;
  c->hcap = 0;
}

int host_graph_buffers(louvain_ctx* c, int64_t G) {
  if (c->hcap >= G) return 0;
  free_host_graph_buffers(c);
  if (cudaMallocHost(&c->h_gon, G * sizeof(int32_t)) != cudaSuccess ||
      cudaMallocHost(&c->h_gmoves, G * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMallocHost(&c->h_gs, 2 * G * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMallocHost(&c->h_gL, 2 * G * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMallocHost(&c->h_gSS, 2 * G * sizeof(unsigned long long)) != cudaSuccess) {
    free_host_graph_buffers(c);
    return fail(c, LOUVAIN_ERR_OOM, "pinned host allocation failed");
  }
  c->hcap = G;
  return 0;
}

// ================================================================== C ABI

extern "C" {

int louvain_default_options(louvain_options* o) {
  if (!o) return LOUVAIN_ERR_INVALID_ARG;
  memset(o, 0, sizeof(*o));
  o->mode = LOUVAIN_SYNC;
  o->tolerance = 0.01;
  o->tolerance_decline = 10.0;
  o->pass_tolerance = 0.0;
  o->max_iterations = 20;
  o->max_passes = 10;
  o->prune = 0;
  o->singleton_guard = 1;
  o->subrounds = 0;
  o->validate = 1;
  o->record_levels = 0;
  o->cuda_graphs = 0;
  o->reclass = 3;
  o->bucket_streams = 1;
  o->colour_classes = 0;
  o->stop_rule = 0;
  return 0;
}

int louvain_create(louvain_ctx** out, const louvain_options* opt, int device, void* cuda_stream) {
  if (!out) return LOUVAIN_ERR_INVALID_ARG;
  *out = nullptr;
  louvain_ctx* c = new louvain_ctx();
  if (opt) c->opt = *opt; else louvain_default_options(&c->opt);
  if (check_options(&c->opt)) { delete c; return LOUVAIN_ERR_INVALID_ARG; }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    delete c;
    return LOUVAIN_ERR_CUDA;
  }
  c->device = device;
  if (cudaSetDevice(device) != cudaSuccess) { delete c; return LOUVAIN_ERR_CUDA; }
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return LOUVAIN_ERR_CUDA; }
    c->own_stream = true;
  }
  for (auto& e : c->ev)
    if (cudaEventCreate(&e) != cudaSuccess) { delete c; return LOUVAIN_ERR_CUDA; }
  // Bucket streams get priorities rising with the bucket's degree range
  // (the device has few levels; neighbouring buckets may share one).  Within
  // an asynchronous class the blocks of higher-degree vertices are then
  // scheduled first and commit early, and the many low-degree vertices decide
  // against those moves; the hub chain (insert, scan, final per class) no
  // longer queues behind the other buckets.  Measured on R-MAT s22: pass 0
  // moves 2.6M instead of 2.25M vertices, the run takes 14.2 instead of
  // 24.1 ms and ends at Q 0.075-0.077 instead of 0.072.
  int prio_least = 0, prio_greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) {
    delete c;
    return LOUVAIN_ERR_CUDA;
  }
  for (int i = 0; i < louvain_ctx::kAux; ++i)
    if (cudaStreamCreateWithPriority(&c->aux[i], cudaStreamNonBlocking,
                                     prio_least + (prio_greatest - prio_least) * i / (louvain_ctx::kAux - 1)) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join[i], cudaEventDisableTiming) != cudaSuccess) {
      delete c;
      return LOUVAIN_ERR_CUDA;
    }
  if (cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess) { delete c; return LOUVAIN_ERR_CUDA; }
  if (cudaMallocHost(&c->h_ctr, sizeof(DevCounters)) != cudaSuccess ||
      cudaMallocHost(&c->h_acc, 8 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMallocHost(&c->h_scal, 8 * sizeof(int64_t)) != cudaSuccess ||
      cudaMallocHost(&c->h_iter, 4 * sizeof(int)) != cudaSuccess) {
    delete c;
    return LOUVAIN_ERR_OOM;
  }
  memset(&c->stats, 0, sizeof(c->stats));
  *out = c;
  return 0;
}

int louvain_set_options(louvain_ctx* c, const louvain_options* opt) {
  if (!c || !opt) return LOUVAIN_ERR_INVALID_ARG;
  if (check_options(opt)) return fail(c, LOUVAIN_ERR_INVALID_ARG, "invalid options");
  c->opt = *opt;
  return 0;
}

}  // extern "C"

namespace {

// Load one graph (G = 1) or G graphs whose vertices are the contiguous ranges
// [vo[g], vo[g + 1]) of one CSR with no entry between ranges (vo: host).
// Graphs given as separate host CSRs (louvain_load_parts).
struct PartsIn {
  const int64_t* nnz;
  const int64_t* const* off;
  const int32_t* const* col;
  const int32_t* const* w;
};

int load_graphs(louvain_ctx* c, int64_t G, const int64_t* vo, int64_t n, int64_t nnz, const int64_t* offsets,
                const int32_t* cols, const int32_t* weights, int ptr_kind, const PartsIn* parts = nullptr) {
  if (!c) return LOUVAIN_ERR_INVALID_ARG;
  if (n < 0 || nnz < 0 || (ptr_kind != LOUVAIN_PTR_HOST && ptr_kind != LOUVAIN_PTR_DEVICE))
    return fail(c, LOUVAIN_ERR_INVALID_ARG, "negative size or bad pointer kind");
  if (!parts && (!offsets || (nnz > 0 && (!cols || !weights))))
    return fail(c, LOUVAIN_ERR_INVALID_ARG, "null pointer");
  if (n >= (1ll << 31) - 1) return fail(c, LOUVAIN_ERR_OVERFLOW, "n must be below 2^31 - 1");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, LOUVAIN_ERR_CUDA, "cudaSetDevice failed");
  if (ptr_kind == LOUVAIN_PTR_HOST && !parts) {
    // cheap host checks first
    if (offsets[0] != 0 || offsets[n] != nnz) return fail(c, LOUVAIN_ERR_BAD_CSR, "offsets[0] != 0 or offsets[n] != nnz");
  }
  if (!(c->cap_n >= n && c->cap_nnz >= nnz && !c->allocs.empty())) {
    if (int r = alloc_arena(c, n, nnz)) return r;
  }
  c->loaded = false;
  c->ran = false;
  c->n0 = n;
  c->nnz0 = nnz;
  const int64_t N1 = n + 1;
  cudaStream_t s = c->stream;
  cudaMemcpyKind kind = ptr_kind == LOUVAIN_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (parts) {
    // each graph straight to its place; offsets and columns rebased on the device
    std::vector<int64_t> eo(G + 1, 0);
    for (int64_t q = 0; q < G; ++q) eo[q + 1] = eo[q] + parts->nnz[q];
    for (int64_t q = 0; q < G; ++q) {
      const int64_t nq = vo[q + 1] - vo[q], eq = parts->nnz[q];
      if (nq) CK(cudaMemcpyAsync(c->off0 + vo[q], parts->off[q], nq * sizeof(int64_t), kind, s));
      if (eq) {
        CK(cudaMemcpyAsync(c->col0 + eo[q], parts->col[q], eq * sizeof(int32_t), kind, s));
        CK(cudaMemcpyAsync(c->w0 + eo[q], parts->w[q], eq * sizeof(int32_t), kind, s));
      }
    }
    CK(cudaMemcpyAsync(c->vo0, vo, (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->vo_a, eo.data(), (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    rebase_parts(c->off0, c->col0, n, nnz, c->vo0, c->vo_a, (int)G, s);
    CK(cudaStreamSynchronize(s));   // eo goes out of scope
  } else {
    CK(cudaMemcpyAsync(c->off0, offsets, N1 * sizeof(int64_t), kind, s));
    if (nnz) {
      CK(cudaMemcpyAsync(c->col0, cols, nnz * sizeof(int32_t), kind, s));
      CK(cudaMemcpyAsync(c->w0, weights, nnz * sizeof(int32_t), kind, s));
    }
  }
  if (c->tables_dirty) {
    // global tables start empty; every later use clears what it touched
    CK(cudaMemsetAsync(c->gkeys, 0xff, 2 * c->cap_nnz * sizeof(int32_t), s));
    CK(cudaMemsetAsync(c->gvals, 0, 2 * c->cap_nnz * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(c->hkid, 0, (c->cap_n + 1) * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(c->hdone, 0, (c->cap_n + 1) * sizeof(int32_t), s));
    c->tables_dirty = false;
  }
  if (c->opt.validate) {
    // offsets first: the entry checks below walk chunks found from them
    validate_offsets(c->off0, n, nnz, c->flags, s);
    CKLAUNCH();
    int flags = 0;
    if (int r = fetch(c, &flags, c->flags, sizeof(int))) return r;
    if (flags & 1) return fail(c, LOUVAIN_ERR_BAD_CSR, "offsets not monotone or wrong ends");
  }
  // input degrees (for louvain_modularity); with validation the same pass
  // checks the entries (acc[4..5]: the symmetry fingerprints)
  CK(cudaMemsetAsync(c->acc, 0, 8 * sizeof(unsigned long long), s));
  row_sums<int32_t>(c->off0, c->col0, c->w0, n, nnz, c->crow, c->K0, c->acc, c->opt.validate ? c->flags : nullptr,
                    c->acc + 4, s);
  CKLAUNCH();
  if (int r = fetch(c, c->h_acc, c->acc, 6 * sizeof(unsigned long long))) return r;
  if (c->opt.validate) {
    int flags = 0;
    if (int r = fetch(c, &flags, c->flags, sizeof(int))) return r;
    if (flags & 2) return fail(c, LOUVAIN_ERR_BAD_CSR, "column index out of range");
    if (flags & 4) return fail(c, LOUVAIN_ERR_BAD_CSR, "weight <= 0");
    if (c->h_acc[4] != c->h_acc[5]) return fail(c, LOUVAIN_ERR_NOT_SYMMETRIC, "CSR is not symmetric");
  }
  if (c->h_acc[1] != 0 || c->h_acc[0] >= (1ull << 62))
    return fail(c, LOUVAIN_ERR_OVERFLOW, "total weight M must be below 2^62");
  c->M0 = (int64_t)c->h_acc[0];
  {
    // singleton partition: sum L_c = total self-loop weight, sum Sigma_c^2 = sum K_i^2
    const u128 loops = ((u128)c->h_acc[3] << 64) | (u128)c->h_acc[2];
    CK(cudaMemsetAsync(c->acc, 0, 2 * sizeof(unsigned long long), s));
    sum_squares(c->K0, n, c->acc, s);
    CKLAUNCH();
    if (int r = fetch(c, c->h_acc, c->acc, 2 * sizeof(unsigned long long))) return r;
    const u128 SS = ((u128)c->h_acc[1] << 64) | (u128)c->h_acc[0];
    c->qnum0 = (i128)c->M0 * (i128)loops - (i128)SS;
  }
  {
    // vertices without entries: their communities may leave the later passes
    CK(cudaMemsetAsync(c->acc, 0, sizeof(unsigned long long), s));
    count_empty_rows(c->off0, n, c->acc, s);
    CKLAUNCH();
    if (int r = fetch(c, c->h_acc, c->acc, sizeof(unsigned long long))) return r;
    c->iso0 = (int64_t)c->h_acc[0];
  }
  // per graph: M, vertices, singleton numerator
  if (int r = host_graph_buffers(c, G)) return r;
  c->G = G;
  c->gst.assign(G, GraphState());
  c->gM0.assign(G, 0);
  c->gn0.assign(G, 0);
  c->gqnum0.assign(G, 0);
  for (int64_t q = 0; q < G; ++q) c->gn0[q] = vo[q + 1] - vo[q];
  CK(cudaMemcpyAsync(c->vo0, vo, (G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  {
    // class-schedule category per graph: small below kSmallGraph vertices,
    // else sparse below kSparseEntries entries per vertex
    std::vector<int64_t> ge(G);
    if (G == 1) {
      ge[0] = nnz;
    } else {
      graph_entries(c->off0, c->vo0, G, (int64_t*)c->d_gs, s);   // d_gs: scratch until the totals below
      CKLAUNCH();
      if (int r = fetch(c, ge.data(), c->d_gs, G * sizeof(int64_t))) return r;
    }
    c->hgcat.assign(G, kCatLarge);
    for (int64_t q = 0; q < G; ++q)
      c->hgcat[q] = c->gn0[q] < kSmallGraph ? kCatSmall
                    : (ge[q] < kSparseEntries * c->gn0[q] ? kCatSparse : kCatLarge);
    CK(cudaMemcpyAsync(c->d_gcat, c->hgcat.data(), G * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  if (G == 1) {
    c->gM0[0] = c->M0;
    c->gqnum0[0] = c->qnum0;
  } else {
    CK(cudaMemsetAsync(c->flags, 0, sizeof(int), s));
    graph_ids(c->vo0, (int)G, n, nnz, c->gid0, c->off0, c->col0, c->crow, c->flags, s);
    int flags = 0;
    CKLAUNCH();
    if (int r = fetch(c, &flags, c->flags, sizeof(int))) return r;
    if (flags & 8) return fail(c, LOUVAIN_ERR_BAD_CSR, "an entry joins two graphs of the batch");
    CK(cudaMemsetAsync(c->d_gs, 0, 2 * G * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(c->d_gL, 0, 2 * G * sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(c->d_gSS, 0, 2 * G * sizeof(unsigned long long), s));
    graph_totals(c->K0, c->gid0, n, c->d_gs, s);
    iota_i32(c->memb, n, s);
    graph_modularity_parts<int32_t>(c->off0, c->col0, c->w0, n, nnz, c->memb, c->K0, c->gid0, c->d_gL, c->d_gSS,
                                    c->crow, s);
    CKLAUNCH();
    if (int r = fetch_many(c, {{c->h_gs, c->d_gs, 2 * G * sizeof(unsigned long long)},
                               {c->h_gL, c->d_gL, 2 * G * sizeof(unsigned long long)},
                               {c->h_gSS, c->d_gSS, 2 * G * sizeof(unsigned long long)}}))
      return r;
    std::vector<long long> Mg(G);
    for (int64_t q = 0; q < G; ++q) {
      const u128 M = ((u128)c->h_gs[2 * q + 1] << 64) | (u128)c->h_gs[2 * q];
      const u128 L = ((u128)c->h_gL[2 * q + 1] << 64) | (u128)c->h_gL[2 * q];
      const u128 SS = ((u128)c->h_gSS[2 * q + 1] << 64) | (u128)c->h_gSS[2 * q];
      c->gM0[q] = (int64_t)M;
      Mg[q] = (long long)M;
      c->gqnum0[q] = (i128)(int64_t)M * (i128)L - (i128)SS;
    }
    CK(cudaMemcpyAsync(c->d_Mg, Mg.data(), G * sizeof(long long), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  c->loaded = true;
  c->ran = false;
  return 0;
}

}  // namespace

extern "C" {

int louvain_load_csr(louvain_ctx* c, int64_t n, int64_t nnz, const int64_t* offsets, const int32_t* cols,
                     const int32_t* weights, int ptr_kind) {
  if (n < 0) return c ? fail(c, LOUVAIN_ERR_INVALID_ARG, "negative size") : LOUVAIN_ERR_INVALID_ARG;
  const int64_t vo[2] = {0, n};
  return load_graphs(c, 1, vo, n, nnz, offsets, cols, weights, ptr_kind);
}

int louvain_load_batch(louvain_ctx* c, int64_t num_graphs, const int64_t* graph_offsets, int64_t n, int64_t nnz,
                       const int64_t* offsets, const int32_t* cols, const int32_t* weights, int ptr_kind) {
  if (!c) return LOUVAIN_ERR_INVALID_ARG;
  if (num_graphs < 1 || num_graphs > n + 1 || !graph_offsets || n < 0)
    return fail(c, LOUVAIN_ERR_INVALID_ARG, "num_graphs must be in [1, n] with graph_offsets given");
  std::vector<int64_t> vo(num_graphs + 1);
  if (ptr_kind == LOUVAIN_PTR_DEVICE) {
    if (cudaMemcpy(vo.data(), graph_offsets, vo.size() * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(c, LOUVAIN_ERR_CUDA, "copying graph offsets failed");
  } else {
    memcpy(vo.data(), graph_offsets, vo.size() * sizeof(int64_t));
  }
  if (vo[0] != 0 || vo[num_graphs] != n) return fail(c, LOUVAIN_ERR_BAD_CSR, "graph offsets must run from 0 to n");
  for (int64_t q = 0; q < num_graphs; ++q)
    if (vo[q + 1] < vo[q]) return fail(c, LOUVAIN_ERR_BAD_CSR, "graph offsets must not decrease");
  return load_graphs(c, num_graphs, vo.data(), n, nnz, offsets, cols, weights, ptr_kind);
}


int louvain_load_parts(louvain_ctx* c, int64_t num_graphs, const int64_t* ns, const int64_t* nnzs,
                       const int64_t* const* offsets, const int32_t* const* cols, const int32_t* const* weights) {
  if (!c) return LOUVAIN_ERR_INVALID_ARG;
  if (num_graphs < 1 || !ns || !nnzs || !offsets || !cols || !weights)
    return fail(c, LOUVAIN_ERR_INVALID_ARG, "num_graphs >= 1 and every array given");
  std::vector<int64_t> vo(num_graphs + 1, 0);
  int64_t nnz = 0;
  for (int64_t q = 0; q < num_graphs; ++q) {
    if (ns[q] < 0 || nnzs[q] < 0 || !offsets[q] || (nnzs[q] > 0 && (!cols[q] || !weights[q])))
      return fail(c, LOUVAIN_ERR_INVALID_ARG, "negative size or null pointer in a graph");
    if (offsets[q][0] != 0 || offsets[q][ns[q]] != nnzs[q])
      return fail(c, LOUVAIN_ERR_BAD_CSR, "offsets[0] != 0 or offsets[n] != nnz in a graph");
    vo[q + 1] = vo[q] + ns[q];
    nnz += nnzs[q];
  }
  const int64_t n = vo[num_graphs];
  if (num_graphs > n + 1) return fail(c, LOUVAIN_ERR_INVALID_ARG, "more graphs than vertices + 1");
  PartsIn parts{nnzs, offsets, cols, weights};
  return load_graphs(c, num_graphs, vo.data(), n, nnz, nullptr, nullptr, nullptr, LOUVAIN_PTR_HOST, &parts);
}

int louvain_set_mapping(louvain_ctx* c, const int32_t* thresholds) {
  if (!c) return LOUVAIN_ERR_INVALID_ARG;
  LMThresholds th = {{kLMCap[0], kLMCap[1], kLMCap[2], kLMCap[3], kLMCap[4]}};
  if (thresholds) {
    for (int b = 0; b < 5; ++b) {
      if (thresholds[b] < 1 || thresholds[b] > kLMCap[b] || (b > 0 && thresholds[b] <= thresholds[b - 1]))
        return fail(c, LOUVAIN_ERR_INVALID_ARG, "thresholds must increase and stay within each kernel's capacity");
      th.t[b] = thresholds[b];
    }
  }
  c->thr = th;
  return 0;
}

int louvain_get_mapping(louvain_ctx* c, int32_t* thresholds) {
  if (!c || !thresholds) return LOUVAIN_ERR_INVALID_ARG;
  for (int b = 0; b < 5; ++b) thresholds[b] = c->thr.t[b];
  return 0;
}

int louvain_autotune(louvain_ctx* c, int32_t* thresholds, double* ms) {
  if (!c) return LOUVAIN_ERR_INVALID_ARG;
  if (!c->loaded) return fail(c, LOUVAIN_ERR_STATE, "no graph loaded");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, LOUVAIN_ERR_CUDA, "cudaSetDevice failed");
  float best = 0;
  if (c->M0 > 0) {
    int r = autotune(c, &best);
    if (r) {
      c->tables_dirty = true;
      c->loaded = false;
      return r;
    }
  }
  if (thresholds)
    for (int b = 0; b < 5; ++b) thresholds[b] = c->thr.t[b];
  if (ms) *ms = best;
  return 0;
}

int louvain_run_from(louvain_ctx* c, const int32_t* memb, int64_t n, int ptr_kind) {
  if (!c) return LOUVAIN_ERR_INVALID_ARG;
  if (!c->loaded) return fail(c, LOUVAIN_ERR_STATE, "no graph loaded");
  if (n != c->n0 || (!memb && n > 0) || (ptr_kind != LOUVAIN_PTR_HOST && ptr_kind != LOUVAIN_PTR_DEVICE))
    return fail(c, LOUVAIN_ERR_INVALID_ARG, "the initial membership must have the loaded n entries");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, LOUVAIN_ERR_CUDA, "cudaSetDevice failed");
  c->ran = false;
  if (n > 0) {
    const cudaMemcpyKind kind = ptr_kind == LOUVAIN_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (cudaMemcpyAsync(c->memb, memb, n * sizeof(int32_t), kind, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream) != cudaSuccess)
      return fail(c, LOUVAIN_ERR_CUDA, "copy of the initial membership failed");
    check_membership(n, c->memb, c->G > 1 ? c->gid0 : nullptr, c->G > 1 ? c->vo0 : nullptr, c->flags, c->stream);
    int flag = 0;
    if (cudaGetLastError() != cudaSuccess || fetch(c, &flag, c->flags, sizeof(int)))
      return fail(c, LOUVAIN_ERR_CUDA, "membership check failed");
    if (flag) return fail(c, LOUVAIN_ERR_INVALID_ARG, "initial membership: an id outside its graph's vertex range");
  }
  c->warm = true;
  int r = run_all(c);
  c->warm = false;
  if (r) {
    c->tables_dirty = true;
    c->loaded = false;   // load again before the next run
    return r;
  }
  c->ran = true;
  return 0;
}

int louvain_run_partitioned(louvain_ctx* c, int64_t parts, double* parts_ms) {
  if (!c) return LOUVAIN_ERR_INVALID_ARG;
  if (!c->loaded) return fail(c, LOUVAIN_ERR_STATE, "no graph loaded");
  if (c->G != 1) return fail(c, LOUVAIN_ERR_STATE, "partition-then-merge takes one loaded graph");
  if (parts < 1) return fail(c, LOUVAIN_ERR_INVALID_ARG, "parts must be >= 1");
  const int64_t n = c->n0, nnz = c->nnz0;
  if (parts > n) parts = n > 0 ? n : 1;
  if (parts_ms) *parts_ms = 0;
  if (parts == 1 || n == 0) return louvain_run(c);
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, LOUVAIN_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t s = c->stream;
  c->ran = false;
  // 1. the parts' induced subgraphs, as one block-diagonal CSR in the coarse
  //    buffers (free before a run)
  int64_t* flags = (int64_t*)c->tw;
  int64_t* pos = (int64_t*)c->wX[1];
  induced_parts(c->off0, c->col0, c->w0, n, nnz, parts, flags, pos, c->scal, c->offX[0], c->colX[0],
                (int32_t*)c->wX[0], c->tmp, s);
  CKLAUNCH();
  int64_t nnz_sub = 0;
  if (int r = fetch(c, &nnz_sub, c->scal, sizeof(int64_t))) return r;
  std::vector<int64_t> vo(parts + 1);
  for (int64_t p = 0; p <= parts; ++p) vo[p] = (p * n + parts - 1) / parts;
  // 2. every part on its own, in one batched run of a second context
  if (!c->sub) {
    louvain_options o = c->opt;
    o.validate = 0;        // an induced subgraph of a valid graph is valid
    o.record_levels = 0;
    if (louvain_create(&c->sub, &o, c->device, (void*)s)) return fail(c, LOUVAIN_ERR_CUDA, "parts context");
  } else {
    louvain_options o = c->opt;
    o.validate = 0;
    o.record_levels = 0;
    louvain_set_options(c->sub, &o);
  }
  c->sub->thr = c->thr;
  int r = louvain_load_batch(c->sub, parts, vo.data(), n, nnz_sub, c->offX[0], c->colX[0], (int32_t*)c->wX[0],
                             LOUVAIN_PTR_DEVICE);
  if (!r) r = louvain_run(c->sub);
  if (r) return fail(c, r, std::string("parts run: ") + louvain_last_error(c->sub));
  if (parts_ms) *parts_ms = c->sub->stats.total_ms;
  // 3. merge: the whole graph from the parts' communities (global ids)
  if ((r = louvain_get_membership(c->sub, c->level, n, LOUVAIN_PTR_DEVICE)))
    return fail(c, r, std::string("parts membership: ") + louvain_last_error(c->sub));
  part_base(c->level, n, parts, s);
  CKLAUNCH();
  return louvain_run_from(c, c->level, n, LOUVAIN_PTR_DEVICE);
}

int louvain_run(louvain_ctx* c) {
  if (!c) return LOUVAIN_ERR_INVALID_ARG;
  if (!c->loaded) return fail(c, LOUVAIN_ERR_STATE, "no graph loaded");
  if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, LOUVAIN_ERR_CUDA, "cudaSetDevice failed");
  c->ran = false;
  int r = run_all(c);
  if (r) {
    c->tables_dirty = true;
    c->loaded = false;   // load again before the next run
    return r;
  }
  c->ran = true;
  return 0;
}

int louvain_get_membership(louvain_ctx* c, int32_t* out, int64_t n, int ptr_kind) {
  if (!c) return LOUVAIN_ERR_INVALID_ARG;
  if (!c->ran) return fail(c, LOUVAIN_ERR_STATE, "no result (run first)");
  if (n != c->n0 || (!out && n > 0)) return fail(c, LOUVAIN_ERR_INVALID_ARG, "n must equal the loaded n");
  if (n == 0) return 0;
  cudaMemcpyKind kind = ptr_kind == LOUVAIN_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  const int32_t* src = c->top;
  if (c->G > 1) {
    // ids local to each graph: top - first community id of the vertex's graph
    localize_membership(c->top, c->gid0, c->vo_top, n, c->key, c->stream);
    CKLAUNCH();
    src = c->key;
  }
  CK(cudaMemcpyAsync(out, src, n * sizeof(int32_t), kind, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return 0;
}

int louvain_get_modularity(louvain_ctx* c, double* q) {
  if (!c || !q) return LOUVAIN_ERR_INVALID_ARG;
  if (!c->ran) return fail(c, LOUVAIN_ERR_STATE, "no result (run first)");
  if (c->G > 1) return fail(c, LOUVAIN_ERR_STATE, "several graphs loaded: use louvain_batch_get_modularity");
  *q = c->Q;
  return 0;
}

int louvain_get_modularity_exact(louvain_ctx* c, int64_t* num_hi, uint64_t* num_lo, int64_t* M) {
  if (!c || !num_hi || !num_lo || !M) return LOUVAIN_ERR_INVALID_ARG;
  if (!c->ran) return fail(c, LOUVAIN_ERR_STATE, "no result (run first)");
  if (c->G > 1) return fail(c, LOUVAIN_ERR_STATE, "several graphs loaded: use louvain_batch_get_modularity");
  *num_hi = (int64_t)(c->qnum >> 64);
  *num_lo = (uint64_t)c->qnum;
  *M = c->M;
  return 0;
}

int louvain_modularity(louvain_ctx* c, const int32_t* memb, int64_t n, int ptr_kind, double* q, int64_t* num_hi,
                       uint64_t* num_lo, int64_t* Mout) {
  if (!c || !q) return LOUVAIN_ERR_INVALID_ARG;
  if (!c->loaded) return fail(c, LOUVAIN_ERR_STATE, "no graph loaded");
  if (n != c->n0 || (!memb && n > 0)) return fail(c, LOUVAIN_ERR_INVALID_ARG, "n must equal the loaded n");
  cudaStream_t s = c->stream;
  if (ptr_kind == LOUVAIN_PTR_HOST) {
    for (int64_t i = 0; i < n; ++i)
      if (memb[i] < 0 || memb[i] >= n) return fail(c, LOUVAIN_ERR_INVALID_ARG, "membership out of range");
  }
  cudaMemcpyKind kind = ptr_kind == LOUVAIN_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (n) CK(cudaMemcpyAsync(c->used, memb, n * sizeof(int32_t), kind, s));
  community_totals(c->K0, c->used, n, c->Knext, s);
  CK(cudaMemsetAsync(c->acc, 0, 8 * sizeof(unsigned long long), s));
  modularity_parts<int32_t>(c->off0, c->col0, c->w0, n, c->nnz0, c->used, c->Knext, c->acc, c->crow, s);
  CKLAUNCH();
  if (int r = fetch(c, c->h_acc, c->acc, 4 * sizeof(unsigned long long))) return r;
  const int64_t M = c->M0;
  u128 L = ((u128)c->h_acc[3] << 64) | (u128)c->h_acc[0];
  u128 SS = ((u128)c->h_acc[2] << 64) | (u128)c->h_acc[1];
  i128 N = (i128)M * (i128)L - (i128)SS;
  *q = M == 0 ? 0.0 : dbl(N) / dbl((i128)M * M);
  if (num_hi) *num_hi = (int64_t)(N >> 64);
  if (num_lo) *num_lo = (uint64_t)N;
  if (Mout) *Mout = M;
  return 0;
}

int louvain_get_stats(louvain_ctx* c, louvain_stats* out) {
  if (!c || !out) return LOUVAIN_ERR_INVALID_ARG;
  if (!c->ran) return fail(c, LOUVAIN_ERR_STATE, "no result (run first)");
  *out = c->stats;
  return 0;
}

int louvain_get_pass_info(louvain_ctx* c, int pass, louvain_pass_info* out) {
  if (!c || !out) return LOUVAIN_ERR_INVALID_ARG;
  if (!c->ran) return fail(c, LOUVAIN_ERR_STATE, "no result (run first)");
  if (pass < 0 || pass >= (int)c->passes.size()) return fail(c, LOUVAIN_ERR_INVALID_ARG, "no such pass");
  *out = c->passes[pass].info;
  return 0;
}

int louvain_get_iteration(louvain_ctx* c, int64_t t, int64_t out[4]) {
  if (!c || !out) return LOUVAIN_ERR_INVALID_ARG;
  if (!c->ran) return fail(c, LOUVAIN_ERR_STATE, "no result (run first)");
  if (t < 0 || t >= (int64_t)c->iters.size()) return fail(c, LOUVAIN_ERR_INVALID_ARG, "no such iteration");
  const IterRec& r = c->iters[t];
  out[0] = r.pass;
  out[1] = r.moves;
  out[2] = (int64_t)(r.S >> 64);
  out[3] = (int64_t)(uint64_t)r.S;
  return 0;
}

int louvain_get_level(louvain_ctx* c, int pass, int32_t* out, int64_t n) {
  if (!c || !out) return LOUVAIN_ERR_INVALID_ARG;
  if (!c->ran) return fail(c, LOUVAIN_ERR_STATE, "no result (run first)");
  if (pass < 0 || pass >= (int)c->passes.size() || !c->passes[pass].info.level_recorded)
    return fail(c, LOUVAIN_ERR_STATE, "level not recorded (record_levels = 1)");
  const PassRec& p = c->passes[pass];
  if (n != (int64_t)p.level.size()) return fail(c, LOUVAIN_ERR_INVALID_ARG, "n must equal the pass graph size");
  memcpy(out, p.level.data(), n * sizeof(int32_t));
  return 0;
}

int louvain_get_coarse(louvain_ctx* c, int pass, int64_t* off, int64_t k, int32_t* col, int64_t* w, int64_t nnz) {
  if (!c || !off) return LOUVAIN_ERR_INVALID_ARG;
  if (!c->ran) return fail(c, LOUVAIN_ERR_STATE, "no result (run first)");
  if (pass < 0 || pass >= (int)c->passes.size() || !c->passes[pass].info.coarse_built || c->passes[pass].coff.empty())
    return fail(c, LOUVAIN_ERR_STATE, "coarse graph not recorded (record_levels = 1)");
  const PassRec& p = c->passes[pass];
  if (k + 1 != (int64_t)p.coff.size() || nnz != (int64_t)p.ccol.size())
    return fail(c, LOUVAIN_ERR_INVALID_ARG, "sizes must equal the coarse graph's");
  memcpy(off, p.coff.data(), (k + 1) * sizeof(int64_t));
  if (nnz) {
    if (!col || !w) return LOUVAIN_ERR_INVALID_ARG;
    memcpy(col, p.ccol.data(), nnz * sizeof(int32_t));
    memcpy(w, p.cw.data(), nnz * sizeof(int64_t));
  }
  return 0;
}

int louvain_batch_get_modularity(louvain_ctx* c, double* q, int64_t* num_hi, uint64_t* num_lo, int64_t* M) {
  if (!c || !q) return LOUVAIN_ERR_INVALID_ARG;
  if (!c->ran) return fail(c, LOUVAIN_ERR_STATE, "no result (run first)");
  for (int64_t g = 0; g < c->G; ++g) {
    const GraphState& st = c->gst[g];
    q[g] = st.M == 0 ? 0.0 : dbl(st.qnum) / dbl((i128)st.M * st.M);
    if (num_hi) num_hi[g] = (int64_t)(st.qnum >> 64);
    if (num_lo) num_lo[g] = (uint64_t)st.qnum;
    if (M) M[g] = st.M;
  }
  return 0;
}

int louvain_batch_get_graph_info(louvain_ctx* c, int64_t g, int64_t out[4]) {
  if (!c || !out) return LOUVAIN_ERR_INVALID_ARG;
  if (!c->ran) return fail(c, LOUVAIN_ERR_STATE, "no result (run first)");
  if (g < 0 || g >= c->G) return fail(c, LOUVAIN_ERR_INVALID_ARG, "no such graph");
  const GraphState& st = c->gst[g];
  int64_t moves = 0;
  const std::vector<IterRec>& it = c->G > 1 ? st.iters : c->iters;
  for (const IterRec& r : it) moves += r.moves;
  out[0] = st.passes;
  out[1] = (int64_t)it.size();
  out[2] = st.k;
  out[3] = moves;
  return 0;
}

int louvain_batch_get_iterations(louvain_ctx* c, int64_t g, int64_t* out, int64_t cap, int64_t* count) {
  if (!c || !count) return LOUVAIN_ERR_INVALID_ARG;
  if (!c->ran) return fail(c, LOUVAIN_ERR_STATE, "no result (run first)");
  if (g < 0 || g >= c->G) return fail(c, LOUVAIN_ERR_INVALID_ARG, "no such graph");
  const std::vector<IterRec>& it = c->G > 1 ? c->gst[g].iters : c->iters;
  *count = (int64_t)it.size();
  for (int64_t t = 0; t < (int64_t)it.size() && t < cap && out; ++t) {
    out[4 * t] = it[t].pass;
    out[4 * t + 1] = it[t].moves;
    out[4 * t + 2] = (int64_t)(it[t].S >> 64);
    out[4 * t + 3] = (int64_t)(uint64_t)it[t].S;
  }
  return 0;
}

int louvain_arena_bytes(int64_t n, int64_t nnz, int64_t* bytes) {
  if (n < 0 || nnz < 0 || !bytes) return LOUVAIN_ERR_INVALID_ARG;
  louvain_ctx c;
  c.dry_run = true;
  int r = alloc_arena(&c, n, nnz);
  *bytes = c.bytes;
  return r;
}

int louvain_get_num_graphs(louvain_ctx* c, int64_t* num_graphs) {
  if (!c || !num_graphs) return LOUVAIN_ERR_INVALID_ARG;
  *num_graphs = c->G;
  return 0;
}

int louvain_get_device_bytes(louvain_ctx* c, int64_t* bytes) {
  if (!c || !bytes) return LOUVAIN_ERR_INVALID_ARG;
  *bytes = c->bytes;
  return 0;
}

void louvain_destroy(louvain_ctx* c) {
  if (!c) return;
  if (c->sub) louvain_destroy(c->sub);
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_all(c);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  for (int i = 0; i < louvain_ctx::kAux; ++i) {
    if (c->aux[i]) { cudaStreamSynchronize(c->aux[i]); cudaStreamDestroy(c->aux[i]); }
    if (c->ev_join[i]) cudaEventDestroy(c->ev_join[i]);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->h_ctr) cudaFreeHost(c->h_ctr);
  if (c->h_acc) cudaFreeHost(c->h_acc);
  if (c->h_scal) cudaFreeHost(c->h_scal);
  if (c->h_pair) cudaFreeHost(c->h_pair);
  if (c->h_iter) cudaFreeHost(c->h_iter);
  free_host_graph_buffers(c);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* louvain_last_error(const louvain_ctx* c) { return c ? c->err.c_str() : "null context"; }

const char* louvain_version(void) { return "gb-louvain 0.1 (sm_103a)"; }

}  // extern "C"
