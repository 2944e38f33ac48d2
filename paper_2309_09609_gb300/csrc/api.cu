// api.cu -- host side of libswgb: the C ABI of include/swgb.h.
//
//   * sw_db_create: sorts subjects by length and builds the two device
//     layouts (interleaved groups of 64 for the inter-task kernel, contiguous
//     for the intra-task kernel); the split of the database by length into a
//     short (inter-task) and long (intra-task) part follows Section III-A.
//   * sw_plan_*: a reusable search context.  Its device memory is allocated
//     once (the host-order scores buffer at the first search that needs it);
//     per search only the query block, the query-stream strip table and a
//     parameter block are copied, and the kernel sequence (reset counters;
//     the two pair-kernel widths on two streams; the two inter-task kernels,
//     of which the plan gives one the items; the int32 kernel for saturated
//     pairs) is replayed from a CUDA graph, one per gap class.  A flag-list
//     overflow is recomputed in further rounds after the graph.
//   * sw_search: through a plan kept by the database.
//   * sw_search_plain: the int32 baseline, one kernel launch per query.
//   * sw_align: optimal alignments with traceback of selected pairs.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include "swgb_internal.h"

using namespace swgb;

// ---- errors ---------------------------------------------------------------------
namespace swgb {
static thread_local char g_err[512] = "";

sw_status sw_set_error(sw_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return st;
}

sw_status sw_set_cuda_error(cudaError_t err, const char* where) {
  cudaGetLastError();  // clear a sticky launch error so the context stays usable
  return sw_set_error(err == cudaErrorMemoryAllocation ? SW_ENOMEM : SW_ECUDA, "%s: %s", where,
                      cudaGetErrorString(err));
}

void sw_clear_error() { g_err[0] = 0; }
}  // namespace swgb

extern "C" const char* sw_last_error(void) { return g_err; }

// ---- alphabet and BLOSUM62 ------------------------------------------------------
static const char kAlphabet[] = "ARNDCQEGHILKMFPSTWYVBZX*";
static constexpr int kCodeX = 22;

extern "C" sw_status sw_encode(const char* text, int64_t n, uint8_t* out) {
  if (n < 0 || (n > 0 && (!text || !out))) return sw_set_error(SW_EINVAL, "sw_encode: bad arguments");
  int8_t table[256];
  for (int i = 0; i < 256; i++) table[i] = kCodeX;
  for (int c = 0; c < ALPHA; c++) {
    const unsigned char u = (unsigned char)kAlphabet[c];
    table[u] = (int8_t)c;
    if (u >= 'A' && u <= 'Z') table[u - 'A' + 'a'] = (int8_t)c;
  }
  for (int64_t i = 0; i < n; i++) out[i] = (uint8_t)table[(unsigned char)text[i]];
  return SW_OK;
}

// BLOSUM62 (Henikoff & Henikoff 1992), NCBI table in the order of kAlphabet.
// The paper searches with BLOSUM62 (Section IV-A) without printing it.
static const int8_t kBlosum62[ALPHA * ALPHA] = {
    4,  -1, -2, -2, 0,  -1, -1, 0,  -2, -1, -1, -1, -1, -2, -1, 1,  0,  -3, -2, 0,  -2, -1, 0,  -4,
    -1, 5,  0,  -2, -3, 1,  0,  -2, 0,  -3, -2, 2,  -1, -3, -2, -1, -1, -3, -2, -3, -1, 0,  -1, -4,
    -2, 0,  6,  1,  -3, 0,  0,  0,  1,  -3, -3, 0,  -2, -3, -2, 1,  0,  -4, -2, -3, 3,  0,  -1, -4,
    -2, -2, 1,  6,  -3, 0,  2,  -1, -1, -3, -4, -1, -3, -3, -1, 0,  -1, -4, -3, -3, 4,  1,  -1, -4,
    0,  -3, -3, -3, 9,  -3, -4, -3, -3, -1, -1, -3, -1, -2, -3, -1, -1, -2, -2, -1, -3, -3, -2, -4,
    -1, 1,  0,  0,  -3, 5,  2,  -2, 0,  -3, -2, 1,  0,  -3, -1, 0,  -1, -2, -1, -2, 0,  3,  -1, -4,
    -1, 0,  0,  2,  -4, 2,  5,  -2, 0,  -3, -3, 1,  -2, -3, -1, 0,  -1, -3, -2, -2, 1,  4,  -1, -4,
    0,  -2, 0,  -1, -3, -2, -2, 6,  -2, -4, -4, -2, -3, -3, -2, 0,  -2, -2, -3, -3, -1, -2, -1, -4,
    -2, 0,  1,  -1, -3, 0,  0,  -2, 8,  -3, -3, -1, -2, -1, -2, -1, -2, -2, 2,  -3, 0,  0,  -1, -4,
    -1, -3, -3, -3, -1, -3, -3, -4, -3, 4,  2,  -3, 1,  0,  -3, -2, -1, -3, -1, 3,  -3, -3, -1, -4,
    -1, -2, -3, -4, -1, -2, -3, -4, -3, 2,  4,  -2, 2,  0,  -3, -2, -1, -2, -1, 1,  -4, -3, -1, -4,
    -1, 2,  0,  -1, -3, 1,  1,  -2, -1, -3, -2, 5,  -1, -3, -1, 0,  -1, -3, -2, -2, 0,  1,  -1, -4,
    -1, -1, -2, -3, -1, 0,  -2, -3, -2, 1,  2,  -1, 5,  0,  -2, -1, -1, -1, -1, 1,  -3, -1, -1, -4,
    -2, -3, -3, -3, -2, -3, -3, -3, -1, 0,  0,  -3, 0,  6,  -4, -2, -2, 1,  3,  -1, -3, -3, -1, -4,
    -1, -2, -2, -1, -3, -1, -1, -2, -2, -3, -3, -1, -2, -4, 7,  -1, -1, -4, -3, -2, -2, -1, -2, -4,
    1,  -1, 1,  0,  -1, 0,  0,  0,  -1, -2, -2, 0,  -1, -2, -1, 4,  1,  -3, -2, -2, 0,  0,  0,  -4,
    0,  -1, 0,  -1, -1, -1, -1, -2, -2, -1, -1, -1, -1, -2, -1, 1,  5,  -2, -2, 0,  -1, -1, 0,  -4,
    -3, -3, -4, -4, -2, -2, -3, -2, -2, -3, -2, -3, -1, 1,  -4, -3, -2, 11, 2,  -3, -4, -3, -2, -4,
    -2, -2, -2, -3, -2, -1, -2, -3, 2,  -1, -1, -2, -1, 3,  -3, -2, -2, 2,  7,  -1, -3, -2, -1, -4,
    0,  -3, -3, -3, -1, -2, -2, -3, -3, 3,  1,  -2, 1,  -1, -2, -2, 0,  -3, -1, 4,  -3, -2, -1, -4,
    -2, -1, 3,  4,  -3, 0,  1,  -1, 0,  -3, -4, 0,  -3, -3, -2, 0,  -1, -4, -3, -3, 4,  1,  -1, -4,
    -1, 0,  0,  1,  -3, 3,  4,  -2, 0,  -3, -3, 1,  -1, -3, -1, 0,  -1, -3, -2, -2, 1,  4,  -1, -4,
    0,  -1, -1, -1, -2, -1, -1, -1, -1, -1, -1, -1, -1, -1, -2, 0,  0,  -2, -1, -1, -1, -1, -1, -4,
    -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, 1,
};

extern "C" void sw_default_matrix(int8_t* out) {
  if (out) memcpy(out, kBlosum62, sizeof kBlosum62);
}

extern "C" void sw_options_default(sw_options* opt) {
  if (!opt) return;
  opt->rows_per_thread = 32;
  opt->warps_per_block = 8;
  opt->long_cutoff = 1500;
  opt->intra_rows = 8;
  opt->use_graph = 1;
  opt->force_int32 = 0;
  opt->auto_cutoff = 0;
  opt->wide_min_len = 0;
  opt->wide_min_subject = 4096;
  opt->inter_columns = 8;
  opt->overlap_kernels = 0;
  opt->two_query = 1;
  opt->two_query_rows = 32;
  opt->two_query_pairs = 0;
  opt->flag_capacity = 0;
  opt->two_query_long = 1;
}

// ---- small helpers ----------------------------------------------------------------
// Host-side fault injection for tests: with SWGB_FAULT=alloc the device
// allocations of sw_db_create and sw_plan_create report out-of-memory, and
// with SWGB_FAULT=copy the first copy of a search reports a failed copy, so
// the error paths run without a device fault.  Read at every call; unset, it
// changes nothing.
static bool injected_fault(const char* what) {
  const char* f = getenv("SWGB_FAULT");
  return f && strcmp(f, what) == 0;
}

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
static cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, count * sizeof(T));
}

static int parallel_threads() {
  unsigned h = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(h, 32u));
}

template <typename F>
static void parallel_for(int64_t n, F f) {
  const int nt = (int)std::min<int64_t>(parallel_threads(), std::max<int64_t>(n, 1));
  if (nt <= 1) {
    for (int64_t i = 0; i < n; i++) f(i);
    return;
  }
  std::atomic<int64_t> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; t++)
    th.emplace_back([&]() {
      for (;;) {
        const int64_t lo = next.fetch_add(64);
        if (lo >= n) break;
        const int64_t hi = std::min(n, lo + 64);
        for (int64_t i = lo; i < hi; i++) f(i);
      }
    });
  for (auto& x : th) x.join();
}

// ---- database -----------------------------------------------------------------------
static void plan_free(sw_plan* p);

struct sw_db {
  int device = 0;
  DbView view{};
  std::vector<int32_t> glen_h;   // padded group lengths (host copy)
  std::vector<int32_t> clen_h;   // sorted lengths (host copy)
  std::vector<int64_t> cres_h;   // [N + 1] residues of sorted subjects [0, s)
  std::vector<int32_t> sorted_of_h;  // caller index -> sorted index
  int64_t residues = 0;
  // owned device buffers
  uint8_t* inter = nullptr;
  int64_t* goff = nullptr;
  int32_t* glen = nullptr;
  uint8_t* cont = nullptr;
  int64_t* coff = nullptr;
  int32_t* clen = nullptr;
  int32_t* perm = nullptr;
  // the plan behind sw_search, kept between calls (guarded by oneshot_mu)
  sw_plan* oneshot = nullptr;
  std::mutex oneshot_mu;
};

static void db_free(sw_db* db) {
  if (!db) return;
  plan_free(db->oneshot);
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(db->device);
  cudaFree(db->inter);
  cudaFree(db->goff);
  cudaFree(db->glen);
  cudaFree(db->cont);
  cudaFree(db->coff);
  cudaFree(db->clen);
  cudaFree(db->perm);
  cudaSetDevice(cur);
  cudaGetLastError();  // a failed free or device switch leaves no stale error
  delete db;
}

extern "C" sw_status sw_db_create(const uint8_t* residues, const int32_t* lengths,
                                  int64_t n_subjects, int device, sw_db** out) {
  sw_clear_error();
  if (!out) return sw_set_error(SW_EINVAL, "sw_db_create: out is NULL");
  *out = nullptr;
  if (n_subjects < 0 || n_subjects > (int64_t)INT32_MAX - GROUP)
    return sw_set_error(SW_EINVAL, "sw_db_create: n_subjects %lld out of range", (long long)n_subjects);
  if (n_subjects > 0 && !lengths) return sw_set_error(SW_EINVAL, "sw_db_create: lengths is NULL");
  const int64_t N = n_subjects;
  std::vector<int64_t> off(N);
  int64_t total = 0;
  int32_t max_len = 0;
  for (int64_t i = 0; i < N; i++) {
    if (lengths[i] < 0) return sw_set_error(SW_EINVAL, "sw_db_create: length[%lld] < 0", (long long)i);
    off[i] = total;
    total += lengths[i];
    max_len = std::max(max_len, lengths[i]);
  }
  if (total > 0 && !residues) return sw_set_error(SW_EINVAL, "sw_db_create: residues is NULL");
  for (int64_t i = 0; i < total; i++)
    if (residues[i] >= ALPHA)
      return sw_set_error(SW_EINVAL, "sw_db_create: residue code %d at %lld (codes are 0..23)",
                          (int)residues[i], (long long)i);
  CUDA_TRY(cudaSetDevice(device));

  // sort by length, longest first (stable: ties keep caller order)
  std::vector<int32_t> order(N);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return lengths[a] > lengths[b]; });
  const int32_t G = (int32_t)((N + GROUP - 1) / GROUP);
  std::vector<int32_t> glen(G), clen(N), perm((size_t)G * GROUP, -1);
  std::vector<int64_t> goff(G), coff(N);
  int64_t inter_bytes = 0, c = 0;
  for (int32_t g = 0; g < G; g++) {
    const int32_t L = lengths[order[(size_t)g * GROUP]];  // the group's longest
    glen[g] = (L + CHUNK - 1) / CHUNK * CHUNK;
    goff[g] = inter_bytes;
    inter_bytes += (int64_t)glen[g] * GROUP;
  }
  for (int64_t s = 0; s < N; s++) {
    perm[s] = order[s];
    clen[s] = lengths[order[s]];
    coff[s] = c;
    c += clen[s];
  }
  std::vector<uint8_t> inter((size_t)std::max<int64_t>(inter_bytes, 1)), cont((size_t)std::max<int64_t>(total, 1));
  parallel_for(G, [&](int64_t g) {
    uint8_t* base = inter.data() + goff[g];
    const int32_t L = glen[g];
    for (int k = 0; k < GROUP; k++) {
      const int64_t s = g * GROUP + k;
      const uint8_t* src = s < N ? residues + off[order[s]] : nullptr;
      const int32_t len = s < N ? lengths[order[s]] : 0;
      uint8_t* dst = base + (k >> 1) * 16 + (k & 1) * 8;
      for (int32_t j = 0; j < L; j++)
        dst[(int64_t)(j / CHUNK) * CHUNK_BYTES + (j % CHUNK)] = j < len ? src[j] : (uint8_t)PAD_CODE;
    }
  });
  parallel_for(N, [&](int64_t s) {
    if (clen[s]) memcpy(cont.data() + coff[s], residues + off[order[s]], (size_t)clen[s]);
  });

  sw_db* db = new sw_db();
  db->device = device;
  db->residues = total;
  cudaError_t e = injected_fault("alloc") ? cudaErrorMemoryAllocation : cudaSuccess;
#define DB_ALLOC_COPY(dst, src, count)                                                     \
  if (e == cudaSuccess) e = dalloc(&db->dst, (count));                                     \
  if (e == cudaSuccess && (count) > 0)                                                     \
    e = cudaMemcpy(db->dst, (src), sizeof(*db->dst) * (size_t)(count), cudaMemcpyHostToDevice);
  DB_ALLOC_COPY(inter, inter.data(), inter_bytes);
  DB_ALLOC_COPY(goff, goff.data(), G);
  DB_ALLOC_COPY(glen, glen.data(), G);
  DB_ALLOC_COPY(cont, cont.data(), total);
  DB_ALLOC_COPY(coff, coff.data(), N);
  DB_ALLOC_COPY(clen, clen.data(), N);
  DB_ALLOC_COPY(perm, perm.data(), (int64_t)G * GROUP);
#undef DB_ALLOC_COPY
  if (e != cudaSuccess) {
    sw_status st = sw_set_cuda_error(e, "sw_db_create: device upload");
    db_free(db);
    return st;
  }
  db->view.inter = db->inter;
  db->view.goff = db->goff;
  db->view.glen = db->glen;
  db->view.cont = db->cont;
  db->view.coff = db->coff;
  db->view.clen = db->clen;
  db->view.perm = db->perm;
  db->view.n = N;
  db->view.groups = G;
  db->view.max_len = max_len;
  db->glen_h = std::move(glen);
  db->cres_h.assign((size_t)N + 1, 0);
  for (int64_t s = 0; s < N; s++) db->cres_h[s + 1] = db->cres_h[s] + clen[s];
  db->clen_h = std::move(clen);
  db->sorted_of_h.resize((size_t)N);
  for (int64_t s2 = 0; s2 < N; s2++) db->sorted_of_h[order[s2]] = (int32_t)s2;
  *out = db;
  return SW_OK;
}

extern "C" void sw_db_destroy(sw_db* db) { db_free(db); }
extern "C" int64_t sw_db_subjects(const sw_db* db) { return db ? db->view.n : 0; }
extern "C" int64_t sw_db_residues(const sw_db* db) { return db ? db->residues : 0; }
extern "C" int32_t sw_db_max_length(const sw_db* db) { return db ? db->view.max_len : 0; }

// ---- query batch validation and parameter block ------------------------------------
struct HostBatch {
  std::vector<uint8_t> res_copy;  // only when the caller's queries live on the device
  std::vector<int32_t> len;
  std::vector<int64_t> off;
  std::vector<int32_t> order;
  const uint8_t* res = nullptr;   // host view of the residues
  int64_t total = 0;
  bool res_on_device = false;
};

static sw_status read_batch(const uint8_t* queries, const int32_t* q_lengths, int32_t nq,
                            HostBatch& hb) {
  if (nq < 0) return sw_set_error(SW_EINVAL, "n_queries < 0");
  if (nq > 0 && !q_lengths) return sw_set_error(SW_EINVAL, "q_lengths is NULL");
  hb.len.resize(nq);
  if (nq > 0) {
    if (is_device_ptr(q_lengths)) {
      CUDA_TRY(cudaMemcpy(hb.len.data(), q_lengths, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost));
    } else {
      memcpy(hb.len.data(), q_lengths, sizeof(int32_t) * nq);
    }
  }
  hb.off.resize(nq);
  hb.total = 0;
  for (int32_t i = 0; i < nq; i++) {
    if (hb.len[i] < 0) return sw_set_error(SW_EINVAL, "q_lengths[%d] < 0", i);
    hb.off[i] = hb.total;
    hb.total += hb.len[i];
  }
  if (hb.total > 0 && !queries) return sw_set_error(SW_EINVAL, "queries is NULL");
  hb.res_on_device = hb.total > 0 && is_device_ptr(queries);
  if (hb.res_on_device) {
    hb.res_copy.resize(hb.total);
    CUDA_TRY(cudaMemcpy(hb.res_copy.data(), queries, hb.total, cudaMemcpyDeviceToHost));
    hb.res = hb.res_copy.data();
  } else {
    hb.res = queries;
  }
  for (int64_t i = 0; i < hb.total; i++)
    if (hb.res[i] >= ALPHA)
      return sw_set_error(SW_EINVAL, "query residue code %d at %lld (codes are 0..23)",
                          (int)hb.res[i], (long long)i);
  hb.order.resize(nq);
  std::iota(hb.order.begin(), hb.order.end(), 0);
  std::stable_sort(hb.order.begin(), hb.order.end(),
                   [&](int32_t a, int32_t b) { return hb.len[a] > hb.len[b]; });
  return SW_OK;
}

// Largest gap penalty sum kept on the packed 16-bit path: E and F stay
// >= -(Go + Ge) >= -32768 there.
static constexpr int kPackedMaxGap = 16384;
// Searches smaller than this many cells skip the load-balancing cutoff.
static constexpr double kAutoCutoffMinCells = 1e10;
static constexpr int kMaxGap = 100000000;

static sw_status fill_scoring(SearchParams& P, int32_t gap_open, int32_t gap_extend,
                              const int8_t* matrix, bool* packed_ok) {
  if (gap_open < 0 || gap_extend < 0 || gap_open > kMaxGap || gap_extend > kMaxGap)
    return sw_set_error(SW_EINVAL, "gap penalties must be in [0, %d]", kMaxGap);
  int8_t m[ALPHA * ALPHA];
  if (matrix) {
    if (is_device_ptr(matrix)) {
      CUDA_TRY(cudaMemcpy(m, matrix, sizeof m, cudaMemcpyDeviceToHost));
    } else {
      memcpy(m, matrix, sizeof m);
    }
  } else {
    memcpy(m, kBlosum62, sizeof m);
  }
  int maxsm = 0;
  for (int a = 0; a < NCODES; a++)
    for (int b = 0; b < NCODES; b++)
      P.sm[a * NCODES + b] = (a < ALPHA && b < ALPHA) ? m[a * ALPHA + b] : (int8_t)PAD_SCORE;
  for (int i = 0; i < ALPHA * ALPHA; i++) maxsm = std::max(maxsm, (int)m[i]);
  P.go = gap_open + gap_extend;
  P.ge = gap_extend;
  P.sat_threshold = S16_LIMIT - maxsm;
  P.one = 1;
  // biased 16-bit border above row 1: H' = 0 + Go, F' = -Go + Go (both subjects)
  const uint32_t go2 = ((uint32_t)(uint16_t)P.go) * 0x00010001u;
  P.init_border = make_uint4(go2, 0u, go2, 0u);
  *packed_ok = (P.go + P.ge) <= kPackedMaxGap;
  return SW_OK;
}

// ---- plan ---------------------------------------------------------------------------------
struct sw_plan {
  sw_db* db = nullptr;
  int device = 0;           // the database's device, kept for plan_free
  sw_options opt{};
  KernelConfig kc{};        // inter-task kernel
  KernelConfig kc2{};       // inter-task kernel, two queries per word
  KernelConfig ikc{};       // int32 intra-task kernel
  int32_t max_queries = 0;
  int64_t max_residues = 0;
  int32_t g_first = 0;      // first inter-task group under the cutoff
  int32_t pair_blocks16 = 0;  // grid of pair_kernel<16>
  int32_t pair_blocks32 = 0;  // grid of pair_kernel<32>
  int32_t pair2_blocks = 0;   // grid of pair2q_kernel
  // device buffers
  uint8_t* qres = nullptr;
  int64_t* qoff = nullptr;
  int32_t* qlen = nullptr;
  int32_t* qorder = nullptr;
  int4* strips = nullptr;         // strip table of the two-query kernel
  int2* spairs = nullptr;         // its stream pairs
  int64_t strip_capacity = 0;
  int32_t spair_capacity = 0;
  int32_t* scores_dev = nullptr;  // used when the caller's scores live on the host:
                                  // allocated by the first such search
  cudaStream_t stream = nullptr;  // the stream of the search in flight
  SearchParams* params = nullptr;
  SearchState* state = nullptr;
  Scratch scr{};
  // pinned host staging
  SearchParams* params_h = nullptr;
  SearchState* state_h = nullptr;
  uint8_t* qres_h = nullptr;
  int64_t* qoff_h = nullptr;
  int32_t* qlen_h = nullptr;
  int32_t* qorder_h = nullptr;
  int4* strips_h = nullptr;
  int2* spairs_h = nullptr;
  // graphs, one per gap class (the packed kernels are compiled per class)
  cudaGraphExec_t graphs[GAP_CLASSES] = {};
  int gclass = 0;  // gap class of the search being staged
  cudaEvent_t done = nullptr;
  // before the pair kernel, before and after the inter-task kernel, after recompute
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  // the two pair-kernel widths run on two streams: fork after the reset, join
  // before the inter-task kernel
  cudaStream_t side = nullptr, side2 = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr, join2 = nullptr;
  cudaEvent_t ev_join = nullptr;  // overlap: after the pair and inter-task kernels
  bool in_flight = false;
  sw_stats stats{};
  sw_stats pending{};
};

static void plan_free(sw_plan* p) {
  if (!p) return;
  int cur = 0;
  cudaGetDevice(&cur);
  // the plan's own device: its database may already be gone (a garbage
  // collector can finalize the two in either order)
  cudaSetDevice(p->device);
  for (auto& g : p->graphs)
    if (g) cudaGraphExecDestroy(g);
  if (p->done) cudaEventDestroy(p->done);
  for (auto& e : p->ev)
    if (e) cudaEventDestroy(e);
  if (p->fork) cudaEventDestroy(p->fork);
  if (p->join) cudaEventDestroy(p->join);
  if (p->join2) cudaEventDestroy(p->join2);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  if (p->side) cudaStreamDestroy(p->side);
  if (p->side2) cudaStreamDestroy(p->side2);
  cudaFree(p->qres);
  cudaFree(p->qoff);
  cudaFree(p->qlen);
  cudaFree(p->qorder);
  cudaFree(p->strips);
  cudaFree(p->spairs);
  cudaFree(p->scores_dev);
  cudaFree(p->params);
  cudaFree(p->state);
  cudaFree(p->scr.inter_border);
  cudaFree(p->scr.intra_border);
  cudaFree(p->scr.flags);
  cudaFree(p->scr.pair_border);
  cudaFreeHost(p->params_h);
  cudaFreeHost(p->state_h);
  cudaFreeHost(p->qres_h);
  cudaFreeHost(p->qoff_h);
  cudaFreeHost(p->qlen_h);
  cudaFreeHost(p->qorder_h);
  cudaFreeHost(p->strips_h);
  cudaFreeHost(p->spairs_h);
  cudaSetDevice(cur);
  cudaGetLastError();  // a failed free or device switch leaves no stale error
  delete p;
}

extern "C" sw_status sw_plan_create(sw_db* db, int32_t max_queries, int64_t max_query_residues,
                                    const sw_options* opt, sw_plan** out) {
  sw_clear_error();
  if (!out) return sw_set_error(SW_EINVAL, "sw_plan_create: out is NULL");
  *out = nullptr;
  if (!db) return sw_set_error(SW_EINVAL, "sw_plan_create: db is NULL");
  if (max_queries < 1 || max_query_residues < 0)
    return sw_set_error(SW_EINVAL, "sw_plan_create: bad capacity");
  sw_options o;
  sw_options_default(&o);
  if (opt) o = *opt;
  if (o.rows_per_thread != 16 && o.rows_per_thread != 32)
    return sw_set_error(SW_EINVAL, "rows_per_thread must be 16 or 32");
  if (o.intra_rows != 8 && o.intra_rows != 16)
    return sw_set_error(SW_EINVAL, "intra_rows must be 8 or 16");
  if (o.warps_per_block < 1 || o.warps_per_block > 8)
    return sw_set_error(SW_EINVAL, "warps_per_block must be 1..8");
  if (o.long_cutoff < 0) return sw_set_error(SW_EINVAL, "long_cutoff < 0");
  if (o.inter_columns != 4 && o.inter_columns != 8)
    return sw_set_error(SW_EINVAL, "inter_columns must be 4 or 8");
  if (o.wide_min_len < 0 || o.wide_min_subject < 0)
    return sw_set_error(SW_EINVAL, "wide_min_len and wide_min_subject must be >= 0");
  if (o.flag_capacity < 0) return sw_set_error(SW_EINVAL, "flag_capacity < 0");
  if (o.two_query < 0 || o.two_query > 2) return sw_set_error(SW_EINVAL, "two_query must be 0, 1 or 2");
  if (o.two_query_rows != 16 && o.two_query_rows != 24 && o.two_query_rows != 32)
    return sw_set_error(SW_EINVAL, "two_query_rows must be 16, 24 or 32");
  if (o.two_query_pairs < 0) return sw_set_error(SW_EINVAL, "two_query_pairs < 0");
  if (o.two_query_long < 0 || o.two_query_long > 2)
    return sw_set_error(SW_EINVAL, "two_query_long must be 0, 1 or 2");
  CUDA_TRY(cudaSetDevice(db->device));

  sw_plan* p = new sw_plan();
  p->db = db;
  p->device = db->device;
  p->opt = o;
  p->max_queries = max_queries;
  p->max_residues = max_query_residues;
  const DbView& v = db->view;
  // groups whose longest subject exceeds the cutoff go to the intra-task kernel
  int32_t gf = 0;
  if (o.force_int32) {
    gf = v.groups;
  } else {
    while (gf < v.groups && db->glen_h[gf] > o.long_cutoff) gf++;
  }
  p->g_first = gf;
  const int32_t L_inter = gf < v.groups ? db->glen_h[gf] : 0;

  int dev_sms = 0;
  cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, db->device);
  // eight columns per wavefront need 32 rows per thread; 16 rows use four
  const int cols = o.rows_per_thread == 32 ? o.inter_columns : 4;
  const int bps = inter_blocks_per_sm(o.rows_per_thread, cols, o.warps_per_block);
  if (bps < 1) {
    plan_free(p);
    return sw_set_error(SW_ECUDA, "inter-task kernel cannot launch with %d warps (rows %d)",
                        o.warps_per_block, o.rows_per_thread);
  }
  p->kc.variant = o.rows_per_thread;
  p->kc.cols = cols;
  p->kc.warps = o.warps_per_block;
  p->kc.blocks = dev_sms * bps;
  p->kc.smem = inter_smem_bytes(o.rows_per_thread, o.warps_per_block);
  // the two-query kernel: one block per SM, as many warps as its shared memory allows
  const int warps2 = inter2q_warps(o.two_query_rows);
  const int bps2 = inter2q_blocks_per_sm(o.two_query_rows, warps2);
  if (bps2 < 1) {
    plan_free(p);
    return sw_set_error(SW_ECUDA, "two-query inter-task kernel cannot launch (rows %d)",
                        o.two_query_rows);
  }
  p->kc2.variant = o.two_query_rows;
  p->kc2.cols = 8;
  p->kc2.warps = warps2;
  p->kc2.blocks = dev_sms * bps2;
  p->kc2.smem = inter2q_smem_bytes(o.two_query_rows, warps2);
  // the two inter-task kernels run one after the other and share the border scratch
  const int64_t W = std::max<int64_t>((int64_t)p->kc.blocks * p->kc.warps,
                                      (int64_t)p->kc2.blocks * p->kc2.warps);
  // one block of INTRA_WARPS per SM: enough for the int32 items, and the
  // border scratch (one subject-length row per warp) stays bounded
  if (intra_blocks_per_sm(o.intra_rows) < 1) {
    plan_free(p);
    return sw_set_error(SW_ECUDA, "int32 intra-task kernel cannot launch (rows %d)", o.intra_rows);
  }
  p->ikc.variant = o.intra_rows;
  p->ikc.warps = INTRA_WARPS;
  p->ikc.blocks = dev_sms;
  p->ikc.smem = intra_smem_bytes(o.intra_rows);
  const int64_t WI = (int64_t)p->ikc.blocks * INTRA_WARPS;
  const int pbps16 = pair_blocks_per_sm(16), pbps32 = pair_blocks_per_sm(32);
  if (pbps16 < 1 || pbps32 < 1) {
    plan_free(p);
    return sw_set_error(SW_ECUDA, "packed intra-task kernel cannot launch");
  }
  p->pair_blocks16 = dev_sms * pbps16;
  p->pair_blocks32 = dev_sms * pbps32;
  const int p2bps = pair2q_blocks_per_sm();
  if (p2bps < 1) {
    plan_free(p);
    return sw_set_error(SW_ECUDA, "two-query packed intra-task kernel cannot launch");
  }
  p->pair2_blocks = dev_sms * p2bps;
  // the two widths may run at the same time, each on its own scratch rows;
  // the two-query kernel runs instead of them and uses the first rows
  const int64_t WP = std::max<int64_t>((int64_t)(p->pair_blocks16 + p->pair_blocks32) * PAIR_WARPS,
                                       (int64_t)p->pair2_blocks * pair2q_warps());
  p->scr.pair_rows16 = (int64_t)p->pair_blocks16 * PAIR_WARPS;

  cudaError_t e = injected_fault("alloc") ? cudaErrorMemoryAllocation : cudaSuccess;
  const int64_t nres = std::max<int64_t>(max_query_residues, 1);
  p->scr.inter_stride_vec = (int64_t)(L_inter / CHUNK) * 4 * 32;
  p->scr.intra_stride = std::max(v.max_len, 1);
  // (+4: the two-query pair kernel loads its border 4 columns ahead)
  p->scr.pair_stride = std::max(v.max_len, 1) + 4;
  p->scr.flag_capacity = o.flag_capacity > 0
                            ? (int64_t)o.flag_capacity
                            : std::min<int64_t>((int64_t)max_queries * std::max<int64_t>(v.n, 1),
                                                DEFAULT_FLAG_CAPACITY);
  if (e == cudaSuccess) e = dalloc(&p->scr.pair_border, (size_t)(WP * p->scr.pair_stride));
  if (e == cudaSuccess) e = dalloc(&p->qres, nres);
  if (e == cudaSuccess) e = dalloc(&p->qoff, max_queries);
  if (e == cudaSuccess) e = dalloc(&p->qlen, max_queries);
  if (e == cudaSuccess) e = dalloc(&p->qorder, 2 * (size_t)max_queries);  // qorder, then qpair
  // strips of the two tables (the inter-task kernel's, at least 16 rows per
  // strip, and the intra-task kernel's, 32): every query padded to whole
  // strips (at least one), and as many empty halves at most; stream pairs:
  // one per two queries at most, per table
  p->strip_capacity = 2 * (max_query_residues / 16 + 2 * (int64_t)max_queries) + 16;
  p->spair_capacity = 2 * (max_queries / 2 + 1);
  if (e == cudaSuccess) e = dalloc(&p->strips, (size_t)p->strip_capacity);
  if (e == cudaSuccess) e = dalloc(&p->spairs, (size_t)p->spair_capacity);
  if (e == cudaSuccess) e = dalloc(&p->params, 1);
  if (e == cudaSuccess) e = dalloc(&p->state, 1);
  if (e == cudaSuccess) e = dalloc(&p->scr.inter_border, (size_t)(W * std::max<int64_t>(p->scr.inter_stride_vec, 1)));
  if (e == cudaSuccess) e = dalloc(&p->scr.intra_border, (size_t)(WI * p->scr.intra_stride));
  if (e == cudaSuccess) e = dalloc(&p->scr.flags, (size_t)p->scr.flag_capacity);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&p->params_h, sizeof(SearchParams));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&p->state_h, sizeof(SearchState));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&p->qres_h, nres);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&p->qoff_h, sizeof(int64_t) * max_queries);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&p->qlen_h, sizeof(int32_t) * max_queries);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&p->qorder_h, sizeof(int32_t) * 2 * max_queries);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&p->strips_h, sizeof(int4) * p->strip_capacity);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&p->spairs_h, sizeof(int2) * p->spair_capacity);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming);
  for (auto& ev : p->ev)
    if (e == cudaSuccess) e = cudaEventCreate(&ev);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->side2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->join2, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&p->ev_join);
  if (e != cudaSuccess) {
    sw_status st = sw_set_cuda_error(e, "sw_plan_create: allocation");
    plan_free(p);
    return st;
  }
  memset(p->params_h, 0, sizeof(SearchParams));
  *out = p;
  return SW_OK;
}

extern "C" void sw_plan_destroy(sw_plan* plan) {
  if (plan && plan->in_flight) cudaEventSynchronize(plan->done);
  plan_free(plan);
}

// The device work of one search: reset the counters, then the packed
// intra-task kernel (long subjects), the inter-task kernel (the rest) and the
// int32 intra-task kernel (saturated pairs, or everything when the packed path
// is off).  Events around the kernels give their device time on the launching
// stream.  Under stream capture an event record only orders the capture
// unless it carries cudaEventRecordExternal, which makes it a real
// event-record node of the graph; outside capture that flag is illegal.
static cudaError_t record(cudaEvent_t ev, cudaStream_t s, bool capturing) {
  return capturing ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                   : cudaEventRecord(ev, s);
}

static cudaError_t enqueue_kernels(sw_plan* p, cudaStream_t s, bool capturing) {
  cudaError_t e = cudaMemsetAsync(p->state, 0, sizeof(SearchState), s);
  if (e == cudaSuccess) e = record(p->ev[0], s, capturing);
  // pair_kernel<32> on the side stream, pair_kernel<16> on this one: the two
  // persistent grids share the SMs as their blocks come and go, so their
  // tails overlap.  Under capture the fork and join become graph edges.
  if (e == cudaSuccess) e = cudaEventRecord(p->fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(p->side, p->fork, 0);
  const int gc = p->gclass;
  if (e == cudaSuccess) e = launch_pairs(32, gc, p->pair_blocks32, p->db->view, p->params, p->state, p->scr, p->side);
  // the two-query intra-task kernel, when the plan chose it for this search
  // (the subject-pair kernels then find no items and return at once)
  if (e == cudaSuccess) e = launch_pair2q(gc, p->pair2_blocks, p->db->view, p->params, p->state, p->scr, p->side);
  if (e == cudaSuccess) e = launch_pairs(16, gc, p->pair_blocks16, p->db->view, p->params, p->state, p->scr, s);
  if (p->opt.overlap_kernels) {
    // the inter-task kernel too, on a third stream and issued after the pair
    // kernels: one of its blocks needs a whole SM's registers, so it starts on
    // an SM when the pair blocks there run out of work, and no SM idles in
    // their tails
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->side2, p->fork, 0);
    if (e == cudaSuccess) e = launch_inter(p->kc, gc, p->db->view, p->params, p->state, p->scr, p->side2);
    if (e == cudaSuccess) e = launch_inter2q(p->kc2, gc, p->db->view, p->params, p->state, p->scr, p->side2);
    if (e == cudaSuccess) e = record(p->ev[2], p->side2, capturing);
    if (e == cudaSuccess) e = cudaEventRecord(p->join2, p->side2);
  }
  if (e == cudaSuccess) e = cudaEventRecord(p->join, p->side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->join, 0);
  if (e == cudaSuccess) e = record(p->ev[1], s, capturing);
  if (p->opt.overlap_kernels) {
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->join2, 0);
    if (e == cudaSuccess) e = record(p->ev_join, s, capturing);
  } else {
    if (e == cudaSuccess) e = launch_inter(p->kc, gc, p->db->view, p->params, p->state, p->scr, s);
    if (e == cudaSuccess) e = launch_inter2q(p->kc2, gc, p->db->view, p->params, p->state, p->scr, s);
    if (e == cudaSuccess) e = record(p->ev[2], s, capturing);
  }
  if (e == cudaSuccess) e = launch_intra(p->ikc, p->db->view, p->params, p->state, p->scr, s);
  if (e == cudaSuccess) e = record(p->ev[3], s, capturing);
  return e;
}

static cudaError_t run_kernels(sw_plan* p, cudaStream_t s) {
  if (!p->opt.use_graph) return enqueue_kernels(p, s, false);
  cudaGraphExec_t& graph = p->graphs[p->gclass];
  if (!graph) {
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = enqueue_kernels(p, cs, true);
      e = cudaStreamEndCapture(cs, &g);
      if (e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      graph = nullptr;
      return e;
    }
  }
  return cudaGraphLaunch(graph, s);
}

// Splits the queries of one stream pair between its two streams so that the
// longer stream is as short as the strip counts allow: an exact subset sum
// over the pair's queries (reachable sums as bit sets, one per prefix of the
// queries, then a walk back from the largest sum not above half the total).
// Dealing longest first leaves the two streams of a pair up to a query's
// length apart; this closes the gap.  Pairs of more than 64 queries keep the
// dealt split (with many short queries it is already even).
static void balance_pair(std::vector<int32_t>& a, std::vector<int32_t>& b, int64_t& la,
                         int64_t& lb, const std::vector<int64_t>& strips_of) {
  std::vector<int32_t> all(a);
  all.insert(all.end(), b.begin(), b.end());
  const size_t n = all.size();
  const int64_t S = la + lb, H = S / 2;
  if (n < 2 || n > 64 || std::max(la, lb) == S - H) return;
  const size_t W = (size_t)(H / 64 + 1);
  const uint64_t top_mask = (H % 64 == 63) ? ~0ull : ((2ull << (H % 64)) - 1);
  std::vector<uint64_t> reach((n + 1) * W, 0);
  reach[0] = 1;  // the empty set sums to 0
  for (size_t i = 0; i < n; i++) {
    const uint64_t* src = &reach[i * W];
    uint64_t* dst = &reach[(i + 1) * W];
    const int64_t sh = strips_of[all[i]];
    const size_t ws = (size_t)(sh / 64);
    const int bs = (int)(sh % 64);
    for (size_t w = 0; w < W; w++) {
      uint64_t v = src[w];
      if (w >= ws) {
        v |= src[w - ws] << bs;
        if (bs && w > ws) v |= src[w - ws - 1] >> (64 - bs);
      }
      dst[w] = v;
    }
    dst[W - 1] &= top_mask;  // sums above H are not kept
  }
  const uint64_t* fin = &reach[n * W];
  int64_t t = H;
  while (t > 0 && !((fin[t / 64] >> (t % 64)) & 1)) t--;
  if (S - t >= std::max(la, lb)) return;
  std::vector<int32_t> taken, rest;
  int64_t r = t;
  for (size_t i = n; i-- > 0;) {
    const uint64_t* prev = &reach[i * W];
    if ((prev[r / 64] >> (r % 64)) & 1) {
      rest.push_back(all[i]);  // the sum r is reachable without query i
    } else {
      taken.push_back(all[i]);
      r -= strips_of[all[i]];
    }
  }
  a.assign(rest.rbegin(), rest.rend());
  b.assign(taken.rbegin(), taken.rend());
  la = S - t;
  lb = t;
}

// Query streams for two queries per word (inter2q_kernel.cu and
// pair2q_kernel.cu): deals the batch's queries to 2K streams, longest first,
// each to the stream with the fewest strips so far (each query padded to
// whole strips of T rows, at least one), pairs streams 2k and 2k + 1 and
// balances each pair's two streams (balance_pair).
// Unless fixed_K > 0, K is the smallest power of two, at most nq / 2, for
// which the largest work item -- the longest column set (len_max) against
// the longest stream pair -- is at most `share` of one worker's share of the
// search (len_sum columns against every stream pair, over `workers`): fewer,
// longer streams pad less (a stream pair is as long as its longer stream,
// and the fewer queries a pair holds the less evenly its two streams
// split), but an item longer than a worker's share finishes late; items run
// longest first, so the last ones are short.  Writes the strip table (per strip: the
// query of each half, its first row | end bit 31; query -1 for an empty
// half) to tab and per stream pair (first strip, counted from first_strip,
// strips) to pairs.  Returns K, or 0 when the table would exceed cap strips;
// *n_strips is the table's length.
static int32_t deal_streams(const HostBatch& hb, int32_t nq, int T, int32_t fixed_K,
                            double workers, double share, double len_max, double len_sum,
                            int4* tab, int2* pairs, int64_t first_strip, int64_t cap,
                            int64_t* n_strips) {
  *n_strips = 0;
  std::vector<int64_t> strips_of((size_t)nq);
  for (int32_t i = 0; i < nq; i++) strips_of[i] = std::max<int64_t>(1, (hb.len[i] + T - 1) / T);
  std::vector<std::vector<int32_t>> streams;
  std::vector<int64_t> load;
  auto deal = [&](int32_t K) {
    streams.assign((size_t)2 * K, {});
    load.assign((size_t)2 * K, 0);
    for (int32_t i = 0; i < nq; i++) {
      const int32_t q = hb.order[i];
      size_t best = 0;
      for (size_t t = 1; t < load.size(); t++)
        if (load[t] < load[best]) best = t;
      streams[best].push_back(q);
      load[best] += strips_of[q];
    }
    for (int32_t k = 0; k < K; k++)
      balance_pair(streams[2 * k], streams[2 * k + 1], load[2 * k], load[2 * k + 1], strips_of);
  };
  auto pair_strips = [&](int32_t k) { return std::max(load[2 * k], load[2 * k + 1]); };
  int32_t K = fixed_K > 0 ? std::min(fixed_K, nq / 2) : 1;
  deal(K);
  while (fixed_K == 0 && 2 * K <= nq / 2) {
    int64_t smax = 0, ssum = 0;
    for (int32_t k = 0; k < K; k++) {
      smax = std::max(smax, pair_strips(k));
      ssum += pair_strips(k);
    }
    if (len_max * (double)smax <= share * len_sum * (double)ssum / workers) break;
    K *= 2;
    deal(K);
  }
  int64_t total = 0;
  for (int32_t k = 0; k < K; k++) total += pair_strips(k);
  if (total > cap) return 0;
  int64_t at = 0;
  for (int32_t k = 0; k < K; k++) {
    const int64_t S = pair_strips(k);
    pairs[k] = make_int2((int32_t)(first_strip + at), (int32_t)S);
    // each half walks its stream: query index, first row, end bit
    int4* t4 = tab + at;
    for (int half = 0; half < 2; half++) {
      const std::vector<int32_t>& st = streams[2 * k + half];
      size_t qi = 0;
      int64_t row = 0;
      for (int64_t s = 0; s < S; s++) {
        int32_t q = -1, first = 0;
        if (qi < st.size()) {
          q = st[qi];
          first = (int32_t)row;
          row += T;
          if (row >= (int64_t)strips_of[q] * T) {  // this query's last strip
            first |= (int32_t)0x80000000u;
            ++qi;
            row = 0;
          }
        }
        if (half == 0) {
          t4[s].x = q;
          t4[s].y = first;
        } else {
          t4[s].z = q;
          t4[s].w = first;
        }
      }
    }
    at += S;
  }
  *n_strips = at;
  return K;
}

// The short subjects' two-query layout (inter2q_kernel.cu): items are
// (stream pair, half of a 64-subject group), the workers its warps.  Returns
// K, or 0 when the one-query kernel should score the short subjects instead:
// with option two_query = 1 the two-query layout must cost less than the
// one-query kernel's 32-row strips, counting a two-query word at 0.9 of a
// one-query word (measured 0.88 on the paper-shaped search, 20 queries, and
// 0.93 on a search of two queries of 375 and 455 residues, where the
// one-query kernel is then the faster).
static int32_t plan_streams(sw_plan* p, const HostBatch& hb, int32_t nq, int32_t g_first,
                            int64_t* n_strips) {
  const int T = p->kc2.variant;
  const DbView& v = p->db->view;
  double glen_sum = 0;
  for (int32_t g = g_first; g < v.groups; g++) glen_sum += p->db->glen_h[g];
  const double glen_max = g_first < v.groups ? p->db->glen_h[g_first] : 0.0;
  const int32_t K = deal_streams(hb, nq, T, p->opt.two_query_pairs,
                                 (double)p->kc2.blocks * p->kc2.warps, 0.35, glen_max, glen_sum,
                                 p->strips_h, p->spairs_h, 0, p->strip_capacity, n_strips);
  if (K == 0) return 0;
  const int64_t cost2 = *n_strips * T;  // words per column and half-group: strips x T rows
  int64_t cost1 = 0;                    // rows per column and group
  for (int32_t i = 0; i < nq; i++) cost1 += (hb.len[i] + 31) / 32 * 32;
  if (p->opt.two_query == 1 && 2.0 * 0.9 * (double)cost2 >= (double)cost1) return 0;
  return K;
}

// The long subjects' two-query layout (pair2q_kernel.cu), its table placed
// after the short subjects' (first_strip, first_pair): items are (stream
// pair, group of PAIR2_GROUP long subjects), the workers its blocks, and the
// largest item may be one worker's share (on the paper-shaped search's long
// subjects, 1, 2, 4 and 8 stream pairs took 45.4, 35.6, 40.0 and 44.2 ms;
// the rule picks 2 there, and 1 on the long-sequence workload).  Returns
// K, or 0 when the subject-pair kernels (pair_kernel.cu) should score the
// long subjects instead: with option two_query_long = 1 when the two-query
// layout, whose passes are 1024 rows of each stream, costs more than those
// kernels' passes of 512 or 1024 rows of each query against half as many
// subject columns, counting a two-query word at 0.85 of a subject-pair word
// of pair_kernel<32> and a word of pair_kernel<16> at 1.15.
static int32_t plan_streams_long(sw_plan* p, const HostBatch& hb, int32_t nq, int64_t n_long,
                                 int64_t first_strip, int32_t first_pair, int64_t* n_strips) {
  *n_strips = 0;
  if (nq < 2 || n_long <= 0) return 0;
  const int32_t* clen = p->db->clen_h.data();
  double len_sum = 0;
  for (int64_t s = 0; s < n_long; s += PAIR2_GROUP) len_sum += clen[s];
  const int32_t K = deal_streams(hb, nq, PAIR2_STRIP, p->opt.two_query_pairs,
                                 (double)p->pair2_blocks, 1.0, clen[0],
                                 len_sum, p->strips_h + first_strip, p->spairs_h + first_pair,
                                 first_strip, p->strip_capacity - first_strip, n_strips);
  if (K == 0 || p->opt.two_query_long == 2) return K;
  // words per column of a subject
  double two = 0, one = 0;
  for (int32_t k = 0; k < K; k++) {
    const int64_t S = p->spairs_h[first_pair + k].y;
    two += (double)((S + 31) / 32) * 32 * PAIR2_STRIP;
  }
  for (int32_t i = 0; i < nq; i++) {
    const int64_t m = hb.len[i];
    one += pair_wide((int32_t)m) ? (double)((m + 1023) / 1024 * 1024) / 2
                                 : 1.15 * (double)((m + 511) / 512 * 512) / 2;
  }
  return 0.85 * two < one ? K : 0;
}

// The stream layout alone, for a given number of stream pairs (host only).
extern "C" sw_status sw_query_streams(const int32_t* q_lengths, int32_t n_queries, int32_t rows,
                                      int32_t n_pairs, int32_t* strips, int64_t strip_capacity,
                                      int32_t* pairs, int64_t* n_strips) {
  sw_clear_error();
  if (rows != 16 && rows != 24 && rows != 32)
    return sw_set_error(SW_EINVAL, "rows must be 16, 24 or 32");
  if (n_queries < 2 || n_pairs < 1 || n_pairs > n_queries / 2)
    return sw_set_error(SW_EINVAL, "n_pairs must be 1..n_queries/2 (n_queries %d)", n_queries);
  if (!q_lengths || !strips || !pairs || !n_strips || strip_capacity < 0)
    return sw_set_error(SW_EINVAL, "sw_query_streams: NULL buffer or negative capacity");
  HostBatch hb;
  hb.len.assign(q_lengths, q_lengths + n_queries);
  for (int32_t i = 0; i < n_queries; i++)
    if (hb.len[i] < 0) return sw_set_error(SW_EINVAL, "q_lengths[%d] < 0", i);
  hb.order.resize(n_queries);
  std::iota(hb.order.begin(), hb.order.end(), 0);
  std::stable_sort(hb.order.begin(), hb.order.end(),
                   [&](int32_t a, int32_t b) { return hb.len[a] > hb.len[b]; });
  // built in aligned storage, then copied: the caller's buffers need only
  // int32 alignment
  int64_t bound = 0;  // the table is at most every query's strips long
  for (int32_t i = 0; i < n_queries; i++) bound += std::max<int64_t>(1, (hb.len[i] + rows - 1) / rows);
  std::vector<int4> tab((size_t)std::min(strip_capacity, bound));
  std::vector<int2> pr((size_t)n_pairs);
  const int32_t K = deal_streams(hb, n_queries, rows, n_pairs, 1.0, 1.0, 0.0, 0.0, tab.data(),
                                 pr.data(), 0, strip_capacity, n_strips);
  if (K == 0) return sw_set_error(SW_EBUSY, "the strip table exceeds %lld strips",
                                  (long long)strip_capacity);
  memcpy(strips, tab.data(), sizeof(int4) * (size_t)*n_strips);
  memcpy(pairs, pr.data(), sizeof(int2) * (size_t)K);
  return SW_OK;
}

// Stages a batch into the plan and enqueues everything up to (not including)
// the copy of the scores to a host buffer.
static sw_status plan_enqueue(sw_plan* p, const HostBatch& hb, int32_t nq, int32_t gap_open,
                              int32_t gap_extend, const int8_t* matrix, int32_t* scores_dev,
                              cudaStream_t s) {
  if (nq > p->max_queries || hb.total > p->max_residues)
    return sw_set_error(SW_EBUSY, "batch (%d queries, %lld residues) exceeds the plan (%d, %lld)",
                        nq, (long long)hb.total, p->max_queries, (long long)p->max_residues);
  SearchParams& P = *p->params_h;
  bool packed_ok = true;
  sw_status st = fill_scoring(P, gap_open, gap_extend, matrix, &packed_ok);
  if (st != SW_OK) return st;
  const DbView& v = p->db->view;
  // packed: long subjects go to the packed intra-task kernel (subject pairs);
  // otherwise (penalties too large for 16 bits, or forced) every subject
  // goes to the int32 intra-task code
  const bool packed = packed_ok && !p->opt.force_int32;
  int32_t gf = packed ? p->g_first : v.groups;
  const double total_cells = (double)hb.total * (double)p->db->residues;
  if (packed && p->opt.auto_cutoff && total_cells >= kAutoCutoffMinCells) {
    // Load balance: a (query, group) item is 64 subjects x the group length x
    // the query length.  Groups whose largest item exceeds a quarter of one
    // warp's share of the search go to the intra-task kernel instead, where
    // each subject is its own item.  Groups are sorted longest first.  Small
    // searches (a few milliseconds) are left alone.
    const double warps = (double)p->kc.blocks * p->kc.warps;
    const double share = total_cells / warps;
    const int32_t mmax = hb.len[hb.order[0]];
    while (gf < v.groups && (double)GROUP * p->db->glen_h[gf] * mmax > 0.25 * share) gf++;
  }
  const int64_t n_long = std::min<int64_t>(v.n, (int64_t)gf * GROUP);
  P.qres = p->qres;
  P.qoff = p->qoff;
  P.qlen = p->qlen;
  P.qorder = p->qorder;
  P.scores = scores_dev;
  P.nq = nq;
  P.n_long = (int32_t)n_long;
  P.g_first = gf;
  P.n_intra_items = packed ? 0 : n_long * nq;
  // the pair kernels' queries: those for pair_kernel<32>, then those for
  // pair_kernel<16>, each longest first (none when the packed path is off)
  int32_t* qpair_h = p->qorder_h + nq;
  int32_t n32 = 0, n16 = 0;
  auto wide = [&](int32_t m) { return m >= p->opt.wide_min_len && pair_wide(m); };
  // subject pairs eligible for the wide kernel: those whose longer subject
  // has at least wide_min_subject residues (a prefix: pairs are sorted
  // longest first), or every pair when there are fewer (pair, query) items
  // than narrow warps -- then each item runs nearly alone and fewer passes win
  const int32_t npairs = packed ? (int32_t)((n_long + 1) / 2) : 0;
  int32_t nwide = 0;
  if ((int64_t)npairs * nq <= (int64_t)p->pair_blocks16 * PAIR_WARPS) {
    nwide = npairs;
  } else {
    while (nwide < npairs && p->db->clen_h[2 * (size_t)nwide] >= p->opt.wide_min_subject) nwide++;
  }
  P.pair_queries = packed ? nq : 0;
  P.n_wide_pairs = nwide;
  if (packed) {
    for (int32_t i = 0; i < nq; i++)
      if (wide(hb.len[hb.order[i]])) qpair_h[n32++] = hb.order[i];
    for (int32_t i = 0; i < nq; i++)
      if (!wide(hb.len[hb.order[i]])) qpair_h[n32 + n16++] = hb.order[i];
  }
  P.qpair = p->qorder + nq;
  P.nq_pair32 = n32;
  P.nq_pair16 = n16;
  P.n_inter_items = (int64_t)(v.groups - gf) * nq;
  // two queries per word for the short subjects, when the plan's options and
  // the cost model say so (the one-query kernel then has no items)
  P.strips = p->strips;
  P.spairs = p->spairs;
  P.n_spairs = 0;
  P.n_inter2_items = 0;
  int64_t n_strips = 0;
  if (packed && gf < v.groups && nq >= 2 && p->opt.two_query > 0) {
    const int32_t K = plan_streams(p, hb, nq, gf, &n_strips);
    if (K > 0) {
      P.n_spairs = K;
      P.n_inter2_items = (int64_t)K * 2 * (v.groups - gf);
      P.n_inter_items = 0;
    } else {
      n_strips = 0;
    }
  }
  // and for the long subjects (the subject-pair kernels then have no items);
  // its table follows the short subjects' in the same buffers
  P.strips2 = p->strips;
  P.spairs2 = p->spairs + P.n_spairs;
  P.n_spairs2 = 0;
  P.n_pair2_items = 0;
  int64_t n_strips2 = 0;
  if (packed && n_long > 0 && nq >= 2 && p->opt.two_query_long > 0) {
    const int32_t K2 = plan_streams_long(p, hb, nq, n_long, n_strips, P.n_spairs, &n_strips2);
    if (K2 > 0) {
      P.n_spairs2 = K2;
      P.n_pair2_items = (int64_t)K2 * ((n_long + PAIR2_GROUP - 1) / PAIR2_GROUP);
      P.pair_queries = 0;
      P.n_wide_pairs = 0;
      P.nq_pair32 = 0;
      P.nq_pair16 = 0;
    } else {
      n_strips2 = 0;
    }
  }
  memcpy(p->qoff_h, hb.off.data(), sizeof(int64_t) * nq);
  memcpy(p->qlen_h, hb.len.data(), sizeof(int32_t) * nq);
  memcpy(p->qorder_h, hb.order.data(), sizeof(int32_t) * nq);
  if (hb.total > 0) memcpy(p->qres_h, hb.res, (size_t)hb.total);
  if (injected_fault("copy"))
    return sw_set_cuda_error(cudaErrorInvalidValue, "query upload (injected fault)");
  CUDA_TRY(cudaMemcpyAsync(p->qres, p->qres_h, (size_t)std::max<int64_t>(hb.total, 1), cudaMemcpyHostToDevice, s));
  if (nq > 0) {
    CUDA_TRY(cudaMemcpyAsync(p->qoff, p->qoff_h, sizeof(int64_t) * nq, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(p->qlen, p->qlen_h, sizeof(int32_t) * nq, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(p->qorder, p->qorder_h, sizeof(int32_t) * 2 * nq, cudaMemcpyHostToDevice, s));
  }
  if (P.n_spairs + P.n_spairs2 > 0) {
    CUDA_TRY(cudaMemcpyAsync(p->strips, p->strips_h, sizeof(int4) * (n_strips + n_strips2),
                             cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(p->spairs, p->spairs_h, sizeof(int2) * (P.n_spairs + P.n_spairs2),
                             cudaMemcpyHostToDevice, s));
  }
  CUDA_TRY(cudaMemcpyAsync(p->params, p->params_h, sizeof(SearchParams), cudaMemcpyHostToDevice, s));
  p->stream = s;
  p->gclass = gap_class(P.go, P.ge);
  CUDA_TRY(run_kernels(p, s));
  CUDA_TRY(cudaMemcpyAsync(p->state_h, p->state, sizeof(SearchState), cudaMemcpyDeviceToHost, s));
  p->pending = sw_stats{};
  int64_t qsum = hb.total;
  p->pending.cells = qsum * p->db->residues;
  p->pending.inter_items = P.n_inter_items;
  p->pending.inter2_items = P.n_inter2_items;
  p->pending.pair2_items = P.n_pair2_items;
  p->pending.intra_items = n_long * nq;  // (query, long subject) pairs, packed or int32
  p->pending.inter_cells = qsum * (p->db->residues - p->db->cres_h[n_long]);
  p->pending.kernels_launched = 6;
  return SW_OK;
}

static void finish_stats(sw_plan* p) {
  p->stats = p->pending;
  // with overlap_kernels the pair and inter-task kernels both start at ev[0]
  const bool ov = p->opt.overlap_kernels != 0;
  if (cudaEventElapsedTime(&p->stats.pair_ms, p->ev[0], p->ev[1]) != cudaSuccess ||
      cudaEventElapsedTime(&p->stats.search_ms, ov ? p->ev[0] : p->ev[1], p->ev[2]) != cudaSuccess ||
      cudaEventElapsedTime(&p->stats.recompute_ms, ov ? p->ev_join : p->ev[2], p->ev[3]) !=
          cudaSuccess) {
    cudaGetLastError();
    p->stats.pair_ms = p->stats.search_ms = p->stats.recompute_ms = -1.f;
  }
  p->stats.recomputed_pairs = (int64_t)p->state_h->n_flags;
  p->in_flight = false;
}

// More saturated pairs than the flag list holds: the packed kernels wrote
// FLAG_SENTINEL for those that found it full.  Each round collects the
// marked pairs into the list (counting all of them) and recomputes the
// listed ones in int32, whose exact scores replace the marks; the round in
// which every marked pair fits the list is the last.  Runs after the search
// has completed, synchronously on its stream.
static cudaError_t overflow_rounds(sw_plan* p, int32_t* rounds) {
  *rounds = 0;
  cudaStream_t s = p->stream;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->db->device);
  unsigned long long nf = p->state_h->n_flags;
  while (nf > (unsigned long long)p->scr.flag_capacity) {
    cudaError_t e = cudaMemsetAsync(p->state, 0, sizeof(SearchState), s);
    if (e == cudaSuccess) e = launch_collect(4 * std::max(sms, 1), p->db->view, p->params, p->state, p->scr, s);
    if (e == cudaSuccess) e = launch_intra(p->ikc, p->db->view, p->params, p->state, p->scr, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->state_h, p->state, sizeof(SearchState), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    nf = p->state_h->n_flags;
    ++*rounds;
  }
  return cudaSuccess;
}

// Statistics, then any overflow rounds, of a search that has completed.
static sw_status complete_search(sw_plan* p) {
  finish_stats(p);
  cudaError_t e = overflow_rounds(p, &p->stats.overflow_rounds);
  if (e != cudaSuccess) return sw_set_cuda_error(e, "recompute of the flag-list overflow");
  return SW_OK;
}

extern "C" sw_status sw_plan_search(sw_plan* plan, const uint8_t* queries, const int32_t* q_lengths,
                                    int32_t n_queries, int32_t gap_open, int32_t gap_extend,
                                    const int8_t* matrix, int32_t* scores, void* stream) {
  sw_clear_error();
  if (!plan) return sw_set_error(SW_EINVAL, "plan is NULL");
  if (plan->in_flight) return sw_set_error(SW_EBUSY, "plan has a search in flight");
  CUDA_TRY(cudaSetDevice(plan->db->device));
  HostBatch hb;
  sw_status st = read_batch(queries, q_lengths, n_queries, hb);
  if (st != SW_OK) return st;
  const int64_t N = plan->db->view.n;
  if (n_queries > 0 && N > 0 && !scores) return sw_set_error(SW_EINVAL, "scores is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const bool dev_out = is_device_ptr(scores);
  if (!dev_out && !plan->scores_dev) {
    // scores for a host buffer are staged on the device: the first such
    // search allocates the plan's staging buffer
    cudaError_t ea = injected_fault("alloc") ? cudaErrorMemoryAllocation
                                             : dalloc(&plan->scores_dev,
                                                      (size_t)plan->max_queries * std::max<int64_t>(N, 1));
    if (ea != cudaSuccess) {
      plan->scores_dev = nullptr;
      return sw_set_cuda_error(ea, "sw_plan_search: host-order scores buffer");
    }
  }
  int32_t* target = dev_out ? scores : plan->scores_dev;
  st = plan_enqueue(plan, hb, n_queries, gap_open, gap_extend, matrix, target, s);
  if (st != SW_OK) return st;
  plan->in_flight = true;
  const size_t out_bytes = sizeof(int32_t) * (size_t)n_queries * (size_t)N;
  if (!dev_out && out_bytes > 0)
    CUDA_TRY(cudaMemcpyAsync(scores, plan->scores_dev, out_bytes, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaEventRecord(plan->done, s));
  cudaError_t e = cudaEventSynchronize(plan->done);
  if (e != cudaSuccess) {
    finish_stats(plan);
    return sw_set_cuda_error(e, "sw_plan_search");
  }
  st = complete_search(plan);
  if (st != SW_OK) return st;
  if (plan->stats.overflow_rounds > 0 && !dev_out && out_bytes > 0) {
    // the copy above predates the overflow rounds' scores
    CUDA_TRY(cudaMemcpyAsync(scores, plan->scores_dev, out_bytes, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  CUDA_TRY(cudaGetLastError());
  return SW_OK;
}

extern "C" sw_status sw_plan_search_async(sw_plan* plan, const uint8_t* queries,
                                          const int32_t* q_lengths, int32_t n_queries,
                                          int32_t gap_open, int32_t gap_extend,
                                          const int8_t* matrix, int32_t* scores, void* stream) {
  sw_clear_error();
  if (!plan) return sw_set_error(SW_EINVAL, "plan is NULL");
  if (plan->in_flight) return sw_set_error(SW_EBUSY, "plan has a search in flight");
  CUDA_TRY(cudaSetDevice(plan->db->device));
  HostBatch hb;
  sw_status st = read_batch(queries, q_lengths, n_queries, hb);
  if (st != SW_OK) return st;
  if (n_queries > 0 && plan->db->view.n > 0 && !is_device_ptr(scores))
    return sw_set_error(SW_EINVAL, "sw_plan_search_async needs device scores");
  cudaStream_t s = (cudaStream_t)stream;
  st = plan_enqueue(plan, hb, n_queries, gap_open, gap_extend, matrix, scores, s);
  if (st != SW_OK) return st;
  CUDA_TRY(cudaEventRecord(plan->done, s));
  plan->in_flight = true;
  return SW_OK;
}

extern "C" sw_status sw_plan_wait(sw_plan* plan, int32_t timeout_ms) {
  if (!plan) return sw_set_error(SW_EINVAL, "plan is NULL");
  if (!plan->in_flight) return SW_OK;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaEventQuery(plan->done);
    if (e == cudaSuccess) return complete_search(plan);
    if (e != cudaErrorNotReady) {
      plan->in_flight = false;
      return sw_set_cuda_error(e, "sw_plan_wait");
    }
    if (timeout_ms >= 0) {
      const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      if (ms >= timeout_ms) return sw_set_error(SW_ETIMEDOUT, "search still running after %d ms", timeout_ms);
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

extern "C" sw_status sw_plan_stats(const sw_plan* plan, sw_stats* out) {
  if (!plan || !out) return sw_set_error(SW_EINVAL, "NULL argument");
  *out = plan->stats;
  return SW_OK;
}

extern "C" sw_status sw_search(sw_db* db, const uint8_t* queries, const int32_t* q_lengths,
                               int32_t n_queries, int32_t gap_open, int32_t gap_extend,
                               const int8_t* matrix, int32_t* scores, void* stream) {
  sw_clear_error();
  if (!db) return sw_set_error(SW_EINVAL, "db is NULL");
  CUDA_TRY(cudaSetDevice(db->device));
  HostBatch hb;
  sw_status st = read_batch(queries, q_lengths, n_queries, hb);
  if (st != SW_OK) return st;
  std::lock_guard<std::mutex> guard(db->oneshot_mu);
  sw_plan*& plan = db->oneshot;
  int32_t want_q = std::max(n_queries, 1);
  int64_t want_res = hb.total;
  if (plan && (plan->max_queries < want_q || plan->max_residues < want_res)) {
    want_q = std::max(want_q, plan->max_queries);
    want_res = std::max(want_res, plan->max_residues);
    plan_free(plan);
    plan = nullptr;
  }
  if (!plan) {
    sw_options o;
    sw_options_default(&o);
    st = sw_plan_create(db, want_q, want_res, &o, &plan);
    if (st != SW_OK) {
      plan = nullptr;
      return st;
    }
  }
  return sw_plan_search(plan, queries, q_lengths, n_queries, gap_open, gap_extend, matrix, scores,
                        stream);
}

// ---- plain baseline ----------------------------------------------------------------------
extern "C" sw_status sw_search_plain(sw_db* db, const uint8_t* queries, const int32_t* q_lengths,
                                     int32_t n_queries, int32_t gap_open, int32_t gap_extend,
                                     const int8_t* matrix, int32_t* scores, void* stream) {
  sw_clear_error();
  if (!db) return sw_set_error(SW_EINVAL, "db is NULL");
  CUDA_TRY(cudaSetDevice(db->device));
  HostBatch hb;
  sw_status st = read_batch(queries, q_lengths, n_queries, hb);
  if (st != SW_OK) return st;
  const DbView& v = db->view;
  const int64_t N = v.n;
  if (n_queries > 0 && N > 0 && !scores) return sw_set_error(SW_EINVAL, "scores is NULL");
  SearchParams P;
  memset(&P, 0, sizeof P);
  bool packed_ok;
  st = fill_scoring(P, gap_open, gap_extend, matrix, &packed_ok);
  if (st != SW_OK) return st;
  if (n_queries == 0 || N == 0) return SW_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, db->device);
  const int bps = std::max(1, std::min(plain_blocks_per_sm(), 8));
  const int grid = (int)std::min<int64_t>((int64_t)sms * bps, v.groups);
  std::vector<int64_t> boff(grid);
  int64_t btotal = 0;
  for (int b = 0; b < grid; b++) {
    boff[b] = btotal;
    btotal += (int64_t)db->glen_h[b] * GROUP;  // a block's first group is its longest
  }
  const bool dev_out = is_device_ptr(scores);
  uint8_t* qres = nullptr;
  int64_t *qoff = nullptr, *boff_d = nullptr;
  int32_t *qlen = nullptr, *sc = nullptr;
  int2* border = nullptr;
  SearchParams* Pd = nullptr;
  cudaError_t e = dalloc(&qres, hb.total);
  if (e == cudaSuccess) e = dalloc(&qoff, n_queries);
  if (e == cudaSuccess) e = dalloc(&qlen, n_queries);
  if (e == cudaSuccess) e = dalloc(&boff_d, grid);
  if (e == cudaSuccess) e = dalloc(&border, btotal);
  if (e == cudaSuccess) e = dalloc(&Pd, 1);
  if (e == cudaSuccess && !dev_out) e = dalloc(&sc, (size_t)n_queries * N);
  if (e == cudaSuccess && hb.total > 0)
    e = cudaMemcpyAsync(qres, hb.res, hb.total, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(qoff, hb.off.data(), sizeof(int64_t) * n_queries, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(qlen, hb.len.data(), sizeof(int32_t) * n_queries, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(boff_d, boff.data(), sizeof(int64_t) * grid, cudaMemcpyHostToDevice, s);
  P.qres = qres;
  P.qoff = qoff;
  P.qlen = qlen;
  P.scores = dev_out ? scores : sc;
  P.nq = n_queries;
  if (e == cudaSuccess) e = cudaMemcpyAsync(Pd, &P, sizeof P, cudaMemcpyHostToDevice, s);
  for (int32_t q = 0; q < n_queries && e == cudaSuccess; q++)
    e = launch_plain(grid, v, Pd, q, border, boff_d, s);
  if (e == cudaSuccess && !dev_out)
    e = cudaMemcpyAsync(scores, sc, sizeof(int32_t) * (size_t)n_queries * N, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(qres);
  cudaFree(qoff);
  cudaFree(qlen);
  cudaFree(boff_d);
  cudaFree(border);
  cudaFree(Pd);
  cudaFree(sc);
  if (e != cudaSuccess) return sw_set_cuda_error(e, "sw_search_plain");
  return SW_OK;
}

// ---- optimal alignments with traceback ------------------------------------------------------
// Largest direction-bit buffer of one chunk of pairs (bytes).
static constexpr int64_t kAlignChunkBytes = 8ll << 30;

extern "C" sw_status sw_align(sw_db* db, const uint8_t* queries, const int32_t* q_lengths,
                              int32_t n_queries, const int32_t* pair_query,
                              const int64_t* pair_subject, int32_t n_pairs, int32_t gap_open,
                              int32_t gap_extend, const int8_t* matrix, sw_alignment* out,
                              uint8_t* ops, int64_t ops_capacity, void* stream) {
  sw_clear_error();
  if (!db) return sw_set_error(SW_EINVAL, "db is NULL");
  if (n_pairs < 0) return sw_set_error(SW_EINVAL, "n_pairs < 0");
  if (n_pairs > 0 && (!pair_query || !pair_subject || !out))
    return sw_set_error(SW_EINVAL, "pair_query, pair_subject or out is NULL");
  CUDA_TRY(cudaSetDevice(db->device));
  HostBatch hb;
  sw_status st = read_batch(queries, q_lengths, n_queries, hb);
  if (st != SW_OK) return st;
  SearchParams P;
  memset(&P, 0, sizeof P);
  bool packed_ok;
  st = fill_scoring(P, gap_open, gap_extend, matrix, &packed_ok);
  if (st != SW_OK) return st;
  const int64_t N = db->view.n;
  // per pair: sorted subject, sizes, and its transcript slot
  std::vector<AlignItem> items((size_t)n_pairs);
  std::vector<int64_t> slot((size_t)n_pairs + 1, 0);
  for (int32_t k = 0; k < n_pairs; k++) {
    const int32_t q = pair_query[k];
    const int64_t sub = pair_subject[k];
    if (q < 0 || q >= n_queries)
      return sw_set_error(SW_EINVAL, "pair_query[%d] = %d is not a query index", k, q);
    if (sub < 0 || sub >= N)
      return sw_set_error(SW_EINVAL, "pair_subject[%d] = %lld is not a subject index", k,
                          (long long)sub);
    const int32_t s = db->sorted_of_h[(size_t)sub];
    items[k].q = q;
    items[k].s = s;
    slot[k + 1] = slot[k] + hb.len[q] + db->clen_h[s];
  }
  if (n_pairs > 0 && slot[n_pairs] > 0 && (!ops || ops_capacity < slot[n_pairs]))
    return sw_set_error(SW_EINVAL, "ops needs %lld bytes, has %lld", (long long)slot[n_pairs],
                        (long long)ops_capacity);
  if (n_pairs == 0) return SW_OK;
  // few pairs: a block of 16 warps per pair; many: a warp per pair
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, db->device);
  const bool block_mode = n_pairs <= std::max(sms, 1);
  const int64_t border_rows = block_mode ? ALIGN_BLOCK_ROWS : 1;
  // chunks of pairs whose direction bits fit kAlignChunkBytes (one pair may exceed it alone)
  std::vector<int32_t> chunk_begin{0};
  int64_t words = 0, max_words = 0, max_border = 0, border = 0;
  for (int32_t k = 0; k < n_pairs; k++) {
    const int64_t w = align_bits_words(hb.len[items[k].q], db->clen_h[items[k].s]);
    if (k > chunk_begin.back() && 4 * (words + w) > kAlignChunkBytes) {
      chunk_begin.push_back(k);
      words = border = 0;
    }
    items[k].bits_off = words;
    items[k].border_off = border;
    items[k].ops_end = slot[k + 1];
    words += w;
    border += border_rows * db->clen_h[items[k].s];
    max_words = std::max(max_words, words);
    max_border = std::max(max_border, border);
  }
  chunk_begin.push_back(n_pairs);
  cudaStream_t cs = (cudaStream_t)stream;
  uint8_t* qres = nullptr;
  int64_t* qoff = nullptr;
  int32_t* qlen = nullptr;
  SearchParams* Pd = nullptr;
  AlignItem* items_d = nullptr;
  AlignOut* out_d = nullptr;
  uint32_t* bits = nullptr;
  int2* border_d = nullptr;
  uint8_t* ops_d = nullptr;
  std::vector<AlignOut> res((size_t)n_pairs);
  cudaError_t e = dalloc(&qres, std::max<int64_t>(hb.total, 1));
  if (e == cudaSuccess) e = dalloc(&qoff, std::max(n_queries, 1));
  if (e == cudaSuccess) e = dalloc(&qlen, std::max(n_queries, 1));
  if (e == cudaSuccess) e = dalloc(&Pd, 1);
  if (e == cudaSuccess) e = dalloc(&items_d, n_pairs);
  if (e == cudaSuccess) e = dalloc(&out_d, n_pairs);
  if (e == cudaSuccess) e = dalloc(&bits, std::max<int64_t>(max_words, 1));
  if (e == cudaSuccess) e = dalloc(&border_d, std::max<int64_t>(max_border, 1));
  if (e == cudaSuccess) e = dalloc(&ops_d, std::max<int64_t>(slot[n_pairs], 1));
  if (e == cudaSuccess && hb.total > 0)
    e = cudaMemcpyAsync(qres, hb.res, hb.total, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess && n_queries > 0)
    e = cudaMemcpyAsync(qoff, hb.off.data(), sizeof(int64_t) * n_queries, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess && n_queries > 0)
    e = cudaMemcpyAsync(qlen, hb.len.data(), sizeof(int32_t) * n_queries, cudaMemcpyHostToDevice, cs);
  P.qres = qres;
  P.qoff = qoff;
  P.qlen = qlen;
  P.nq = n_queries;
  if (e == cudaSuccess) e = cudaMemcpyAsync(Pd, &P, sizeof P, cudaMemcpyHostToDevice, cs);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(items_d, items.data(), sizeof(AlignItem) * n_pairs, cudaMemcpyHostToDevice, cs);
  for (size_t c = 0; c + 1 < chunk_begin.size() && e == cudaSuccess; c++) {
    const int32_t k0 = chunk_begin[c], nk = chunk_begin[c + 1] - k0;
    e = launch_align(db->view, Pd, items_d + k0, nk, block_mode, bits, border_d, out_d + k0, ops_d,
                     cs);
    // the next chunk reuses the bits: its kernels run after this one's on the stream
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(res.data(), out_d, sizeof(AlignOut) * n_pairs, cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess && slot[n_pairs] > 0)
    e = cudaMemcpyAsync(ops, ops_d, (size_t)slot[n_pairs], cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  cudaFree(qres);
  cudaFree(qoff);
  cudaFree(qlen);
  cudaFree(Pd);
  cudaFree(items_d);
  cudaFree(out_d);
  cudaFree(bits);
  cudaFree(border_d);
  cudaFree(ops_d);
  if (e != cudaSuccess) return sw_set_cuda_error(e, "sw_align");
  for (int32_t k = 0; k < n_pairs; k++) {
    const AlignOut& r = res[k];
    out[k].score = r.score;
    out[k].q_begin = r.q_begin;
    out[k].q_end = r.score > 0 ? r.i_end : 0;
    out[k].s_begin = r.s_begin;
    out[k].s_end = r.score > 0 ? r.j_end : 0;
    out[k].n_ops = r.n_ops;
    out[k].ops_offset = r.ops_offset;
  }
  return SW_OK;
}

// ---- microbenchmark ----------------------------------------------------------------------
extern "C" sw_status sw_intpeak(int32_t op, int32_t blocks_per_sm, int32_t threads, int32_t iters,
                                double* out) {
  sw_clear_error();
  if (!out) return sw_set_error(SW_EINVAL, "out is NULL");
  int rc = intpeak_run(op, blocks_per_sm, threads, iters, &out[0], &out[1], &out[2]);
  if (rc == SW_EINVAL) return sw_set_error(SW_EINVAL, "sw_intpeak: bad arguments");
  return (sw_status)rc;
}
