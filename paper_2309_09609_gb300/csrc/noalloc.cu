// noalloc.cu -- sw_search_pairs_noalloc: exact scores without allocating memory.
//
// Every other search entry point allocates device memory (a database, a plan,
// scratch for the kernels).  Some callers cannot allow that: a host framework
// that owns every device allocation through its own pool, a service that
// must not allocate once it is serving (so memory use stays fixed and no call
// can fail with out-of-memory), or code that is not permitted to call
// cudaMalloc at all.  This entry point takes the caller's device buffers for
// inputs and outputs and keeps its scratch -- one (H, F) border row per warp,
// a work counter and a status word -- in the file-scope array below, whose
// size is fixed at build time.  Every GPU that loads the library holds that
// array until the process exits.
//
// The kernel is a variant of the int32 intra-task warp wavefront of
// intra_kernel.cu: one warp per (query, subject) pair, lane k owning TI
// query rows of a 32*TI-row pass, (H, F) borders handed to the next lane by
// __shfl_up_sync, and the border between passes kept in this array.
#include <mutex>

#include "swgb_internal.h"

namespace swgb {
namespace {

constexpr int NA_MAX_LEN = 4096;         // longest subject accepted
constexpr int NA_WARPS_PER_BLOCK = 4;
constexpr int NA_BLOCKS = 128;
constexpr int NA_WARPS = NA_BLOCKS * NA_WARPS_PER_BLOCK;
constexpr int NA_TI = 8;                 // query rows per lane
constexpr int NA_HEADER = 32;            // int2 slots (256 bytes) for the counter and status
constexpr size_t NA_SCRATCH = NA_HEADER + (size_t)NA_WARPS * NA_MAX_LEN;  // int2: ~16 MiB
constexpr unsigned NA_FULL = 0xffffffffu;
constexpr unsigned NA_BAD_LENGTH = 1u, NA_BAD_CODE = 2u;

// The scratch of sw_search_pairs_noalloc.  In host code this name is only a
// stand-in for the device array: its device address comes from
// cudaGetSymbolAddress, once per device (see scratch_for_current_device).
static __device__ __align__(256) int2 g_noalloc_scratch[NA_SCRATCH];

struct NaMatrix {
  int8_t sm[NCODES * NCODES];  // SM(query code, subject code), PAD row/column = PAD_SCORE
};

__device__ __forceinline__ int na_sext_byte(uint32_t w, int k) {
  uint32_t r;
  const uint32_t sel = (uint32_t)(k | ((8 | k) << 4) | ((8 | k) << 8) | ((8 | k) << 12));
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(w), "r"(0u), "r"(sel));
  return (int)r;
}

__global__ void __launch_bounds__(NA_WARPS_PER_BLOCK * 32)
noalloc_kernel(const uint8_t* __restrict__ qres, const int64_t* __restrict__ qoff,
               const int32_t* __restrict__ qlen, int nq, const uint8_t* __restrict__ sres,
               const int64_t* __restrict__ soff, const int32_t* __restrict__ slen, int ns,
               int go, int ge, NaMatrix mat, int32_t* __restrict__ scores, int2* scratch) {
  __shared__ __align__(16) uint8_t prof_all[NA_WARPS_PER_BLOCK][NCODES * 32 * NA_TI];
  __shared__ int8_t sm[NCODES * NCODES];
  for (int i = threadIdx.x; i < NCODES * NCODES; i += blockDim.x) sm[i] = mat.sm[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint8_t* prof = prof_all[wib];
  unsigned long long* next = (unsigned long long*)scratch;
  unsigned int* status = (unsigned int*)(scratch + 1);
  int2* hb = scratch + NA_HEADER + (size_t)(blockIdx.x * NA_WARPS_PER_BLOCK + wib) * NA_MAX_LEN;
  const long long total = (long long)nq * ns;
  constexpr int ROWS = 32 * NA_TI;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(next, 1ull);
    it = __shfl_sync(NA_FULL, it, 0);
    if ((long long)it >= total) break;
    const int q = (int)((long long)it / ns), s = (int)((long long)it % ns);
    const int m = qlen[q], n = slen[s];
    // rejected, with nothing read or written: a negative length, a subject
    // over the limit, or residues to read from a NULL buffer
    if (m < 0 || n < 0 || n > NA_MAX_LEN || (m > 0 && !qres) || (n > 0 && !sres)) {
      if (lane == 0) atomicOr(status, NA_BAD_LENGTH);
      continue;
    }
    const uint8_t* qr = qres + (m > 0 ? qoff[q] : 0);
    const uint8_t* d = sres + (n > 0 ? soff[s] : 0);
    const int npass = (m + ROWS - 1) / ROWS;
    int S = 0;
    int bad = 0;  // this lane met a residue code >= 24: the pair gets no score
    for (int p = 0; p < npass && n > 0; p++) {
      __syncwarp();
      const int i0 = p * ROWS + lane * NA_TI;
      int qc[NA_TI];
#pragma unroll
      for (int r = 0; r < NA_TI; r++) {
        int c = (i0 + r < m) ? (int)qr[i0 + r] : -1;
        if (c >= ALPHA) {
          atomicOr(status, NA_BAD_CODE);
          bad = 1;
          c = -1;
        }
        qc[r] = c;
      }
      for (int c = 0; c < NCODES; c++) {
        uint32_t w0 = 0, w1 = 0;
#pragma unroll
        for (int r = 0; r < NA_TI; r++) {
          const int v = qc[r] >= 0 ? (int)sm[qc[r] * NCODES + c] : PAD_SCORE;
          const uint32_t b = (uint32_t)(uint8_t)(int8_t)v << (8 * (r & 3));
          if (r < 4) w0 |= b; else w1 |= b;
        }
        *(uint2*)(prof + (c * 32 + lane) * NA_TI) = make_uint2(w0, w1);
      }
      __syncwarp();
      int Hp[NA_TI], E[NA_TI];
#pragma unroll
      for (int r = 0; r < NA_TI; r++) {
        Hp[r] = 0;
        E[r] = -go;
      }
      int hdiag = 0, out_h = 0, out_f = -go;
      const bool last_pass = (p == npass - 1);
      for (int t = 0; t < n + 31; t++) {
        int in_h = __shfl_up_sync(NA_FULL, out_h, 1);
        int in_f = __shfl_up_sync(NA_FULL, out_f, 1);
        const int j = t - lane;
        if (lane == 0) {
          if (p > 0 && j < n) {
            const int2 v = hb[j];
            in_h = v.x;
            in_f = v.y;
          } else {
            in_h = 0;
            in_f = -go;
          }
        }
        if (j >= 0 && j < n) {
          int c = d[j];
          if (c >= ALPHA) {
            atomicOr(status, NA_BAD_CODE);
            bad = 1;
            c = PAD_CODE;  // keeps the profile read in bounds; the score is dropped
          }
          const uint2 pw = *(const uint2*)(prof + (c * 32 + lane) * NA_TI);
          int hd = hdiag;
          hdiag = in_h;
          int f = in_f;
#pragma unroll
          for (int r = 0; r < NA_TI; r++) {
            const int w = na_sext_byte(r < 4 ? pw.x : pw.y, r & 3);
            const int e = E[r];
            const int h = max(max(hd + w, max(e, f)), 0);
            hd = Hp[r];
            Hp[r] = h;
            const int tt = h - go;
            E[r] = max(e - ge, tt);
            f = max(f - ge, tt);
            S = max(S, h);
          }
          out_h = Hp[NA_TI - 1];
          out_f = f;
          if (lane == 31 && !last_pass) hb[j] = make_int2(out_h, out_f);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) S = max(S, __shfl_xor_sync(NA_FULL, S, o));
    if (__any_sync(NA_FULL, bad)) continue;  // warp-uniform: the pair is not scored
    if (lane == 0) scores[(long long)q * ns + s] = S;
  }
}

// True when p is device memory of device `dev` (or managed memory), which a
// kernel launched on `dev` may read and write.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

std::mutex g_na_lock;
int2* g_na_ptr[64] = {};

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (cudaGetSymbolAddress needs that device current).
sw_status scratch_for_current_device(int2** out) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return sw_set_error(SW_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> g(g_na_lock);
  if (!g_na_ptr[dev]) {
    int2* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess) return sw_set_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_na_ptr[dev] = p;
  }
  *out = g_na_ptr[dev];
  return SW_OK;
}

}  // namespace
}  // namespace swgb

using namespace swgb;

extern "C" sw_status sw_search_pairs_noalloc(const uint8_t* queries, const int64_t* q_offsets,
                                             const int32_t* q_lengths, int32_t n_queries,
                                             const uint8_t* subjects, const int64_t* s_offsets,
                                             const int32_t* s_lengths, int32_t n_subjects,
                                             int32_t gap_open, int32_t gap_extend,
                                             const int8_t* matrix, int32_t* scores,
                                             void* stream) {
  sw_clear_error();
  if (n_queries < 0 || n_subjects < 0)
    return sw_set_error(SW_EINVAL, "sw_search_pairs_noalloc: negative count");
  if (gap_open < 0 || gap_extend < 0 || gap_open > 100000000 || gap_extend > 100000000)
    return sw_set_error(SW_EINVAL, "sw_search_pairs_noalloc: gap penalties must be in [0, 1e8]");
  if (n_queries == 0 || n_subjects == 0) return SW_OK;
  // the residue buffers may be NULL when every length on that side is 0
  // (the kernel refuses to read a NULL buffer); the others are always read
  if (!q_offsets || !q_lengths || !s_offsets || !s_lengths || !scores)
    return sw_set_error(SW_EINVAL, "sw_search_pairs_noalloc: NULL buffer");
  int cur = 0;
  CUDA_TRY(cudaGetDevice(&cur));
  const void* bufs[7] = {queries, q_offsets, q_lengths, subjects, s_offsets, s_lengths, scores};
  static const char* names[7] = {"queries", "q_offsets", "q_lengths", "subjects",
                                 "s_offsets", "s_lengths", "scores"};
  for (int i = 0; i < 7; i++) {
    if (!bufs[i]) continue;
    if (!on_device(bufs[i], cur))
      return sw_set_error(SW_EINVAL, "sw_search_pairs_noalloc: %s is not device memory of the "
                          "current device (%d)", names[i], cur);
  }
  NaMatrix mat;
  int8_t m[ALPHA * ALPHA];
  if (matrix)
    for (int i = 0; i < ALPHA * ALPHA; i++) m[i] = matrix[i];
  else
    sw_default_matrix(m);
  for (int a = 0; a < NCODES; a++)
    for (int b = 0; b < NCODES; b++)
      mat.sm[a * NCODES + b] = (a < ALPHA && b < ALPHA) ? m[a * ALPHA + b] : (int8_t)PAD_SCORE;
  int2* scratch = nullptr;
  sw_status st = scratch_for_current_device(&scratch);
  if (st != SW_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // the counter and the status word must start at zero on every call
  CUDA_TRY(cudaMemsetAsync(scratch, 0, NA_HEADER * sizeof(int2), s));
  noalloc_kernel<<<NA_BLOCKS, NA_WARPS_PER_BLOCK * 32, 0, s>>>(
      queries, q_offsets, q_lengths, n_queries, subjects, s_offsets, s_lengths, n_subjects,
      gap_open + gap_extend, gap_extend, mat, scores, scratch);
  CUDA_TRY(cudaGetLastError());
  unsigned int status = 0;
  CUDA_TRY(cudaMemcpyAsync(&status, scratch + 1, sizeof status, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (status & NA_BAD_LENGTH)
    return sw_set_error(SW_EINVAL, "sw_search_pairs_noalloc: a length is negative or a subject "
                        "is longer than %d residues; those pairs were not scored", NA_MAX_LEN);
  if (status & NA_BAD_CODE)
    return sw_set_error(SW_EINVAL, "sw_search_pairs_noalloc: residue code >= 24 in the input");
  return SW_OK;
}
