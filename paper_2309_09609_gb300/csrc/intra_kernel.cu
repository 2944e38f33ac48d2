// intra_kernel.cu -- the int32 intra-task kernel of libswgb: exact scores of
// the pairs that the packed 16-bit kernels cannot score.
//
// The warp wavefront of Section II-B (intra-task parallelism with neighbour
// border exchange) in int32: lane k owns TI query rows of a 32*TI-row pass and
// sweeps the subject one step behind lane k-1, which hands it the (H, F)
// border of its last row through __shfl_up_sync.  The bottom row of a pass is
// the top border of the next one and goes through a per-warp scratch row.
//
// One launch does two kinds of work, of which a search has only one:
//   * int32 intra-task items (query, subject), one warp each -- every subject
//     when the packed path is off (forced, or gaps too large for 16 bits);
//   * the pairs flagged by the packed kernels (16-bit score at the saturation
//     threshold), one block each: the passes of the query are dealt round-robin
//     to the block's warps, pass p starting LAG stages of 32 steps after pass
//     p - 1, so a flagged pair of two 35,000-residue sequences runs on sixteen
//     warps instead of one.  Stages end at __syncthreads, which orders each
//     border write before its read and each read before the next overwrite.
#include "device_common.cuh"

namespace swgb {

template <int TI>
struct IntraSlice {
  static constexpr int BYTES = NCODES * 32 * TI;  // lane_profile<TI> of one pass
};

constexpr int LAG = 3;  // stages between the starts of consecutive passes (block items)

// The TI cells of one lane at one column: (in_h, in_f) are H and F of the row
// above the lane's first row at this column; lp is the lane's profile row of
// the column's residue.  Eq. 1-3 in the shared-gap form, int32.
template <int TI>
__device__ __forceinline__ void intra_cells(int (&Hp)[TI], int (&E)[TI], int& hdiag, int& out_h,
                                            int& out_f, int& S, int in_h, int in_f,
                                            const uint8_t* lp, int go, int ge) {
  uint32_t pw[TI / 4];
  if constexpr (TI == 8) {
    const uint2 v = *(const uint2*)lp;
    pw[0] = v.x;
    pw[1] = v.y;
  } else {
    const uint4 v = *(const uint4*)lp;
    pw[0] = v.x;
    pw[1] = v.y;
    pw[2] = v.z;
    pw[3] = v.w;
  }
  int hd = hdiag;
  hdiag = in_h;
  int f = in_f;
#pragma unroll
  for (int r = 0; r < TI; r++) {
    const int w = sext_byte(pw[r / 4], r & 3);
    const int e = E[r];
    const int h = __viaddmax_s32_relu(hd, w, max(e, f));  // Eq. 1
    hd = Hp[r];
    Hp[r] = h;
    const int tt = h - go;
    E[r] = __viaddmax_s32(e, -ge, tt);  // Eq. 2, next column
    f = __viaddmax_s32(f, -ge, tt);     // Eq. 3, next row
    S = max(S, h);
  }
  out_h = Hp[TI - 1];
  out_f = f;
}

template <int TI>
__device__ __forceinline__ void intra_start(int (&Hp)[TI], int (&E)[TI], int& hdiag, int& out_h,
                                            int& out_f, int go) {
#pragma unroll
  for (int r = 0; r < TI; r++) {
    Hp[r] = 0;   // H(i, 0)
    E[r] = -go;  // E(i, 1)
  }
  hdiag = 0;
  out_h = 0;
  out_f = -go;
}

// One (query, subject) pair on one warp, all passes in order.
template <int TI>
__device__ void intra_warp_item(const DbView& db, const SearchParams* __restrict__ P,
                                const int8_t* __restrict__ sm, uint8_t* slice, int lane,
                                int2* hb, int q, int s) {
  const int n = db.clen[s];
  const int m = P->qlen[q];
  const uint8_t* __restrict__ d = db.cont + db.coff[s];
  const uint8_t* __restrict__ qr = P->qres + P->qoff[q];
  const int go = P->go, ge = P->ge;
  constexpr int ROWS = 32 * TI;
  const int npass = (m + ROWS - 1) / ROWS;
  int S = 0;
  for (int p = 0; p < npass && n > 0; p++) {
    __syncwarp();
    lane_profile<TI>(slice, sm, qr, m, p * ROWS + lane * TI, lane);
    __syncwarp();
    int Hp[TI], E[TI], hdiag, out_h, out_f;
    intra_start<TI>(Hp, E, hdiag, out_h, out_f, go);
    const bool last_pass = (p == npass - 1);
    const int steps = n + 31;
    for (int t = 0; t < steps; t++) {
      int in_h = __shfl_up_sync(FULL, out_h, 1);
      int in_f = __shfl_up_sync(FULL, out_f, 1);
      const int j = t - lane;
      if (lane == 0) {
        if (p > 0 && j < n) {
          const int2 v = hb[j];
          in_h = v.x;
          in_f = v.y;
        } else {
          in_h = 0;    // H(0, j)
          in_f = -go;  // F(1, j)
        }
      }
      if (j >= 0 && j < n) {
        intra_cells<TI>(Hp, E, hdiag, out_h, out_f, S, in_h, in_f, slice + (d[j] * 32 + lane) * TI,
                        go, ge);
        if (lane == 31 && !last_pass) hb[j] = make_int2(out_h, out_f);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) S = max(S, __shfl_xor_sync(FULL, S, o));
  if (lane == 0) emit_score(db, P, q, s, S);
}

// One (query, subject) pair on the whole block.  Pass p runs on warp
// p % INTRA_WARPS and starts at stage (p / W) * period + (p % W) * LAG, with
// period = max(stages of a pass, LAG * W): consecutive passes are LAG stages
// apart, and a warp's next pass starts after its previous one ends.  Lane 0 of
// pass p at column j needs the bottom row of pass p - 1 at column j, written
// by that pass at its step j + 31, i.e. at most two of its stages after the
// stage holding its step j; LAG = 3 leaves one stage in between, in which the
// warp fetches the next 32 border values with one coalesced load.
template <int TI>
__device__ void intra_block_item(const DbView& db, const SearchParams* __restrict__ P,
                                 const int8_t* __restrict__ sm, uint8_t* slice, int lane, int wib,
                                 int2* border, int64_t stride, int* red, int q, int s) {
  constexpr int W = INTRA_WARPS;
  constexpr int ROWS = 32 * TI;
  const int n = db.clen[s];
  const int m = P->qlen[q];
  const uint8_t* __restrict__ d = db.cont + db.coff[s];
  const uint8_t* __restrict__ qr = P->qres + P->qoff[q];
  const int go = P->go, ge = P->ge;
  const int npass = n > 0 ? (m + ROWS - 1) / ROWS : 0;
  const int spass = (n + 31 + 31) / 32;  // stages of one pass (n + 31 steps)
  const int period = max(spass, LAG * W);
  const int nstages =
      npass > 0 ? ((npass - 1) / W) * period + ((npass - 1) % W) * LAG + spass : 0;
  int2* own = border + wib * stride;                    // bottom rows of this warp's passes
  const int2* src = border + ((wib + W - 1) % W) * stride;  // those of the pass before
  const int2 top = make_int2(0, -go);                   // (H(0, j), F(1, j))
  int S = 0;
  int Hp[TI], E[TI], hdiag = 0, out_h = 0, out_f = -go;
  int p = 0;
  int2 bcur = top, bnext = top;  // border of columns 32k + lane and 32(k + 1) + lane
  for (int g = 0; g < nstages; g++) {
    const int rel = g - wib * LAG;
    int k = -1;
    if (rel >= 0) {
      const int r = rel / period;
      const int kk = rel - r * period;
      if (kk < spass && wib + r * W < npass) {
        k = kk;
        p = wib + r * W;
      }
    }
    if (k >= 0) {  // warp-uniform
      if (k == 0) {
        __syncwarp();
        lane_profile<TI>(slice, sm, qr, m, p * ROWS + lane * TI, lane);
        __syncwarp();
        intra_start<TI>(Hp, E, hdiag, out_h, out_f, go);
        bcur = (p > 0 && lane < n) ? src[lane] : top;
      } else {
        bcur = bnext;
      }
      const int jn = 32 * (k + 1) + lane;
      bnext = (p > 0 && jn < n) ? src[jn] : top;
      const bool last_pass = (p == npass - 1);
      const int t0 = 32 * k;
      const int tend = min(t0 + 32, n + 31);
#pragma unroll 4
      for (int t = t0; t < tend; t++) {
        int in_h = __shfl_up_sync(FULL, out_h, 1);
        int in_f = __shfl_up_sync(FULL, out_f, 1);
        const int bh = __shfl_sync(FULL, bcur.x, t - t0);
        const int bf = __shfl_sync(FULL, bcur.y, t - t0);
        if (lane == 0) {
          in_h = bh;
          in_f = bf;
        }
        const int j = t - lane;
        if (j >= 0 && j < n) {
          intra_cells<TI>(Hp, E, hdiag, out_h, out_f, S, in_h, in_f,
                          slice + (d[j] * 32 + lane) * TI, go, ge);
          if (lane == 31 && !last_pass) own[j] = make_int2(out_h, out_f);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) S = max(S, __shfl_xor_sync(FULL, S, o));
  if (lane == 0) red[wib] = S;
  __syncthreads();
  if (threadIdx.x == 0) {
    int best = 0;
    for (int w = 0; w < W; w++) best = max(best, red[w]);
    emit_score(db, P, q, s, best);
  }
}

template <int TI>
__global__ void __launch_bounds__(INTRA_WARPS * 32)
intra_kernel(DbView db, const SearchParams* __restrict__ P, SearchState* st, Scratch scr) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ unsigned long long s_item;
  __shared__ int red[INTRA_WARPS];
  int8_t* sm = (int8_t*)smem;
  load_matrix(sm, P);
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint8_t* slice = smem + MATRIX_SMEM + wib * IntraSlice<TI>::BYTES;
  const int64_t warp0 = (int64_t)blockIdx.x * INTRA_WARPS;
  int2* border = scr.intra_border + warp0 * scr.intra_stride;
  const int nq = P->nq;
  if (nq <= 0) return;  // uniform over the grid
  // int32 intra-task items, one warp each (longest subjects first)
  const int64_t n_items = P->n_intra_items;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(&st->intra_work, 1ull);
    it = __shfl_sync(FULL, it, 0);
    if ((int64_t)it >= n_items) break;
    const int s = (int)((int64_t)it / nq);
    const int q = P->qorder[(int64_t)it % nq];
    intra_warp_item<TI>(db, P, sm, slice, lane, border + wib * scr.intra_stride, q, s);
  }
  __syncthreads();
  // flagged pairs, one block each
  const unsigned long long nf = *(volatile unsigned long long*)&st->n_flags;
  const unsigned long long total =
      nf < (unsigned long long)scr.flag_capacity ? nf : (unsigned long long)scr.flag_capacity;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(&st->recompute, 1ull);
    __syncthreads();
    const unsigned long long it = s_item;
    __syncthreads();  // every thread has read s_item before thread 0 rewrites it
    if (it >= total) break;
    const int2 fl = scr.flags[it];
    intra_block_item<TI>(db, P, sm, slice, lane, wib, border, scr.intra_stride, red, fl.x, fl.y);
  }
}

// Pairs marked FLAG_SENTINEL by a packed kernel whose flag list was full:
// each (query, sorted subject) slot is read once, grid-stride, and every
// marked pair is counted and, while there is room, listed.
__global__ void collect_kernel(DbView db, const SearchParams* __restrict__ P, SearchState* st,
                               Scratch scr) {
  const int64_t slots = (int64_t)db.groups * GROUP;
  const int64_t total = (int64_t)P->nq * slots;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(i / slots);
    const int s = (int)(i - (int64_t)q * slots);
    const int orig = db.perm[s];
    if (orig < 0 || P->scores[(int64_t)q * db.n + orig] != FLAG_SENTINEL) continue;
    const unsigned long long k = atomicAdd(&st->n_flags, 1ull);
    if ((int64_t)k < scr.flag_capacity) scr.flags[k] = make_int2(q, s);
  }
}

cudaError_t launch_collect(int blocks, const DbView& db, const SearchParams* params,
                           SearchState* state, const Scratch& scr, cudaStream_t stream) {
  cudaGetLastError();  // a stale error must not be read as this launch's
  collect_kernel<<<blocks, 256, 0, stream>>>(db, params, state, scr);
  return cudaGetLastError();
}

typedef void (*IntraKernel)(DbView, const SearchParams*, SearchState*, Scratch);

static IntraKernel pick_intra(int rows) {
  if (rows == 8) return intra_kernel<8>;
  if (rows == 16) return intra_kernel<16>;
  return nullptr;
}

size_t intra_smem_bytes(int rows) {
  const int slice = rows == 8 ? IntraSlice<8>::BYTES : IntraSlice<16>::BYTES;
  return (size_t)MATRIX_SMEM + (size_t)INTRA_WARPS * slice;
}

int intra_blocks_per_sm(int rows) {
  IntraKernel k = pick_intra(rows);
  if (!k) return 0;
  const size_t smem = intra_smem_bytes(rows);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, INTRA_WARPS * 32, smem) !=
      cudaSuccess)
    return 0;
  return nb;
}

cudaError_t launch_intra(const KernelConfig& kc, const DbView& db, const SearchParams* params,
                         SearchState* state, const Scratch& scr, cudaStream_t stream) {
  IntraKernel k = pick_intra(kc.variant);
  if (!k) return cudaErrorInvalidValue;
  cudaGetLastError();  // a stale error must not be read as this launch's
  k<<<kc.blocks, INTRA_WARPS * 32, kc.smem, stream>>>(db, params, state, scr);
  return cudaGetLastError();
}

}  // namespace swgb
