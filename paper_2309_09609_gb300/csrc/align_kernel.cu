// align_kernel.cu -- optimal local alignments with traceback (sw_align).
//
// The score kernels return S only.  For selected pairs this file also
// recovers the alignment behind S, by the traceback of Section II-B:
//
//   * align_forward: one warp per pair runs the int32 warp wavefront of
//     Eq. 1-3 (lane k owns AT query rows of a 32*AT-row pass, (H, F) borders
//     by __shfl_up_sync, pass borders in scratch) and stores four bits per
//     cell -- where H came from, and whether E of the next column and F of
//     the next row open a gap here -- plus the cell holding S;
//   * align_traceback: one thread per pair walks those bits back from that
//     cell and writes the transcript.
//
// Which of several optimal alignments is returned:
//   1. it ends at the first cell (i, j) in row-major order whose H equals S;
//   2. walking back in state H: the diagonal term first, then E, then F,
//      whichever equals H;
//   3. in a gap state the gap opens from H when that reaches the gap's
//      value, else it extends;
//   4. the walk ends with the diagonal step into a cell whose H is 0.
// Transcript, first column to last: 'M' (query and subject residue), 'I'
// (query residue against a gap), 'D' (subject residue against a gap).
#include <algorithm>

#include "device_common.cuh"

namespace swgb {

constexpr int AT = 8;            // query rows per lane
constexpr int AROWS = 32 * AT;   // rows per pass
constexpr int ALIGN_WARPS = 4;   // warps per block

// Cell nibble: bits 0-1 the source of H (0: H is 0, 1: diagonal, 2: E,
// 3: F); bit 2: E of the next column opens here; bit 3: F of the next row
// opens here.  Word (pass p, step t, lane k) holds the nibbles of the lane's
// AT rows at column t - k, row r of the lane in bits 4r..4r+3.
__device__ __forceinline__ int64_t bits_word(int64_t base, int n, int p, int t, int lane) {
  return base + ((int64_t)p * (n + 31) + t) * 32 + lane;
}

__device__ __forceinline__ bool end_before(int v, int i, int j, int bv, int bi, int bj) {
  return v > bv || (v == bv && (i < bi || (i == bi && j < bj)));
}

__global__ void __launch_bounds__(ALIGN_WARPS * 32)
align_forward(DbView db, const SearchParams* __restrict__ P, const AlignItem* __restrict__ items,
              int n_items, uint32_t* __restrict__ bits, int2* __restrict__ border,
              AlignOut* __restrict__ out) {
  __shared__ __align__(16) uint8_t prof_all[ALIGN_WARPS][NCODES * 32 * AT];
  __shared__ int8_t sm[NCODES * NCODES];
  load_matrix(sm, P);
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint8_t* prof = prof_all[wib];
  const int go = P->go, ge = P->ge;
  const int warps = gridDim.x * ALIGN_WARPS;
  for (int k = blockIdx.x * ALIGN_WARPS + wib; k < n_items; k += warps) {
    const AlignItem it = items[k];
    const int m = P->qlen[it.q];
    const int n = db.clen[it.s];
    const uint8_t* __restrict__ qr = P->qres + P->qoff[it.q];
    const uint8_t* __restrict__ d = db.cont + db.coff[it.s];
    int2* hb = border + it.border_off;
    const int npass = n > 0 ? (m + AROWS - 1) / AROWS : 0;
    // this lane's best cell so far: (H, 1-based row, 1-based column)
    int bv = 0, bi = INT32_MAX, bj = INT32_MAX;
    for (int p = 0; p < npass; p++) {
      __syncwarp();
      lane_profile<AT>(prof, sm, qr, m, p * AROWS + lane * AT, lane);
      __syncwarp();
      int Hp[AT], E[AT];
#pragma unroll
      for (int r = 0; r < AT; r++) {
        Hp[r] = 0;    // H(i, 0)
        E[r] = -go;   // E(i, 1)
      }
      int hdiag = 0, out_h = 0, out_f = -go;
      const bool last_pass = (p == npass - 1);
      const int row0 = p * AROWS + lane * AT;  // 0-based row of this lane's first row
      for (int t = 0; t < n + 31; t++) {
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
          const uint2 pv = *(const uint2*)(prof + ((int)d[j] * 32 + lane) * AT);
          int hd = hdiag;
          hdiag = in_h;
          int f = in_f;
          uint32_t word = 0;
#pragma unroll
          for (int r = 0; r < AT; r++) {
            const int w = sext_byte(r < 4 ? pv.x : pv.y, r & 3);
            const int e = E[r];
            const int diag = hd + w;
            const int h = max(max(diag, e), max(f, 0));                  // Eq. 1
            const uint32_t src = h == 0 ? 0u : h == diag ? 1u : h == e ? 2u : 3u;
            hd = Hp[r];
            Hp[r] = h;
            const int t_open = h - go, e_ext = e - ge, f_ext = f - ge;
            E[r] = max(e_ext, t_open);                                   // Eq. 2, next column
            f = max(f_ext, t_open);                                      // Eq. 3, next row
            word |= (src | (t_open >= e_ext ? 4u : 0u) | (t_open >= f_ext ? 8u : 0u)) << (4 * r);
            const int row = row0 + r;
            if (h > 0 && row < m && end_before(h, row + 1, j + 1, bv, bi, bj)) {
              bv = h;
              bi = row + 1;
              bj = j + 1;
            }
          }
          out_h = Hp[AT - 1];
          out_f = f;
          bits[bits_word(it.bits_off, n, p, t, lane)] = word;
          if (lane == 31 && !last_pass) hb[j] = make_int2(out_h, out_f);
        }
      }
    }
    // the first cell in row-major order holding the largest H
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int v2 = __shfl_xor_sync(FULL, bv, o);
      const int i2 = __shfl_xor_sync(FULL, bi, o);
      const int j2 = __shfl_xor_sync(FULL, bj, o);
      if (end_before(v2, i2, j2, bv, bi, bj)) {
        bv = v2;
        bi = i2;
        bj = j2;
      }
    }
    if (lane == 0) {
      AlignOut r{};
      r.score = bv;
      r.i_end = bv > 0 ? bi : 0;
      r.j_end = bv > 0 ? bj : 0;
      out[k] = r;
    }
  }
}

// The same forward pass with a whole block per pair, for few long pairs:
// the 16 warps take the query's passes round-robin on the stage schedule of
// the int32 recompute (pass p starts LAG stages of 32 steps after pass p - 1,
// every stage ends at __syncthreads, each warp writes the bottom rows of its
// passes to its own scratch row and reads those of the pass before).  Cells,
// bits and the end cell are exactly those of align_forward.
constexpr int ABW = 16;   // warps per block
constexpr int ALAG = 3;   // stages between the starts of consecutive passes

__global__ void __launch_bounds__(ABW * 32)
align_forward_block(DbView db, const SearchParams* __restrict__ P,
                    const AlignItem* __restrict__ items, int n_items, uint32_t* __restrict__ bits,
                    int2* __restrict__ border, AlignOut* __restrict__ out) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int red_v[ABW], red_i[ABW], red_j[ABW];
  int8_t* sm = (int8_t*)smem;
  load_matrix(sm, P);
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint8_t* prof = smem + MATRIX_SMEM + wib * (NCODES * 32 * AT);
  const int go = P->go, ge = P->ge;
  for (int k = blockIdx.x; k < n_items; k += gridDim.x) {  // uniform over the block
    const AlignItem it = items[k];
    const int m = P->qlen[it.q];
    const int n = db.clen[it.s];
    const uint8_t* __restrict__ qr = P->qres + P->qoff[it.q];
    const uint8_t* __restrict__ d = db.cont + db.coff[it.s];
    int2* own = border + it.border_off + (int64_t)wib * n;               // this warp's rows
    const int2* src = border + it.border_off + (int64_t)((wib + ABW - 1) % ABW) * n;
    const int npass = n > 0 ? (m + AROWS - 1) / AROWS : 0;
    const int spass = (n + 31 + 31) / 32;
    const int period = max(spass, ALAG * ABW);
    const int nstages =
        npass > 0 ? ((npass - 1) / ABW) * period + ((npass - 1) % ABW) * ALAG + spass : 0;
    const int2 top = make_int2(0, -go);
    int bv = 0, bi = INT32_MAX, bj = INT32_MAX;
    int Hp[AT], E[AT], hdiag = 0, out_h = 0, out_f = -go;
    int p = 0;
    int2 bcur = top, bnext = top;
    for (int g = 0; g < nstages; g++) {
      const int rel = g - wib * ALAG;
      int ks = -1;
      if (rel >= 0) {
        const int r = rel / period;
        const int kk = rel - r * period;
        if (kk < spass && wib + r * ABW < npass) {
          ks = kk;
          p = wib + r * ABW;
        }
      }
      if (ks >= 0) {  // warp-uniform
        if (ks == 0) {
          __syncwarp();
          lane_profile<AT>(prof, sm, qr, m, p * AROWS + lane * AT, lane);
          __syncwarp();
#pragma unroll
          for (int r = 0; r < AT; r++) {
            Hp[r] = 0;
            E[r] = -go;
          }
          hdiag = 0;
          out_h = 0;
          out_f = -go;
          bcur = (p > 0 && lane < n) ? src[lane] : top;
        } else {
          bcur = bnext;
        }
        const int jn = 32 * (ks + 1) + lane;
        bnext = (p > 0 && jn < n) ? src[jn] : top;
        const bool last_pass = (p == npass - 1);
        const int row0 = p * AROWS + lane * AT;
        const int t0 = 32 * ks;
        const int tend = min(t0 + 32, n + 31);
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
            const uint2 pv = *(const uint2*)(prof + ((int)d[j] * 32 + lane) * AT);
            int hd = hdiag;
            hdiag = in_h;
            int f = in_f;
            uint32_t word = 0;
#pragma unroll
            for (int r = 0; r < AT; r++) {
              const int w = sext_byte(r < 4 ? pv.x : pv.y, r & 3);
              const int e = E[r];
              const int diag = hd + w;
              const int h = max(max(diag, e), max(f, 0));                // Eq. 1
              const uint32_t srcc = h == 0 ? 0u : h == diag ? 1u : h == e ? 2u : 3u;
              hd = Hp[r];
              Hp[r] = h;
              const int t_open = h - go, e_ext = e - ge, f_ext = f - ge;
              E[r] = max(e_ext, t_open);                                 // Eq. 2
              f = max(f_ext, t_open);                                    // Eq. 3
              word |= (srcc | (t_open >= e_ext ? 4u : 0u) | (t_open >= f_ext ? 8u : 0u)) << (4 * r);
              const int row = row0 + r;
              if (h > 0 && row < m && end_before(h, row + 1, j + 1, bv, bi, bj)) {
                bv = h;
                bi = row + 1;
                bj = j + 1;
              }
            }
            out_h = Hp[AT - 1];
            out_f = f;
            bits[bits_word(it.bits_off, n, p, t, lane)] = word;
            if (lane == 31 && !last_pass) own[j] = make_int2(out_h, out_f);
          }
        }
      }
      __syncthreads();
    }
    // the first cell in row-major order holding the largest H, over the block
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int v2 = __shfl_xor_sync(FULL, bv, o);
      const int i2 = __shfl_xor_sync(FULL, bi, o);
      const int j2 = __shfl_xor_sync(FULL, bj, o);
      if (end_before(v2, i2, j2, bv, bi, bj)) {
        bv = v2;
        bi = i2;
        bj = j2;
      }
    }
    if (lane == 0) {
      red_v[wib] = bv;
      red_i[wib] = bi;
      red_j[wib] = bj;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < ABW; w++)
        if (end_before(red_v[w], red_i[w], red_j[w], bv, bi, bj)) {
          bv = red_v[w];
          bi = red_i[w];
          bj = red_j[w];
        }
      AlignOut r{};
      r.score = bv;
      r.i_end = bv > 0 ? bi : 0;
      r.j_end = bv > 0 ? bj : 0;
      out[k] = r;
    }
    __syncthreads();  // red_* are rewritten by the next pair
  }
}

__global__ void __launch_bounds__(128)
align_traceback(DbView db, const SearchParams* __restrict__ P, const AlignItem* __restrict__ items,
                int n_items, const uint32_t* __restrict__ bits, AlignOut* __restrict__ out,
                uint8_t* __restrict__ ops) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_items) return;
  const AlignItem it = items[k];
  AlignOut r = out[k];
  const int m = P->qlen[it.q];
  const int n = db.clen[it.s];
  int64_t pos = it.ops_end;  // the transcript is written backwards, ending here
  r.q_begin = r.s_begin = 0;
  if (r.score > 0) {
    auto nib = [&](int i, int j) -> uint32_t {  // 1-based cell
      const int row = i - 1, lane = (row % AROWS) / AT;
      const uint32_t w = bits[bits_word(it.bits_off, n, row / AROWS, j - 1 + lane, lane)];
      return (w >> (4 * (row % AT))) & 15u;
    };
    int i = r.i_end, j = r.j_end, state = 0;  // 0: H, 1: E, 2: F
    // at most m + n columns, each gap run entered by one more step from
    // state H: the bound only guards against a broken bit matrix
    for (int64_t guard = 0; guard < 2 * ((int64_t)m + n) + 2; guard++) {
      if (state == 0) {
        const uint32_t src = nib(i, j) & 3u;
        if (src == 1u) {
          ops[--pos] = 'M';
          i--;
          j--;
          if (i == 0 || j == 0 || (nib(i, j) & 3u) == 0u) break;
        } else {
          state = src == 2u ? 1 : 2;
        }
      } else if (state == 1) {
        ops[--pos] = 'D';
        state = (nib(i, j - 1) & 4u) ? 0 : 1;
        j--;
      } else {
        ops[--pos] = 'I';
        state = (nib(i - 1, j) & 8u) ? 0 : 2;
        i--;
      }
    }
    r.q_begin = i;
    r.s_begin = j;
  }
  r.n_ops = (int32_t)(it.ops_end - pos);
  r.ops_offset = pos;
  out[k] = r;
}

cudaError_t launch_align(const DbView& db, const SearchParams* params, const AlignItem* items,
                         int n_items, bool block_mode, uint32_t* bits, int2* border, AlignOut* out,
                         uint8_t* ops, cudaStream_t stream) {
  if (n_items <= 0) return cudaSuccess;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (block_mode) {
    const size_t smem = (size_t)MATRIX_SMEM + (size_t)ABW * NCODES * 32 * AT;
    e = cudaFuncSetAttribute(align_forward_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    cudaGetLastError();  // a stale error must not be read as this launch's
    align_forward_block<<<std::min(n_items, std::max(sms, 1)), ABW * 32, smem, stream>>>(
        db, params, items, n_items, bits, border, out);
  } else {
    const int blocks = std::min((n_items + ALIGN_WARPS - 1) / ALIGN_WARPS, std::max(sms, 1) * 8);
    cudaGetLastError();  // a stale error must not be read as this launch's
    align_forward<<<blocks, ALIGN_WARPS * 32, 0, stream>>>(db, params, items, n_items, bits,
                                                           border, out);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cudaGetLastError();  // a stale error must not be read as this launch's
  align_traceback<<<(n_items + 127) / 128, 128, 0, stream>>>(db, params, items, n_items, bits, out,
                                                             ops);
  return cudaGetLastError();
}

int64_t align_bits_words(int32_t m, int32_t n) {
  if (m <= 0 || n <= 0) return 0;
  return (int64_t)((m + AROWS - 1) / AROWS) * (n + 31) * 32;
}

}  // namespace swgb
