// device_common.cuh -- device helpers shared by the alignment kernels of
// libswgb: inter_kernel.cu, intra_kernel.cu, pair_kernel.cu, plain_kernel.cu.
//
// Every kernel computes Eq. 1-3 of arxiv 2309.09609 (Section II-B) in the
// shared-gap form
//
//   h = max(hdiag + SM(q_i, d_j), E(i,j), F(i,j), 0)          (Eq. 1)
//   t = h - Go
//   E(i,j+1) = max(E(i,j) - Ge, t)                             (Eq. 2, next column)
//   F(i+1,j) = max(F(i,j) - Ge, t)                             (Eq. 3, next row)
//   S = max(S, h)
//
// which reorders Algorithm 1 so that H - Go is computed once per cell and E
// and F are produced one step ahead (the paper's future work, Section VI,
// names instruction reordering and narrower integers; the packed kernels do
// both).
//
// Threads wait on one another only at __syncwarp / __syncthreads; the only
// interaction between blocks is an atomic work counter, so nothing can spin.
#pragma once

#include <stdint.h>

#include "swgb_internal.h"

namespace swgb {

constexpr unsigned FULL = 0xffffffffu;
constexpr int MATRIX_SMEM = 640;  // 25 x 25 int8, rounded up to 16 bytes

__device__ __forceinline__ uint32_t pack2(int v) {
  return ((uint32_t)(uint16_t)(int16_t)v) * 0x00010001u;
}

// prmt with sign replication: result = (sext(a.byte k), sext(b.byte k)) as s16x2
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
  return r;
}
// selector for byte k: nibbles (low to high) k, 8|k, 4+k, 8|(4+k)
__device__ __forceinline__ constexpr uint32_t sext_pair_sel(int k) {
  return (uint32_t)(k | ((8 | k) << 4) | ((4 + k) << 8) | ((12 + k) << 12));
}
// int8 byte k of w, sign-extended to int32
__device__ __forceinline__ int sext_byte(uint32_t w, int k) {
  return (int)prmt(w, 0u, (uint32_t)(k | ((8 | k) << 4) | ((8 | k) << 8) | ((8 | k) << 12)));
}

__device__ __forceinline__ uint4 ldg_nc(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// 16-byte asynchronous global -> shared copy (L2 only), and its group fences.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---- score output ------------------------------------------------------------
__device__ __forceinline__ void emit_score(const DbView& db, const SearchParams* __restrict__ P,
                                           int q, int s, int score) {
  const int orig = db.perm[s];
  if (orig >= 0) P->scores[(int64_t)q * db.n + orig] = score;
}

// SM into shared memory (every thread of the block takes part; the caller syncs)
__device__ __forceinline__ void load_matrix(int8_t* sm, const SearchParams* __restrict__ P) {
  for (int i = threadIdx.x; i < NCODES * NCODES; i += blockDim.x) sm[i] = P->sm[i];
}

// int8 profile of one lane's R query rows [i0, i0 + R) of a pass, for every
// code c: byte r of the R-byte row at prof + (c * 32 + lane) * R is
// SM(q[i0 + r], c), and PAD_SCORE past the end of the query.
template <int R>
__device__ __forceinline__ void lane_profile(uint8_t* prof, const int8_t* __restrict__ sm,
                                             const uint8_t* __restrict__ qr, int m, int i0,
                                             int lane) {
  static_assert(R % 8 == 0, "rows per lane must be a multiple of 8");
  int qc[R];
#pragma unroll
  for (int r = 0; r < R; r++) qc[r] = (i0 + r < m) ? (int)qr[i0 + r] : -1;
  for (int c = 0; c < NCODES; c++) {
    uint32_t wv[R / 4];
#pragma unroll
    for (int w = 0; w < R / 4; w++) {
      uint32_t acc = 0;
#pragma unroll
      for (int b = 0; b < 4; b++) {
        const int r = w * 4 + b;
        const int v = qc[r] >= 0 ? (int)sm[qc[r] * NCODES + c] : PAD_SCORE;
        acc |= ((uint32_t)(uint8_t)(int8_t)v) << (8 * b);
      }
      wv[w] = acc;
    }
    uint8_t* dst = prof + (c * 32 + lane) * R;
    if constexpr (R % 16 == 0) {
#pragma unroll
      for (int w = 0; w < R / 4; w += 4)
        *(uint4*)(dst + 4 * w) = make_uint4(wv[w], wv[w + 1], wv[w + 2], wv[w + 3]);
    } else {
#pragma unroll
      for (int w = 0; w < R / 4; w += 2) *(uint2*)(dst + 4 * w) = make_uint2(wv[w], wv[w + 1]);
    }
  }
}

// ---- packed 16-bit cells (two subjects per 32-bit word) ---------------------
//
// Values are held with a bias of +Go: X' = X + Go for H, E, F and S.  Then
//   * the zero term of Eq. 1 becomes a max with the constant Go, folded into
//     the three-input max of E' and F';
//   * every H' is >= Go in each 16-bit half, so t' = H' - Go never borrows
//     across halves and is one 32-bit integer multiply-add (FMA pipe);
//   * E' - Ge >= -Ge and H' <= 32767 as long as H <= 32767 - Go: nothing
//     wraps before a score reaches the recompute threshold.
// A pair is recomputed in int32 when S' >= 32767 - max(SM): the first cell
// whose H' could exceed 32767 has exact inputs, so it is recorded in S'.
__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}

// The packed words of the gap penalties: GO2 = (Go, Go) (H' of H = 0),
// NGE2 = (-Ge, -Ge) and MGO = -(Go, Go) as one 32-bit word.  Gap class G > 0
// fixes them at compile time for a common setting, so they enter the
// instructions as immediates instead of registers (on the paper-shaped search
// the two-query kernel ran 6% faster so); G = 0 reads them from the
// parameter block.  The classes are listed in swgb_internal.h (gap_class).
template <int G>
__device__ __forceinline__ void gap_words(const SearchParams* __restrict__ P, uint32_t& GO2,
                                          uint32_t& NGE2, uint32_t& MGO) {
  if constexpr (G == 0) {
    const int go = P->go;
    GO2 = pack2(go);
    NGE2 = pack2(-P->ge);
    MGO = (uint32_t)(-(int)((uint32_t)go * 65537u));
  } else {
    constexpr int go = GapClass<G>::GO, ge = GapClass<G>::GE;
    GO2 = ((uint32_t)(uint16_t)go) * 0x00010001u;
    NGE2 = ((uint32_t)(uint16_t)(int16_t)(-ge)) * 0x00010001u;
    MGO = (uint32_t)(-(int)((uint32_t)go * 65537u));
  }
}

// One packed cell update (Eq. 1-3, biased by +Go): returns H'; updates E' of
// the next column in e and F' of the next row in f.  H' - Go goes to the FMA
// pipe either way: with compile-time penalties (G > 0) as a 16x2 subtract of
// the immediate (Go, Go), otherwise as one 32-bit IMAD by the run-time
// register `one` (no borrow crosses the halves, since H' >= Go in each).  On
// the paper-shaped search the subtract took the two-query kernel from 826 to
// 801 ms with compile-time penalties, and from 881 to 898 ms with run-time
// ones.
template <int G>
__device__ __forceinline__ uint32_t packed_cell(uint32_t hd, uint32_t w, uint32_t& e, uint32_t& f,
                                                uint32_t GO2, uint32_t NGE2, uint32_t MGO,
                                                uint32_t one) {
  const uint32_t h = __viaddmax_s16x2(hd, w, __vimax3_s16x2(e, f, GO2));  // H'
  uint32_t t;                                                              // H' - Go
  if constexpr (G > 0)
    t = __vsub2(h, GO2);
  else
    t = imad(h, one, MGO);
  e = __viaddmax_s16x2(e, NGE2, t);  // E' of the next column
  f = __viaddmax_s16x2(f, NGE2, t);  // F' of the next row
  return h;
}

}  // namespace swgb
