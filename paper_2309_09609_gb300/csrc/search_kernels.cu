// search_kernels.cu -- the alignment kernels of libswgb.
//
// All kernels compute Eq. 1-3 of arxiv 2309.09609 (Section II-B) in the
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
// names instruction reordering and narrower integers; this is both).
//
// Kernels:
//   * search_kernel<T, TI>, mode 0 -- one persistent launch over work items
//     taken longest-first from an atomic counter:
//       - intra-task items (query, long subject): one warp per pair; lane k
//         owns TI query rows of a 32*TI-row pass and sweeps the subject one
//         step behind lane k-1, which hands it the (H, F) border of its last
//         row through __shfl_up_sync (Section II-B: intra-task parallelism
//         with neighbour border exchange).  int32 cells.
//       - inter-task items (query, group of 64 short subjects): each lane owns
//         two subjects, packed as the two 16-bit halves of every 32-bit word,
//         and T query rows held in registers (Section II-B: inter-task
//         parallelism, one matrix per processing element).  A pair whose
//         16-bit score reaches 32767 - max(SM) is appended to a flag list.
//   * search_kernel<T, TI>, mode 1 -- recomputes every flagged pair with the
//     int32 intra-task code, so every score is exact.
//   * plain_kernel -- the baseline: Algorithm 1 verbatim in int32, one thread
//     per subject, one launch per query.
//
// No kernel waits on another thread, block or kernel: the only cross-warp
// interaction is the atomic work counter, so nothing here can spin.
#include <stdio.h>

#include <type_traits>

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

// ---- shared-memory profile slices ------------------------------------------
// Inter-task (packed) strip profile for T query rows, int8, replicated 8x so
// that the 8 lanes of a quarter-warp read 16-byte rows of any residue codes
// from 8 distinct bank groups (no bank conflicts for random residues):
//   byte (c, half h, copy p, row r) at ((c * (T/16) + h) * 8 + p) * 16 + (r - 16h)
// After the profile, the inter-task slice holds the cp.async staging ring of
// CRING 8-column chunks: per chunk, the 4 border vectors (one per column pair)
// and the residue vector of every lane.
constexpr int CRING = 3;  // chunks in flight per warp
template <int T>
struct InterProfile {
  static constexpr int PROFILE = NCODES * 8 * T;
  static constexpr int BORDER_RING = PROFILE;                     // CRING x 4 x 32 x 16 bytes
  static constexpr int RES_RING = BORDER_RING + CRING * 4 * 512;  // CRING x 32 x 16 bytes
  static constexpr int BYTES = RES_RING + CRING * 512;
};
// Intra-task pass profile, int8: lane k's TI rows for code c at (c * 32 + k) * TI.
template <int TI>
struct IntraProfile {
  static constexpr int BYTES = NCODES * 32 * TI;
};

template <int T, int TI>
struct SliceBytes {
  static constexpr int A = InterProfile<T>::BYTES, B = IntraProfile<TI>::BYTES;
  static constexpr int BYTES = ((A > B ? A : B) + 15) / 16 * 16;
};

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

// ---- intra-task warp wavefront, int32 (Section II-B, intra-task) -----------
template <int TI>
__device__ void intra_item(const DbView& db, const SearchParams* __restrict__ P,
                           const int8_t* __restrict__ sm, uint8_t* slice, int lane,
                           int64_t warp_id, const Scratch& scr, int q, int s) {
  const int n = db.clen[s];
  const int m = P->qlen[q];
  const uint8_t* __restrict__ d = db.cont + db.coff[s];
  const uint8_t* __restrict__ qr = P->qres + P->qoff[q];
  int2* hb = scr.intra_border + warp_id * scr.intra_stride;
  const int go = P->go, ge = P->ge;
  constexpr int ROWS = 32 * TI;
  const int npass = (m + ROWS - 1) / ROWS;
  int S = 0;
  for (int p = 0; p < npass && n > 0; p++) {
    __syncwarp();
    // profile: this lane's TI rows for every code
    {
      const int i0 = p * ROWS + lane * TI;
      int qc[TI];
#pragma unroll
      for (int r = 0; r < TI; r++) qc[r] = (i0 + r < m) ? (int)qr[i0 + r] : -1;
      for (int c = 0; c < NCODES; c++) {
        uint32_t wv[TI / 4];
#pragma unroll
        for (int w = 0; w < TI / 4; w++) {
          uint32_t acc = 0;
#pragma unroll
          for (int b = 0; b < 4; b++) {
            const int r = w * 4 + b;
            const int v = qc[r] >= 0 ? (int)sm[qc[r] * NCODES + c] : PAD_SCORE;
            acc |= ((uint32_t)(uint8_t)(int8_t)v) << (8 * b);
          }
          wv[w] = acc;
        }
        uint32_t* dst = (uint32_t*)(slice + (c * 32 + lane) * TI);
#pragma unroll
        for (int w = 0; w < TI / 4; w++) dst[w] = wv[w];
      }
    }
    __syncwarp();
    int Hp[TI], E[TI];
#pragma unroll
    for (int r = 0; r < TI; r++) {
      Hp[r] = 0;    // H(i, 0)
      E[r] = -go;   // E(i, 1)
    }
    int hdiag = 0, out_h = 0, out_f = -go;
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
          in_h = 0;     // H(0, j)
          in_f = -go;   // F(1, j)
        }
      }
      if (j >= 0 && j < n) {
        const int c = d[j];
        uint32_t pw[TI / 4];
        if constexpr (TI == 8) {
          const uint2 v = *(const uint2*)(slice + (c * 32 + lane) * TI);
          pw[0] = v.x;
          pw[1] = v.y;
        } else {
          const uint4 v = *(const uint4*)(slice + (c * 32 + lane) * TI);
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
          const int h = __viaddmax_s32_relu(hd, w, max(e, f));
          hd = Hp[r];
          Hp[r] = h;
          const int tt = h - go;
          E[r] = __viaddmax_s32(e, -ge, tt);
          f = __viaddmax_s32(f, -ge, tt);
          S = max(S, h);
        }
        out_h = Hp[TI - 1];
        out_f = f;
        if (lane == 31 && !last_pass) hb[j] = make_int2(out_h, out_f);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) S = max(S, __shfl_xor_sync(FULL, S, o));
  if (lane == 0) emit_score(db, P, q, s, S);
}

// ---- inter-task, packed 16-bit pairs (Section II-B, inter-task) ------------
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

// Profile word of row r for this lane's two subjects: (SM(q_r, a_j), SM(q_r, b_j)).
template <int T>
__device__ __forceinline__ uint32_t profile_word(const uint4 (&va)[T / 16], const uint4 (&vb)[T / 16],
                                                 int r) {
  const uint4& A = va[r / 16];
  const uint4& B = vb[r / 16];
  const int wq = (r / 4) & 3;
  const uint32_t a32 = wq == 0 ? A.x : wq == 1 ? A.y : wq == 2 ? A.z : A.w;
  const uint32_t b32 = wq == 0 ? B.x : wq == 1 ? B.y : wq == 2 ? B.z : B.w;
  return prmt(a32, b32, sext_pair_sel(r & 3));
}

// One packed cell update (Eq. 1-3, biased by +Go): returns H'; updates E' of
// the next column in e and F' of the next row in f.
__device__ __forceinline__ uint32_t packed_cell(uint32_t hd, uint32_t w, uint32_t& e, uint32_t& f,
                                                uint32_t GO2, uint32_t NGE2, uint32_t MGO,
                                                uint32_t one) {
  const uint32_t h = __viaddmax_s16x2(hd, w, __vimax3_s16x2(e, f, GO2));  // H'
  const uint32_t t = imad(h, one, MGO);  // H' - Go in both halves (FMA pipe)
  e = __viaddmax_s16x2(e, NGE2, t);      // E' of the next column
  f = __viaddmax_s16x2(f, NGE2, t);      // F' of the next row
  return h;
}

// Four adjacent columns of T rows as a wavefront: at step k, column c
// updates row k - c.  Column c's row r needs E' of column c - 1 at row r
// (written one step earlier) and its H' at row r - 1 (two steps earlier), so
// the up to four updates of a step are independent.  Hp[r] / E[r] hold H' / E'
// of the previous column on entry and of the fourth column on exit; b0, b1
// are the border vectors (H'_c, F'_c) above the strip for columns 0,1 and 2,3;
// o0, o1 receive the strip's bottom row in the same layout.
template <int T>
__device__ __forceinline__ void packed_quad(uint32_t (&Hp)[T], uint32_t (&E)[T], uint32_t& hdiag,
                                            uint32_t& smax, const uint8_t* slice, int p16,
                                            uint32_t wa, uint32_t wb, const uint4& b0,
                                            const uint4& b1, uint4& o0, uint4& o1, uint32_t GO2,
                                            uint32_t NGE2, uint32_t MGO, uint32_t one) {
  constexpr int HALVES = T / 16;
  constexpr int W = 4;
  uint4 pa[W][HALVES], pb[W][HALVES];
#pragma unroll
  for (int c = 0; c < W; c++) {
    const uint32_t ca = (wa >> (8 * c)) & 0xffu;
    const uint32_t cb = (wb >> (8 * c)) & 0xffu;
#pragma unroll
    for (int h = 0; h < HALVES; h++) {
      pa[c][h] = *(const uint4*)(slice + (ca * HALVES + h) * 128 + p16);
      pb[c][h] = *(const uint4*)(slice + (cb * HALVES + h) * 128 + p16);
    }
  }
  const uint32_t htop[W] = {b0.x, b0.z, b1.x, b1.z};  // H' above the strip, per column
  uint32_t f[W] = {b0.y, b0.w, b1.y, b1.w};           // F' of the strip's first row
  uint32_t last[W] = {0, 0, 0, 0}, last2[W] = {0, 0, 0, 0}, bottom[W] = {0, 0, 0, 0};
  uint32_t hd0 = hdiag;  // column 0's diagonal: previous column, previous row
  hdiag = htop[W - 1];
#pragma unroll
  for (int k = 0; k < T + W - 1; k++) {
    uint32_t out[W] = {0, 0, 0, 0};
#pragma unroll
    for (int c = 0; c < W; c++) {
      const int r = k - c;
      if (r < 0 || r >= T) continue;
      uint32_t hd;
      if (c == 0) {
        hd = hd0;
        hd0 = Hp[r];
      } else {
        hd = r == 0 ? htop[c - 1] : last2[c - 1];  // H' of column c - 1, row r - 1
      }
      uint32_t e = E[r];
      out[c] = packed_cell(hd, profile_word<T>(pa[c], pb[c], r), e, f[c], GO2, NGE2, MGO, one);
      E[r] = e;
      if (c == W - 1) Hp[r] = out[c];
      if (r == T - 1) bottom[c] = out[c];
    }
    // S' over this step's cells (pairs through a three-input max)
    const int lo = k - (T - 1) > 0 ? k - (T - 1) : 0;
    const int hi = k < W - 1 ? k : W - 1;
    int c = lo;
    for (; c + 1 <= hi; c += 2) smax = __vimax3_s16x2(smax, out[c], out[c + 1]);
    if (c == hi) smax = __vmaxs2(smax, out[c]);
#pragma unroll
    for (int c2 = 0; c2 < W; c2++) {
      last2[c2] = last[c2];
      last[c2] = out[c2];
    }
  }
  o0 = make_uint4(bottom[0], f[0], bottom[1], f[1]);
  o1 = make_uint4(bottom[2], f[2], bottom[3], f[3]);
}

template <int T>
__device__ void inter_item(const DbView& db, const SearchParams* __restrict__ P, SearchState* st,
                           const int8_t* __restrict__ sm, uint8_t* slice, int lane,
                           int64_t warp_id, const Scratch& scr, int q, int g) {
  const int L = db.glen[g];  // multiple of CHUNK
  const int m = P->qlen[q];
  const uint8_t* __restrict__ qr = P->qres + P->qoff[q];
  const uint4* __restrict__ res = (const uint4*)(db.inter + db.goff[g]) + lane;
  uint4* bd = scr.inter_border + warp_id * scr.inter_stride_vec + lane;
  const int go = P->go;
  const uint32_t GO2 = pack2(go);                                  // H' of H = 0
  const uint32_t NGE2 = pack2(-P->ge);
  const uint32_t MGO = (uint32_t)(-(int)((uint32_t)go * 65537u));  // - (Go, Go) as one word
  const uint32_t ZERO2 = 0u;                                       // E' of E = -Go
  const uint32_t one = (uint32_t)P->one;
  const int p16 = (lane & 7) * 16;
  constexpr int HALVES = T / 16;
  const int nstrips = L > 0 ? (m + T - 1) / T : 0;
  const int nch = L / CHUNK;
  uint4* bring = (uint4*)(slice + InterProfile<T>::BORDER_RING) + lane;  // [slot][pair][lane]
  uint4* rring = (uint4*)(slice + InterProfile<T>::RES_RING) + lane;     // [slot][lane]
  uint32_t smax = GO2;  // S' of S = 0
  for (int s = 0; s < nstrips; s++) {
    __syncwarp();
    if (lane < NCODES) {  // code c = lane: T bytes, written to all 8 copies
      const int i0 = s * T;
      uint32_t wv[T / 4];
#pragma unroll
      for (int w = 0; w < T / 4; w++) {
        uint32_t acc = 0;
#pragma unroll
        for (int b = 0; b < 4; b++) {
          const int i = i0 + w * 4 + b;
          const int v = i < m ? (int)sm[(int)qr[i] * NCODES + lane] : PAD_SCORE;
          acc |= ((uint32_t)(uint8_t)(int8_t)v) << (8 * b);
        }
        wv[w] = acc;
      }
#pragma unroll
      for (int h = 0; h < HALVES; h++) {
        const uint4 v = make_uint4(wv[4 * h], wv[4 * h + 1], wv[4 * h + 2], wv[4 * h + 3]);
#pragma unroll
        for (int p = 0; p < 8; p++)
          *(uint4*)(slice + ((lane * HALVES + h) * 8 + p) * 16) = v;
      }
    }
    __syncwarp();
    uint32_t Hp[T], E[T];
#pragma unroll
    for (int r = 0; r < T; r++) {
      Hp[r] = GO2;    // H(i, 0) = 0
      E[r] = ZERO2;   // E(i, 1) = -Go
    }
    uint32_t hdiag = GO2;
    const bool last = (s == nstrips - 1);
    // Staging ring of CRING chunks, copied with cp.async CRING - 1 chunks ahead
    // (commit group c = chunk c).  The first strip's border is the row above
    // the matrix, (H, F) = (0, -Go) for every column: it is copied from the
    // parameter block, so the compute loop has no branch on it.  A slot is
    // refilled only after the registers read from it were consumed.
    const uint4* bsrc = s == 0 ? (const uint4*)&P->init_border : bd;
    const int bstep = s == 0 ? 0 : 32;
#pragma unroll
    for (int j = 0; j < CRING - 1; j++) {
      if (j < nch) {
#pragma unroll
        for (int k = 0; k < 4; k++)
          cp_async16(bring + ((j % CRING) * 4 + k) * 32, bsrc + (j * 4 + k) * bstep);
        cp_async16(rring + (j % CRING) * 32, res + j * 32);
      }
      cp_async_commit();
    }
#pragma unroll 1
    for (int c = 0; c < nch; c++) {
      const int cn = c + CRING - 1;
      if (cn < nch) {
        const int sl = cn % CRING;
#pragma unroll
        for (int k = 0; k < 4; k++)
          cp_async16(bring + (sl * 4 + k) * 32, bsrc + (cn * 4 + k) * bstep);
        cp_async16(rring + sl * 32, res + cn * 32);
      }
      cp_async_commit();
      cp_async_wait<CRING - 1>();  // chunk c has landed
      const int slot = c % CRING;
      const uint4 rr = rring[slot * 32];
      // two groups of 4 columns (one residue word per subject each); for
      // T = 16 both are unrolled so the second group's profile loads can be
      // issued during the first group's wavefront tail
      auto group = [&](int hq) {
        const uint32_t wa = hq ? rr.y : rr.x;
        const uint32_t wb = hq ? rr.w : rr.z;
        const uint4 b0 = bring[(slot * 4 + 2 * hq) * 32];
        const uint4 b1 = bring[(slot * 4 + 2 * hq + 1) * 32];
        uint4 o0, o1;
        packed_quad<T>(Hp, E, hdiag, smax, slice, p16, wa, wb, b0, b1, o0, o1, GO2, NGE2, MGO,
                       one);
        if (!last) {
          bd[(c * 4 + 2 * hq) * 32] = o0;
          bd[(c * 4 + 2 * hq + 1) * 32] = o1;
        }
      };
      if constexpr (T == 16) {
        group(0);
        group(1);
      } else {
#pragma unroll 1
        for (int hq = 0; hq < 2; hq++) group(hq);
      }
    }
    cp_async_wait<0>();
  }
  // two scores per lane; a possibly saturated one goes to the int32 recompute list
  const int base = g * GROUP + 2 * lane;
#pragma unroll
  for (int half = 0; half < 2; half++) {
    const int sidx = base + half;
    const int orig = db.perm[sidx];
    if (orig < 0) continue;
    const int sb = (int)(int16_t)(half ? (smax >> 16) : (smax & 0xffffu));  // S'
    if (sb >= P->sat_threshold) {
      const unsigned long long k = atomicAdd(&st->n_flags, 1ull);
      if ((int64_t)k < scr.flag_capacity) scr.flags[k] = make_int2(q, sidx);
    } else {
      P->scores[(int64_t)q * db.n + orig] = sb - go;
    }
  }
}

// ---- the persistent kernel ----------------------------------------------------
template <int T, int TI>
__global__ void __launch_bounds__(256, (T == 16 ? 2 : 1))
search_kernel(int mode, DbView db, const SearchParams* __restrict__ P, SearchState* st,
              Scratch scr) {
  extern __shared__ __align__(16) uint8_t smem[];
  int8_t* sm = (int8_t*)smem;
  for (int i = threadIdx.x; i < NCODES * NCODES; i += blockDim.x) sm[i] = P->sm[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint8_t* slice = smem + MATRIX_SMEM + wib * SliceBytes<T, TI>::BYTES;
  const int64_t warp_id = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const int nq = P->nq;
  if (nq <= 0) return;
  if (mode == 0) {
    const int64_t n_intra = P->n_intra_items;
    const int64_t total = n_intra + P->n_inter_items;
    for (;;) {
      unsigned long long it = 0;
      if (lane == 0) it = atomicAdd(&st->work, 1ull);
      it = __shfl_sync(FULL, it, 0);
      if ((int64_t)it >= total) break;
      if ((int64_t)it < n_intra) {
        const int s = (int)((int64_t)it / nq);
        const int q = P->qorder[(int64_t)it % nq];
        intra_item<TI>(db, P, sm, slice, lane, warp_id, scr, q, s);
      } else {
        const int64_t k = (int64_t)it - n_intra;
        const int g = P->g_first + (int)(k / nq);
        const int q = P->qorder[k % nq];
        inter_item<T>(db, P, st, sm, slice, lane, warp_id, scr, q, g);
      }
    }
  } else {
    const unsigned long long nf = *(volatile unsigned long long*)&st->n_flags;
    const unsigned long long total =
        nf < (unsigned long long)scr.flag_capacity ? nf : (unsigned long long)scr.flag_capacity;
    for (;;) {
      unsigned long long it = 0;
      if (lane == 0) it = atomicAdd(&st->recompute, 1ull);
      it = __shfl_sync(FULL, it, 0);
      if (it >= total) break;
      const int2 fl = scr.flags[it];
      intra_item<TI>(db, P, sm, slice, lane, warp_id, scr, fl.x, fl.y);
    }
  }
}

typedef void (*SearchKernel)(int, DbView, const SearchParams*, SearchState*, Scratch);

static SearchKernel pick_search(int rows, int intra_rows) {
  if (rows == 16 && intra_rows == 8) return search_kernel<16, 8>;
  if (rows == 16 && intra_rows == 16) return search_kernel<16, 16>;
  if (rows == 32 && intra_rows == 8) return search_kernel<32, 8>;
  if (rows == 32 && intra_rows == 16) return search_kernel<32, 16>;
  return nullptr;
}

static int slice_bytes(int rows, int intra_rows) {
  if (rows == 16 && intra_rows == 8) return SliceBytes<16, 8>::BYTES;
  if (rows == 16 && intra_rows == 16) return SliceBytes<16, 16>::BYTES;
  if (rows == 32 && intra_rows == 8) return SliceBytes<32, 8>::BYTES;
  if (rows == 32 && intra_rows == 16) return SliceBytes<32, 16>::BYTES;
  return 0;
}

size_t search_smem_bytes(int rows, int intra_rows, int warps) {
  return (size_t)MATRIX_SMEM + (size_t)warps * slice_bytes(rows, intra_rows);
}

int search_blocks_per_sm(int rows, int intra_rows, int warps) {
  SearchKernel k = pick_search(rows, intra_rows);
  if (!k || warps < 1 || warps > 8) return 0;
  const size_t smem = search_smem_bytes(rows, intra_rows, warps);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, warps * 32, smem) != cudaSuccess)
    return 0;
  return nb;
}

cudaError_t launch_search(const KernelConfig& kc, int mode, const DbView& db,
                          const SearchParams* params, SearchState* state, const Scratch& scr,
                          cudaStream_t stream) {
  // the dynamic shared-memory attribute was set by search_blocks_per_sm when
  // the plan was created; nothing here may be an unsafe call under capture
  SearchKernel k = pick_search(kc.rows, kc.intra_rows);
  if (!k) return cudaErrorInvalidValue;
  k<<<kc.blocks, kc.warps * 32, kc.smem, stream>>>(mode, db, params, state, scr);
  return cudaGetLastError();
}

// ---- packed intra-task kernel: one warp per pair of long subjects ----------
// The two subjects of a pair are adjacent in length order, packed as the two
// 16-bit halves of every word (the shorter one reads pad columns past its
// end, which cannot raise its score).  Lane k owns PR query rows of a
// 32*PR-row pass, split into PQ quarters of PQR rows; quarter q of lane k
// updates column t - PQ*k - q at step t (Section II-B, intra-task
// parallelism with neighbour border exchange):
//   * quarter q needs the bottom row of quarter q - 1 at the same column
//     (produced one step earlier) and its H' one column back (two steps
//     earlier), so the PQ quarter updates of a step are independent;
//   * quarter 0 receives the bottom row of lane k - 1 (its quarter PQ - 1,
//     one step earlier) by __shfl_up_sync; lane 0 reads the previous pass's
//     bottom row from this warp's border scratch and lane 31 writes it (index
//     c is read at step c and rewritten at step c + 32*PQ - 1).
// Residues are staged in a per-warp shared-memory ring 128 columns ahead;
// quarter 0 loads the 16-byte profile row of its column and later quarters
// reuse its words.  Values carry the +Go bias of the inter-task kernel, and a
// pair half whose S' reaches the threshold is recomputed in int32 like any
// other saturated pair.
constexpr int PR = 16;                          // packed rows per lane
constexpr int PQ = 4;                           // quarters (independent chains) per lane
constexpr int PQR = PR / PQ;                    // rows per quarter
constexpr int PAIR_PROFILE = NCODES * 32 * PR;  // int8 [code][lane][PR]
constexpr int PRING = 384;                      // residue ring per subject: 3 blocks of 128
constexpr int PAIR_SLICE = PAIR_PROFILE + 2 * PRING;

__global__ void __launch_bounds__(PAIR_WARPS * 32, 4)
pair_kernel(DbView db, const SearchParams* __restrict__ P, SearchState* st, Scratch scr) {
  extern __shared__ __align__(16) uint8_t smem[];
  int8_t* sm = (int8_t*)smem;
  for (int i = threadIdx.x; i < NCODES * NCODES; i += blockDim.x) sm[i] = P->sm[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint8_t* prof = smem + MATRIX_SMEM + wib * PAIR_SLICE;
  uint8_t* ring0 = prof + PAIR_PROFILE;
  uint8_t* ring1 = ring0 + PRING;
  const int64_t warp_id = (int64_t)blockIdx.x * PAIR_WARPS + wib;
  uint2* hb = scr.pair_border + warp_id * scr.pair_stride;
  const int nq = P->nq;
  if (nq <= 0) return;
  const int64_t total = P->n_pair_items;
  const int go = P->go;
  const uint32_t GO2 = pack2(go), NGE2 = pack2(-P->ge);
  const uint32_t MGO = (uint32_t)(-(int)((uint32_t)go * 65537u));
  const uint32_t one = (uint32_t)P->one;
  constexpr int ROWS = 32 * PR;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(&st->pair_work, 1ull);
    it = __shfl_sync(FULL, it, 0);
    if ((int64_t)it >= total) break;
    const int pair = (int)((int64_t)it / nq);
    const int q = P->qorder[(int64_t)it % nq];
    const int s0 = 2 * pair, s1 = 2 * pair + 1;
    const bool has1 = s1 < P->n_long;
    const int n0 = db.clen[s0], n1 = has1 ? db.clen[s1] : 0;  // n0 >= n1 (sorted)
    const uint8_t* __restrict__ d0 = db.cont + db.coff[s0];
    const uint8_t* __restrict__ d1 = has1 ? db.cont + db.coff[s1] : d0;
    const int m = P->qlen[q];
    const uint8_t* __restrict__ qr = P->qres + P->qoff[q];
    const int npass = n0 > 0 ? (m + ROWS - 1) / ROWS : 0;
    // residues of columns [128 b, 128 b + 128) into ring slot b % 3 (pad past the end)
    auto load_block = [&](int b) {
      const int c = 128 * b + 4 * lane;
      uint32_t w0 = 0, w1 = 0;
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const int cc = c + i;
        w0 |= (uint32_t)(cc < n0 ? d0[cc] : PAD_CODE) << (8 * i);
        w1 |= (uint32_t)(cc < n1 ? d1[cc] : PAD_CODE) << (8 * i);
      }
      *(uint32_t*)(ring0 + c % PRING) = w0;
      *(uint32_t*)(ring1 + c % PRING) = w1;
    };
    uint32_t smax = GO2;
    for (int p = 0; p < npass; p++) {
      __syncwarp();
      {  // this lane's PR rows for every code
        const int i0 = p * ROWS + lane * PR;
        int qc[PR];
#pragma unroll
        for (int r = 0; r < PR; r++) qc[r] = (i0 + r < m) ? (int)qr[i0 + r] : -1;
        for (int c = 0; c < NCODES; c++) {
          uint32_t wv[PR / 4];
#pragma unroll
          for (int w = 0; w < PR / 4; w++) {
            uint32_t acc = 0;
#pragma unroll
            for (int b = 0; b < 4; b++) {
              const int r = w * 4 + b;
              const int v = qc[r] >= 0 ? (int)sm[qc[r] * NCODES + c] : PAD_SCORE;
              acc |= ((uint32_t)(uint8_t)(int8_t)v) << (8 * b);
            }
            wv[w] = acc;
          }
          *(uint4*)(prof + (c * 32 + lane) * PR) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
      }
      load_block(0);
      __syncwarp();
      uint32_t Hp[PR], E[PR];
#pragma unroll
      for (int r = 0; r < PR; r++) {
        Hp[r] = GO2;  // H(i, 0) = 0
        E[r] = 0u;    // E(i, 1) = -Go
      }
      // quarter q's bottom-row H' one and two steps back, its F' one step back
      uint32_t qh1[PQ], qh2[PQ], qf1[PQ];
#pragma unroll
      for (int k = 0; k < PQ; k++) {
        qh1[k] = GO2;
        qh2[k] = GO2;
        qf1[k] = 0u;
      }
      // profile vectors of the last four steps in slot (t mod 4): quarter q at
      // step t uses word q of the vector loaded at step t - q; steps run in
      // blocks of four so every slot index is a compile-time constant
      uint4 VA[PQ], VB[PQ];
#pragma unroll
      for (int k = 0; k < PQ; k++) {
        VA[k] = make_uint4(0u, 0u, 0u, 0u);
        VB[k] = make_uint4(0u, 0u, 0u, 0u);
      }
      uint32_t hdiag = GO2, out_h = GO2, out_f = 0u;
      const bool last_pass = (p == npass - 1);
      const int steps = n0 + 32 * PQ - 1;
      // ring position of column t0 - PQ*lane; a multiple of 4, as is PRING
      int pos = (PRING - (PQ * lane) % PRING) % PRING;
      // one step of the wavefront; CHECK: some quarter may lie outside the
      // columns (ramp-up and drain); in the steady state every quarter of
      // every lane is inside, so the step needs no per-quarter test
      auto step = [&](const int t, auto checked, auto slot) {
        constexpr bool CHECK = decltype(checked)::value;
        constexpr int U = decltype(slot)::value;  // t mod 4
        if constexpr (U == 0) {
          if ((t & 127) == 0) {
            load_block((t >> 7) + 1);
            __syncwarp();
          }
        }
        uint32_t in_h = __shfl_up_sync(FULL, out_h, 1);
        uint32_t in_f = __shfl_up_sync(FULL, out_f, 1);
        const int c0 = t - PQ * lane;  // quarter 0's column
        if (lane == 0) {
          if (p > 0 && c0 < n0) {
            const uint2 v = hb[c0];
            in_h = v.x;
            in_f = v.y;
          } else {
            in_h = GO2;  // H(0, j) = 0
            in_f = 0u;   // F(1, j) = -Go
          }
        }
        // a ring slot not yet filled (this lane has not started) may hold any
        // byte: clamp so the profile address stays inside this warp's slice
        const int ra = min((int)ring0[pos + U], PAD_CODE);
        const int rb = min((int)ring1[pos + U], PAD_CODE);
        VA[U] = *(const uint4*)(prof + (ra * 32 + lane) * PR);
        VB[U] = *(const uint4*)(prof + (rb * 32 + lane) * PR);
        const uint32_t wa[PQ] = {VA[U].x, VA[(U + 3) & 3].y, VA[(U + 2) & 3].z, VA[(U + 1) & 3].w};
        const uint32_t wb[PQ] = {VB[U].x, VB[(U + 3) & 3].y, VB[(U + 2) & 3].z, VB[(U + 1) & 3].w};
        uint32_t nh[PQ], nf[PQ];
#pragma unroll
        for (int k = 0; k < PQ; k++) {
          const int col = c0 - k;
          bool active = true;
          if constexpr (CHECK) active = col >= 0 && col < n0;
          nh[k] = qh1[k];
          nf[k] = qf1[k];
          if (active) {
            uint32_t hd = k == 0 ? hdiag : qh2[k - 1];  // H' one row up, one column back
            uint32_t f = k == 0 ? in_f : qf1[k - 1];    // F' of this quarter's first row
            uint32_t hprev = 0;
#pragma unroll
            for (int i = 0; i < PQR; i++) {
              const int r = k * PQR + i;
              uint32_t e = E[r];
              const uint32_t h = packed_cell(hd, prmt(wa[k], wb[k], sext_pair_sel(i)), e, f, GO2,
                                             NGE2, MGO, one);
              hd = Hp[r];
              Hp[r] = h;
              E[r] = e;
              if (i & 1)
                smax = __vimax3_s16x2(smax, hprev, h);
              else
                hprev = h;
            }
            nh[k] = Hp[k * PQR + PQR - 1];
            nf[k] = f;
            if (k == PQ - 1 && lane == 31 && !last_pass) hb[col] = make_uint2(nh[k], f);
          } else if (col < 0) {
            nh[k] = GO2;  // left of the matrix: H = 0
          }
        }
        hdiag = in_h;
        out_h = nh[PQ - 1];
        out_f = nf[PQ - 1];
#pragma unroll
        for (int k = 0; k < PQ; k++) {
          qh2[k] = qh1[k];
          qh1[k] = nh[k];
          qf1[k] = nf[k];
        }
      };
      auto block = [&](const int t0, auto checked) {
        step(t0, checked, std::integral_constant<int, 0>{});
        step(t0 + 1, checked, std::integral_constant<int, 1>{});
        step(t0 + 2, checked, std::integral_constant<int, 2>{});
        step(t0 + 3, checked, std::integral_constant<int, 3>{});
        pos = pos + 4 == PRING ? 0 : pos + 4;
      };
      // every quarter of every lane is inside the columns for 32*PQ-1 <= t < n0;
      // the last block may run past `steps`, where every quarter is outside
      int t0 = 0;
      for (; t0 < 32 * PQ; t0 += 4) block(t0, std::true_type{});
#pragma unroll 1
      for (; t0 + 4 <= n0; t0 += 4) block(t0, std::false_type{});
      for (; t0 < steps; t0 += 4) block(t0, std::true_type{});
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) smax = __vmaxs2(smax, __shfl_xor_sync(FULL, smax, o));
    if (lane < 2 && (lane == 0 || has1)) {
      const int sidx = lane ? s1 : s0;
      const int sb = (int)(int16_t)(lane ? (smax >> 16) : (smax & 0xffffu));  // S'
      const int orig = db.perm[sidx];
      if (orig >= 0) {
        if (sb >= P->sat_threshold) {
          const unsigned long long k = atomicAdd(&st->n_flags, 1ull);
          if ((int64_t)k < scr.flag_capacity) scr.flags[k] = make_int2(q, sidx);
        } else {
          P->scores[(int64_t)q * db.n + orig] = sb - go;
        }
      }
    }
  }
}

size_t pair_smem_bytes() { return (size_t)MATRIX_SMEM + (size_t)PAIR_WARPS * PAIR_SLICE; }

int pair_blocks_per_sm() {
  const size_t smem = pair_smem_bytes();
  if (cudaFuncSetAttribute(pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pair_kernel, PAIR_WARPS * 32, smem) !=
      cudaSuccess)
    return 0;
  return nb;
}

cudaError_t launch_pairs(int blocks, const DbView& db, const SearchParams* params,
                         SearchState* state, const Scratch& scr, cudaStream_t stream) {
  pair_kernel<<<blocks, PAIR_WARPS * 32, pair_smem_bytes(), stream>>>(db, params, state, scr);
  return cudaGetLastError();
}

// ---- plain int32 baseline: Algorithm 1, one launch per query ---------------
constexpr int PT = 8;  // query rows per thread
constexpr int NEG = -(1 << 28);

__global__ void __launch_bounds__(GROUP)
plain_kernel(DbView db, const SearchParams* __restrict__ P, int q, int2* border,
             const int64_t* __restrict__ border_off) {
  __shared__ int8_t sm[NCODES * NCODES];
  __shared__ int prof[NCODES][PT];
  for (int i = threadIdx.x; i < NCODES * NCODES; i += blockDim.x) sm[i] = P->sm[i];
  const int k = threadIdx.x;  // subject slot in the group
  const int m = P->qlen[q];
  const uint8_t* __restrict__ qr = P->qres + P->qoff[q];
  const int go = P->go, ge = P->ge;
  int2* bd = border + border_off[blockIdx.x] + k;
  __syncthreads();
  for (int g = blockIdx.x; g < db.groups; g += gridDim.x) {
    const int L = db.glen[g];
    const uint2* __restrict__ res = (const uint2*)(db.inter + db.goff[g]) + k;
    const int nstrips = L > 0 ? (m + PT - 1) / PT : 0;
    int S = 0;
    for (int s = 0; s < nstrips; s++) {
      __syncthreads();
      for (int i = threadIdx.x; i < NCODES * PT; i += blockDim.x) {
        const int c = i / PT, r = i % PT, row = s * PT + r;
        prof[c][r] = row < m ? (int)sm[(int)qr[row] * NCODES + c] : PAD_SCORE;
      }
      __syncthreads();
      int Hl[PT], El[PT];
#pragma unroll
      for (int r = 0; r < PT; r++) {
        Hl[r] = 0;
        El[r] = NEG;
      }
      int hul = 0;
      const bool last = (s == nstrips - 1);
      for (int c = 0; c < L / CHUNK; c++) {
        const uint2 rr = res[c * GROUP];
#pragma unroll
        for (int jj = 0; jj < CHUNK; jj++) {
          const int cj = ((jj < 4 ? rr.x : rr.y) >> (8 * (jj & 3))) & 0xff;
          int hu = 0, fu = NEG;  // H and F of the row above the strip
          if (s > 0) {
            const int2 v = bd[(c * CHUNK + jj) * GROUP];
            hu = v.x;
            fu = v.y;
          }
          int hd = hul;
          hul = hu;
#pragma unroll
          for (int r = 0; r < PT; r++) {
            // Algorithm 1: E, F, H, S
            const int e = max(El[r] - ge, Hl[r] - go);
            const int f = max(fu - ge, hu - go);
            int h = hd + prof[cj][r];
            h = max(h, e);
            h = max(h, f);
            h = max(h, 0);
            S = max(h, S);
            hd = Hl[r];
            Hl[r] = h;
            El[r] = e;
            hu = h;
            fu = f;
          }
          if (!last) bd[(c * CHUNK + jj) * GROUP] = make_int2(hu, fu);
        }
      }
    }
    const int orig = db.perm[g * GROUP + k];
    if (orig >= 0) P->scores[(int64_t)q * db.n + orig] = S;
  }
}

int plain_blocks_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, plain_kernel, GROUP, 0) != cudaSuccess)
    return 0;
  return nb;
}

cudaError_t launch_plain(int blocks, const DbView& db, const SearchParams* params, int query,
                         int2* border, const int64_t* border_off, cudaStream_t stream) {
  plain_kernel<<<blocks, GROUP, 0, stream>>>(db, params, query, border, border_off);
  return cudaGetLastError();
}

}  // namespace swgb
