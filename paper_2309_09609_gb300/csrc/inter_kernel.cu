// inter_kernel.cu -- the inter-task kernel of libswgb: packed 16-bit pairs.
//
// Item = (query, group of 64 length-sorted subjects).  Each lane owns two
// subjects, packed as the two 16-bit halves of every 32-bit word, and T query
// rows held in registers; it sweeps the group's columns strip by strip
// (Section II-B: inter-task parallelism, one matrix per processing element).
// One persistent launch takes (query, group) items longest-first from an
// atomic counter.  A pair whose 16-bit score reaches 32767 - max(SM) is
// appended to the flag list for the int32 recompute (intra_kernel.cu).
#include "device_common.cuh"

namespace swgb {

// ---- shared-memory slice of a warp ------------------------------------------
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


// Four adjacent columns of T rows as a wavefront: at step k, column c
// updates row k - c.  Column c's row r needs E' of column c - 1 at row r
// (written one step earlier) and its H' at row r - 1 (two steps earlier), so
// the up to four updates of a step are independent.  Hp[r] / E[r] hold H' / E'
// of the previous column on entry and of the fourth column on exit; b0, b1
// are the border vectors (H'_c, F'_c) above the strip for columns 0,1 and 2,3;
// o0, o1 receive the strip's bottom row in the same layout.
template <int T, int G>
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
      out[c] = packed_cell<G>(hd, profile_word<T>(pa[c], pb[c], r), e, f[c], GO2, NGE2, MGO, one);
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

// Eight adjacent columns -- a whole 8-residue chunk -- as one wavefront, for
// T = 32: the same skew as packed_quad (column c updates row k - c at step
// k), with up to eight independent cell updates per step.  Each column holds
// only the 16-row half of its profile row that its current rows need,
// loaded when the column reaches row 0 and row 16, so eight columns take the
// profile registers of four.  b[q] / o[q] hold (H'_c, F'_c) of columns 2q and
// 2q + 1 above / at the bottom of the strip.
template <int T, int G>
__device__ __forceinline__ void packed_oct(uint32_t (&Hp)[T], uint32_t (&E)[T], uint32_t& hdiag,
                                           uint32_t& smax, const uint8_t* slice, int p16,
                                           const uint4& rr, const uint4 (&b)[4], uint4 (&o)[4],
                                           uint32_t GO2, uint32_t NGE2, uint32_t MGO,
                                           uint32_t one) {
  static_assert(T == 32, "the eight-column wavefront is for 32 rows");
  constexpr int HALVES = 2;
  constexpr int W = 8;
  uint32_t ca[W], cb[W];
#pragma unroll
  for (int c = 0; c < W; c++) {
    ca[c] = ((c < 4 ? rr.x : rr.y) >> (8 * (c & 3))) & 0xffu;
    cb[c] = ((c < 4 ? rr.z : rr.w) >> (8 * (c & 3))) & 0xffu;
  }
  uint4 pa[W], pb[W];
  uint32_t htop[W], f[W], last[W], last2[W], bottom[W];
#pragma unroll
  for (int q = 0; q < 4; q++) {
    htop[2 * q] = b[q].x;
    f[2 * q] = b[q].y;
    htop[2 * q + 1] = b[q].z;
    f[2 * q + 1] = b[q].w;
  }
#pragma unroll
  for (int c = 0; c < W; c++) last[c] = last2[c] = bottom[c] = 0u;
  uint32_t hd0 = hdiag;  // column 0's diagonal: previous column, previous row
  hdiag = htop[W - 1];
#pragma unroll
  for (int k = 0; k < T + W - 1; k++) {
    uint32_t out[W];
#pragma unroll
    for (int c = 0; c < W; c++) {
      out[c] = 0u;
      const int r = k - c;
      if (r < 0 || r >= T) continue;
      if ((r & 15) == 0) {  // this column enters a new 16-row half of its profile row
        const int h = r >> 4;
        pa[c] = *(const uint4*)(slice + (ca[c] * HALVES + h) * 128 + p16);
        pb[c] = *(const uint4*)(slice + (cb[c] * HALVES + h) * 128 + p16);
      }
      uint32_t hd;
      if (c == 0) {
        hd = hd0;
        hd0 = Hp[r];
      } else {
        hd = r == 0 ? htop[c - 1] : last2[c - 1];  // H' of column c - 1, row r - 1
      }
      const int wq = (r >> 2) & 3;
      const uint32_t a32 = wq == 0 ? pa[c].x : wq == 1 ? pa[c].y : wq == 2 ? pa[c].z : pa[c].w;
      const uint32_t b32 = wq == 0 ? pb[c].x : wq == 1 ? pb[c].y : wq == 2 ? pb[c].z : pb[c].w;
      uint32_t e = E[r];
      out[c] = packed_cell<G>(hd, prmt(a32, b32, sext_pair_sel(r & 3)), e, f[c], GO2, NGE2, MGO, one);
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
#pragma unroll
  for (int q = 0; q < 4; q++) o[q] = make_uint4(bottom[2 * q], f[2 * q], bottom[2 * q + 1], f[2 * q + 1]);
}

template <int T, int WC, int G>
__device__ void inter_item(const DbView& db, const SearchParams* __restrict__ P, SearchState* st,
                           const int8_t* __restrict__ sm, uint8_t* slice, int lane,
                           int64_t warp_id, const Scratch& scr, int q, int g) {
  const int L = db.glen[g];  // multiple of CHUNK
  const int m = P->qlen[q];
  const uint8_t* __restrict__ qr = P->qres + P->qoff[q];
  const uint4* __restrict__ res = (const uint4*)(db.inter + db.goff[g]) + lane;
  uint4* bd = scr.inter_border + warp_id * scr.inter_stride_vec + lane;
  const int go = P->go;
  uint32_t GO2, NGE2, MGO;  // (Go, Go), (-Ge, -Ge), -(Go, Go)
  gap_words<G>(P, GO2, NGE2, MGO);
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
      if constexpr (WC == 8) {  // the whole chunk as one eight-column wavefront
        const uint4 bv[4] = {bring[(slot * 4 + 0) * 32], bring[(slot * 4 + 1) * 32],
                             bring[(slot * 4 + 2) * 32], bring[(slot * 4 + 3) * 32]};
        uint4 ov[4];
        packed_oct<T, G>(Hp, E, hdiag, smax, slice, p16, rr, bv, ov, GO2, NGE2, MGO, one);
        if (!last) {
#pragma unroll
          for (int q = 0; q < 4; q++) bd[(c * 4 + q) * 32] = ov[q];
        }
        continue;
      }
      // two groups of 4 columns (one residue word per subject each); for
      // T = 16 both are unrolled so the second group's profile loads can be
      // issued during the first group's wavefront tail
      auto group = [&](int hq) {
        const uint32_t wa = hq ? rr.y : rr.x;
        const uint32_t wb = hq ? rr.w : rr.z;
        const uint4 b0 = bring[(slot * 4 + 2 * hq) * 32];
        const uint4 b1 = bring[(slot * 4 + 2 * hq + 1) * 32];
        uint4 o0, o1;
        packed_quad<T, G>(Hp, E, hdiag, smax, slice, p16, wa, wb, b0, b1, o0, o1, GO2, NGE2, MGO,
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
      if ((int64_t)k < scr.flag_capacity)
        scr.flags[k] = make_int2(q, sidx);
      else  // the list is full: mark the pair for the host's next recompute round
        P->scores[(int64_t)q * db.n + orig] = FLAG_SENTINEL;
    } else {
      P->scores[(int64_t)q * db.n + orig] = sb - go;
    }
  }
}

template <int T, int WC, int G>
__global__ void __launch_bounds__(256, (T == 16 ? 2 : 1))
inter_kernel(DbView db, const SearchParams* __restrict__ P, SearchState* st, Scratch scr) {
  extern __shared__ __align__(16) uint8_t smem[];
  int8_t* sm = (int8_t*)smem;
  load_matrix(sm, P);
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint8_t* slice = smem + MATRIX_SMEM + wib * InterProfile<T>::BYTES;
  const int64_t warp_id = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const int nq = P->nq;
  if (nq <= 0) return;
  const int64_t total = P->n_inter_items;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(&st->work, 1ull);
    it = __shfl_sync(FULL, it, 0);
    if ((int64_t)it >= total) break;
    const int g = P->g_first + (int)((int64_t)it / nq);
    const int q = P->qorder[(int64_t)it % nq];
    inter_item<T, WC, G>(db, P, st, sm, slice, lane, warp_id, scr, q, g);
  }
}

typedef void (*InterKernel)(DbView, const SearchParams*, SearchState*, Scratch);

// The default shape (32 rows, eight columns) is compiled for each gap class;
// the others read the penalties at run time.
static InterKernel pick_inter(int rows, int cols, int gclass) {
  if (rows == 16 && cols == 4) return inter_kernel<16, 4, 0>;
  if (rows == 32 && cols == 4) return inter_kernel<32, 4, 0>;
  if (rows == 32 && cols == 8)
    return gclass == 1 ? inter_kernel<32, 8, 1> : gclass == 2 ? inter_kernel<32, 8, 2>
                                                              : inter_kernel<32, 8, 0>;
  return nullptr;
}

size_t inter_smem_bytes(int rows, int warps) {
  const int slice = rows == 16 ? InterProfile<16>::BYTES : InterProfile<32>::BYTES;
  return (size_t)MATRIX_SMEM + (size_t)warps * slice;
}

int inter_blocks_per_sm(int rows, int cols, int warps) {
  InterKernel k = pick_inter(rows, cols, 0);
  if (!k || warps < 1 || warps > 8) return 0;
  const size_t smem = inter_smem_bytes(rows, warps);
  for (int g = 0; g < GAP_CLASSES; g++)  // every variant the plan may launch
    if (cudaFuncSetAttribute(pick_inter(rows, cols, g), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, warps * 32, smem) != cudaSuccess)
    return 0;
  return nb;
}

cudaError_t launch_inter(const KernelConfig& kc, int gclass, const DbView& db,
                         const SearchParams* params, SearchState* state, const Scratch& scr,
                         cudaStream_t stream) {
  // the dynamic shared-memory attribute was set by inter_blocks_per_sm when
  // the plan was created; nothing here may be an unsafe call under capture
  InterKernel k = pick_inter(kc.variant, kc.cols, gclass);
  if (!k) return cudaErrorInvalidValue;
  cudaGetLastError();  // a stale error must not be read as this launch's
  k<<<kc.blocks, kc.warps * 32, kc.smem, stream>>>(db, params, state, scr);
  return cudaGetLastError();
}

}  // namespace swgb
