// inter2q_kernel.cu -- the inter-task kernel of libswgb with two queries per
// 32-bit word.
//
// The packed inter-task kernel (inter_kernel.cu) puts two subjects in the two
// 16-bit halves of a word, so each cell's substitution score SM(q_i, d_j)
// comes from two profile rows (one per subject's residue) and costs one
// byte-merge instruction per word.  Here each lane owns ONE subject and the
// two halves hold two different queries: the word of query rows (a_i, b_i)
// against residue d_j is (SM(a_i, d_j), SM(b_i, d_j)), a single entry of a
// per-strip profile built for the query pair, read ready-made from shared
// memory.  The cell update is the same biased packed update (Eq. 1-3), so a
// word costs 4.5 ALU-pipe operations instead of 5.5.
//
// Queries are laid out in "query streams": the plan deals the batch's queries
// to pairs of streams (longest first, each to the shorter stream), each query
// padded to whole strips of T rows, and a warp sweeps the two streams of a
// stream pair together, strip by strip -- half 0 holding stream 0's rows,
// half 1 stream 1's.  A strip table gives, per strip, each half's query and
// first row and whether the strip is that query's last: there the half's
// score S is emitted (or flagged for the int32 recompute) and reset, and the
// strip's bottom row is stored as the empty row above the matrix (H = 0,
// F = -Go) for the next query of that half.
//
// Item = (stream pair, half of a 64-subject group): lane l scores subject
// 2l + h of the group in the interleaved layout of the database.  One
// persistent launch takes items from an atomic counter, longest groups first.
#include "device_common.cuh"

namespace swgb {

constexpr int Q2RING = 3;  // chunks in flight per warp

// Warp slice: the strip profile, int16 pairs.  The 20 standard amino acids
// (codes 0..19) are replicated 8x so that the 8 lanes of a quarter-warp read
// 16-byte blocks of any of them from 8 distinct bank groups:
//   word (code c, row r) of copy p at ((c * RB + r / 4) * 8 + p) * 16 + 4 * (r % 4)
// The rare codes B, Z, X, * and the padding code (20..24) are stored once,
// each block of 4 rows in its own 16-byte column of a 128-byte line, so two
// lanes reading one of them share a broadcast and lanes reading different
// ones hit different bank groups:
//   word (code c, row r) at RARE + (r / 4) * 128 + (c - 20) * 16 + 4 * (r % 4)
// Either way a column's block b lies at base(c) + b * 128.  Then the
// cp.async ring: per chunk, the 4 border vectors of every lane and the
// lane's 8 residues.  With the rare codes compacted, 12 warps fit an SM at
// 16 rows, 10 at 24 and 8 at 32.
constexpr int Q2COMMON = 20;  // replicated codes
template <int T>
struct Q2Shape {
  static_assert(T % 8 == 0 && T >= 16 && T <= 32, "16, 24 or 32 rows per strip");
  static constexpr int RB = T / 4;                               // 4-row profile blocks
  static constexpr int RARE = Q2COMMON * RB * 8 * 16;
  static constexpr int PROFILE = RARE + RB * 128;
  static constexpr int BORDER_RING = PROFILE;                    // Q2RING x 4 x 32 x 16 bytes
  static constexpr int RES_RING = BORDER_RING + Q2RING * 4 * 512;  // Q2RING x 32 x 8 bytes
  static constexpr int BYTES = RES_RING + Q2RING * 256;
  static constexpr int WARPS = T == 16 ? 12 : T == 24 ? 10 : 8;  // per block, one block per SM
};

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem_src) : "memory");
}

// W adjacent columns -- columns C0 .. C0 + W - 1 of an 8-residue chunk of the
// lane's subject -- as one wavefront: column c updates row k - c at step k,
// so up to W cell updates of a step are independent.  A column loads its
// profile words 4 rows at a time (one 16-byte read) when it enters a 4-row
// block.  b[q] / o[q] hold (H'_c, F'_c) of columns 2q and 2q + 1 above / at
// the bottom of the strip.  A chunk runs as two wavefronts of four columns:
// on the paper-shaped search that was 3% faster than one of eight (880
// against 907 ms at 32 rows) and no slower than four of two.
template <int T, int W, int C0, int G>
__device__ __forceinline__ void q2_wave(uint32_t (&Hp)[T], uint32_t (&E)[T], uint32_t& hdiag,
                                       uint32_t& smax, const uint8_t* prof, int p16, const uint2 rr,
                                       const uint4* b, uint4* o, uint32_t GO2,
                                       uint32_t NGE2, uint32_t MGO, uint32_t one) {
  constexpr int RB = Q2Shape<T>::RB;
  uint32_t cb[W];  // base(c) of each column's residue code
#pragma unroll
  for (int c = 0; c < W; c++) {
    const int cc = C0 + c;
    const uint32_t code = prmt(cc < 4 ? rr.x : rr.y, 0u, 0x4440u + (cc & 3));  // byte cc % 4
    // base(code) as the smaller of the two layouts' offsets: a standard code's
    // (code * RB * 128 + p16, at most RARE - RB * 128 + 112) is below any rare
    // one's (RARE + (code - 20) * 16, at least RARE - 320), and for a rare code
    // the replicated formula gives at least RARE + p16; two multiply-adds on
    // the FMA pipe and one min instead of a compare and select
    cb[c] = min(imad(code, (uint32_t)(RB * 128), (uint32_t)p16),
                imad(code, 16u, (uint32_t)(Q2Shape<T>::RARE - Q2COMMON * 16)));
  }
  uint4 pw[W];
  uint32_t htop[W], f[W], last[W], last2[W], bottom[W];
#pragma unroll
  for (int q = 0; q < W / 2; q++) {
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
      if ((r & 3) == 0) pw[c] = *(const uint4*)(prof + cb[c] + (r >> 2) * 128);
      const uint32_t w = (r & 3) == 0 ? pw[c].x : (r & 3) == 1 ? pw[c].y : (r & 3) == 2 ? pw[c].z : pw[c].w;
      uint32_t hd;
      if (c == 0) {
        hd = hd0;
        hd0 = Hp[r];
      } else {
        hd = r == 0 ? htop[c - 1] : last2[c - 1];  // H' of column c - 1, row r - 1
      }
      uint32_t e = E[r];
      out[c] = packed_cell<G>(hd, w, e, f[c], GO2, NGE2, MGO, one);
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
  for (int q = 0; q < W / 2; q++)
    o[q] = make_uint4(bottom[2 * q], f[2 * q], bottom[2 * q + 1], f[2 * q + 1]);
}

// The 16-bit S' of one half: recorded (or flagged for the int32 recompute
// when it may have saturated) as the score of (query q, sorted subject sidx).
__device__ __forceinline__ void q2_emit(const DbView& db, const SearchParams* __restrict__ P,
                                        SearchState* st, const Scratch& scr, int q, int sidx,
                                        int orig, int sb) {
  if (q < 0 || orig < 0) return;
  if (sb >= P->sat_threshold) {
    const unsigned long long k = atomicAdd(&st->n_flags, 1ull);
    if ((int64_t)k < scr.flag_capacity)
      scr.flags[k] = make_int2(q, sidx);
    else  // the list is full: mark the pair for the host's next recompute round
      P->scores[(int64_t)q * db.n + orig] = FLAG_SENTINEL;
  } else {
    P->scores[(int64_t)q * db.n + orig] = sb - P->go;
  }
}

template <int T, int G>
__device__ void q2_item(const DbView& db, const SearchParams* __restrict__ P, SearchState* st,
                        const int8_t* __restrict__ sm, uint8_t* slice, int lane, int64_t warp_id,
                        const Scratch& scr, int k, int g, int h) {
  constexpr int RB = Q2Shape<T>::RB;
  const int L = db.glen[g];  // multiple of CHUNK
  const int2 sp = P->spairs[k];  // (first strip, strips) of this stream pair
  // this lane's 8 residues of chunk c: bytes [8h, 8h + 8) of its 16-byte vector
  const uint2* __restrict__ res = (const uint2*)(db.inter + db.goff[g]) + lane * 2 + h;
  uint4* bd = scr.inter_border + warp_id * scr.inter_stride_vec + lane;
  uint32_t GO2, NGE2, MGO;  // (Go, Go), (-Ge, -Ge), -(Go, Go)
  gap_words<G>(P, GO2, NGE2, MGO);
  const uint32_t one = (uint32_t)P->one;
  const int p16 = (lane & 7) * 16;
  const int nch = L / CHUNK;
  const int sidx = g * GROUP + 2 * lane + h;
  const int orig = db.perm[sidx];
  uint4* bring = (uint4*)(slice + Q2Shape<T>::BORDER_RING) + lane;  // [slot][pair][lane]
  uint2* rring = (uint2*)(slice + Q2Shape<T>::RES_RING) + lane;     // [slot][lane]
  uint32_t smax = GO2;  // S' of S = 0, both halves
  for (int s = 0; s < sp.y; s++) {
    const int4 si = P->strips[sp.x + s];
    const int qa = si.x, qb = si.z;                // -1: no query in that half
    const int ia = si.y & 0x7fffffff, ib = si.w & 0x7fffffff;
    const bool enda = si.y < 0, endb = si.w < 0;   // the strip is that query's last
    __syncwarp();
    if (lane < NCODES) {  // code c = lane: its T words (8 copies of a standard code)
      const uint8_t* __restrict__ qra = qa >= 0 ? P->qres + P->qoff[qa] : nullptr;
      const uint8_t* __restrict__ qrb = qb >= 0 ? P->qres + P->qoff[qb] : nullptr;
      const int ma = qa >= 0 ? P->qlen[qa] : 0, mb = qb >= 0 ? P->qlen[qb] : 0;
      uint32_t wv[T];
#pragma unroll
      for (int r = 0; r < T; r++) {
        const int va = ia + r < ma ? (int)sm[(int)qra[ia + r] * NCODES + lane] : PAD_SCORE;
        const int vb = ib + r < mb ? (int)sm[(int)qrb[ib + r] * NCODES + lane] : PAD_SCORE;
        wv[r] = (uint32_t)(uint16_t)(int16_t)va | ((uint32_t)(uint16_t)(int16_t)vb << 16);
      }
#pragma unroll
      for (int blk = 0; blk < RB; blk++) {
        const uint4 v = make_uint4(wv[4 * blk], wv[4 * blk + 1], wv[4 * blk + 2], wv[4 * blk + 3]);
        if (lane < Q2COMMON) {
#pragma unroll
          for (int p = 0; p < 8; p++)  // copies in a lane-rotated order: fewer bank conflicts
            *(uint4*)(slice + ((lane * RB + blk) * 8 + ((p + lane) & 7)) * 16) = v;
        } else {
          *(uint4*)(slice + Q2Shape<T>::RARE + blk * 128 + (lane - Q2COMMON) * 16) = v;
        }
      }
    }
    __syncwarp();
    uint32_t Hp[T], E[T];
#pragma unroll
    for (int r = 0; r < T; r++) {
      Hp[r] = GO2;   // H(i, 0) = 0
      E[r] = 0u;     // E(i, 1) = -Go
    }
    uint32_t hdiag = GO2;
    const bool last = (s == sp.y - 1);
    // keep-mask of the bottom row: the halves whose query ends here store
    // the empty row above the next query instead (H' = Go, F' = 0)
    const uint32_t keep = (enda ? 0u : 0x0000ffffu) | (endb ? 0u : 0xffff0000u);
    // staging ring as in the packed inter-task kernel; the first strip's
    // border is the row above the matrix, copied from the parameter block
    const uint4* bsrc = s == 0 ? (const uint4*)&P->init_border : bd;
    const int bstep = s == 0 ? 0 : 32;
#pragma unroll
    for (int j = 0; j < Q2RING - 1; j++) {
      if (j < nch) {
#pragma unroll
        for (int q = 0; q < 4; q++)
          cp_async16(bring + ((j % Q2RING) * 4 + q) * 32, bsrc + (j * 4 + q) * bstep);
        cp_async8(rring + (j % Q2RING) * 32, res + j * 64);
      }
      cp_async_commit();
    }
#pragma unroll 1
    for (int c = 0; c < nch; c++) {
      const int cn = c + Q2RING - 1;
      if (cn < nch) {
        const int sl = cn % Q2RING;
#pragma unroll
        for (int q = 0; q < 4; q++)
          cp_async16(bring + (sl * 4 + q) * 32, bsrc + (cn * 4 + q) * bstep);
        cp_async8(rring + sl * 32, res + cn * 64);
      }
      cp_async_commit();
      cp_async_wait<Q2RING - 1>();  // chunk c has landed
      const int slot = c % Q2RING;
      const uint2 rr = rring[slot * 32];
      const uint4 bv[4] = {bring[(slot * 4 + 0) * 32], bring[(slot * 4 + 1) * 32],
                           bring[(slot * 4 + 2) * 32], bring[(slot * 4 + 3) * 32]};
      uint4 ov[4];
      q2_wave<T, 4, 0, G>(Hp, E, hdiag, smax, slice, p16, rr, bv, ov, GO2, NGE2, MGO, one);
      q2_wave<T, 4, 4, G>(Hp, E, hdiag, smax, slice, p16, rr, bv + 2, ov + 2, GO2, NGE2, MGO, one);
      if (!last) {
        if (keep != 0xffffffffu) {  // uniform: some query ends in this strip
#pragma unroll
          for (int q = 0; q < 4; q++) {
            ov[q].x = (ov[q].x & keep) | (GO2 & ~keep);
            ov[q].y &= keep;
            ov[q].z = (ov[q].z & keep) | (GO2 & ~keep);
            ov[q].w &= keep;
          }
        }
#pragma unroll
        for (int q = 0; q < 4; q++) bd[(c * 4 + q) * 32] = ov[q];
      }
    }
    cp_async_wait<0>();
    if (enda) {
      q2_emit(db, P, st, scr, qa, sidx, orig, (int)(int16_t)(smax & 0xffffu));
      smax = (smax & 0xffff0000u) | (GO2 & 0xffffu);
    }
    if (endb) {
      q2_emit(db, P, st, scr, qb, sidx, orig, (int)(int16_t)(smax >> 16));
      smax = (smax & 0x0000ffffu) | (GO2 & 0xffff0000u);
    }
  }
}

template <int T, int G>
__global__ void __launch_bounds__(Q2Shape<T>::WARPS * 32, 1)
inter2q_kernel(DbView db, const SearchParams* __restrict__ P, SearchState* st, Scratch scr) {
  extern __shared__ __align__(16) uint8_t smem[];
  int8_t* sm = (int8_t*)smem;
  load_matrix(sm, P);
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint8_t* slice = smem + MATRIX_SMEM + wib * Q2Shape<T>::BYTES;
  const int64_t warp_id = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
  const int K = P->n_spairs;
  const int64_t total = P->n_inter2_items;
  if (K <= 0 || total <= 0) return;  // uniform over the grid
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(&st->work2, 1ull);
    it = __shfl_sync(FULL, it, 0);
    if ((int64_t)it >= total) break;
    const int64_t gh = (int64_t)it / K;  // group halves, longest groups first
    const int k = (int)((int64_t)it - gh * K);
    q2_item<T, G>(db, P, st, sm, slice, lane, warp_id, scr, k, P->g_first + (int)(gh >> 1),
                  (int)(gh & 1));
  }
}

typedef void (*Inter2qKernel)(DbView, const SearchParams*, SearchState*, Scratch);

// The default strip height (32 rows) is compiled for each gap class; 16
// and 24 rows read the penalties at run time.
static Inter2qKernel pick_inter2q(int rows, int gclass) {
  if (rows == 16) return inter2q_kernel<16, 0>;
  if (rows == 24) return inter2q_kernel<24, 0>;
  if (rows == 32)
    return gclass == 1 ? inter2q_kernel<32, 1> : gclass == 2 ? inter2q_kernel<32, 2>
                                                             : inter2q_kernel<32, 0>;
  return nullptr;
}

size_t inter2q_smem_bytes(int rows, int warps) {
  const int slice = rows == 16 ? Q2Shape<16>::BYTES
                    : rows == 24 ? Q2Shape<24>::BYTES
                                 : Q2Shape<32>::BYTES;
  return (size_t)MATRIX_SMEM + (size_t)warps * slice;
}

int inter2q_warps(int rows) {
  return rows == 16 ? Q2Shape<16>::WARPS : rows == 24 ? Q2Shape<24>::WARPS : Q2Shape<32>::WARPS;
}

int inter2q_blocks_per_sm(int rows, int warps) {
  Inter2qKernel k = pick_inter2q(rows, 0);
  if (!k || warps < 1 || warps > inter2q_warps(rows)) return 0;
  const size_t smem = inter2q_smem_bytes(rows, warps);
  for (int g = 0; g < GAP_CLASSES; g++) {  // every variant the plan may launch
    if (cudaFuncSetAttribute(pick_inter2q(rows, g), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, warps * 32, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

cudaError_t launch_inter2q(const KernelConfig& kc, int gclass, const DbView& db,
                           const SearchParams* params, SearchState* state, const Scratch& scr,
                           cudaStream_t stream) {
  Inter2qKernel k = pick_inter2q(kc.variant, gclass);
  if (!k) return cudaErrorInvalidValue;
  cudaGetLastError();  // a stale error must not be read as this launch's
  k<<<kc.blocks, kc.warps * 32, kc.smem, stream>>>(db, params, state, scr);
  return cudaGetLastError();
}

}  // namespace swgb
