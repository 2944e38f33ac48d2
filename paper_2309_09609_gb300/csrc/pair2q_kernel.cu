// pair2q_kernel.cu -- the packed intra-task kernel of libswgb with two
// queries per 32-bit word (long subjects).
//
// pair_kernel.cu packs two SUBJECTS into the halves of a word, so every word
// of substitution scores is merged from two profile rows (one byte-permute
// per word).  Here a warp scores ONE long subject, and the halves hold two
// query streams (the layout of inter2q_kernel.cu): the word of rows (a_i,
// b_i) against residue d_j is (SM(a_i, d_j), SM(b_i, d_j)), read ready-made
// from a profile built for the pass.  The cell update is the same biased
// packed update (Eq. 1-3), 4.5 ALU-pipe operations per word instead of 5.5.
//
// Intra-task parallelism (Section II-B): lane k owns one 32-row strip of each
// stream per 1024-row pass, split into four quarters of 8 rows; quarter q of
// lane k updates column t - 4k - q at step t, and lane k's first quarter takes
// the bottom row of lane k - 1 by __shfl_up_sync.  Lane 0 reads the previous
// pass's bottom row from this warp's border scratch, lane 31 writes it.
//
// The strips of a pass are 32 consecutive entries of the strip table (query,
// first row, end bit per half), so a query boundary may fall between any two
// lanes (or passes).  A lane whose strip starts a query in a half replaces
// that half of its top border by the empty row above the matrix (H = 0,
// F = -Go).  At the end of a pass the warp takes, per half, a segmented
// maximum of S' over the lanes of each query (with the maximum carried from
// the previous pass), and the lane holding a query's last strip emits the
// score.
//
// The profile of a pass is shared by the block: its PAIR2_GROUP (12) warps
// score as many adjacent subjects of the length order (nearly equal lengths)
// against the same stream pair, pass by pass.  Item = (stream pair, group of
// PAIR2_GROUP long subjects), longest groups first, from an atomic counter.
// Twelve warps per SM (168 registers each) ran the long-sequence workload
// 9% faster than eight (206 registers): three warps per scheduler hide more
// of the cell chain's latency.
#include <type_traits>

#include "device_common.cuh"

namespace swgb {

constexpr int P2_WARPS = PAIR2_GROUP;                // warps per block (one subject each), one block per SM
static_assert(PAIR2_STRIP == 32, "a lane owns one 32-row strip");
constexpr int P2_QUARTERS = 4;                       // independent chains per lane
constexpr int P2_LANE_BYTES = 144;                   // a lane's 32 words + 16 bytes of skew
constexpr int P2_CODE_BYTES = 32 * P2_LANE_BYTES;    // one code's rows for the 32 lanes
constexpr int P2_PROFILE = NCODES * P2_CODE_BYTES;   // 115,200 bytes
constexpr int P2_RING = 384;                         // residue ring: 3 blocks of 128 columns
constexpr int P2_SMEM = MATRIX_SMEM + P2_PROFILE + P2_WARPS * P2_RING + 16;

// Profile of a pass: word (code c, lane l, row r of l's strip) at
//   c * P2_CODE_BYTES + l * P2_LANE_BYTES + 4 * r.
// A lane's 8-row quarter is two 16-byte reads at the same offsets for every
// lane; the 144-byte lane stride puts the 8 lanes of a quarter-warp on 8
// distinct bank groups whatever codes they read.  Built by the whole block:
// thread (l, c0) writes the rows of lane l for codes c0, c0 + 8, ...
__device__ __forceinline__ void p2_profile(uint8_t* prof, const int8_t* __restrict__ sm,
                                           const SearchParams* __restrict__ P, int2 sp, int pass) {
  const int l = threadIdx.x & 31;
  int qa = -1, qb = -1, ia = 0, ib = 0;
  if (32 * pass + l < sp.y) {
    const int4 si = P->strips2[sp.x + 32 * pass + l];
    qa = si.x;
    ia = si.y & 0x7fffffff;
    qb = si.z;
    ib = si.w & 0x7fffffff;
  }
  const uint8_t* __restrict__ ra = qa >= 0 ? P->qres + P->qoff[qa] + ia : nullptr;
  const uint8_t* __restrict__ rb = qb >= 0 ? P->qres + P->qoff[qb] + ib : nullptr;
  const int na = qa >= 0 ? P->qlen[qa] - ia : 0, nb = qb >= 0 ? P->qlen[qb] - ib : 0;
  // the strip's codes, four to a word (the padding code past a query's end)
  uint32_t ca[8], cb[8];
#pragma unroll
  for (int w = 0; w < 8; w++) {
    uint32_t x = 0, y = 0;
#pragma unroll
    for (int b = 0; b < 4; b++) {
      const int r = 4 * w + b;
      x |= (uint32_t)(r < na ? ra[r] : PAD_CODE) << (8 * b);
      y |= (uint32_t)(r < nb ? rb[r] : PAD_CODE) << (8 * b);
    }
    ca[w] = x;
    cb[w] = y;
  }
  for (int c = threadIdx.x >> 5; c < NCODES; c += P2_WARPS) {
    uint8_t* dst = prof + c * P2_CODE_BYTES + l * P2_LANE_BYTES;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      uint32_t v[4];
#pragma unroll
      for (int b = 0; b < 4; b++) {
        const int xa = (ca[j] >> (8 * b)) & 0xff, xb = (cb[j] >> (8 * b)) & 0xff;
        v[b] = (uint32_t)(uint16_t)(int16_t)sm[xa * NCODES + c] |
               ((uint32_t)(uint16_t)(int16_t)sm[xb * NCODES + c] << 16);
      }
      *(uint4*)(dst + 16 * j) = make_uint4(v[0], v[1], v[2], v[3]);
    }
  }
}

// The 16-bit S' of one half (biased by +Go): recorded, or flagged for the
// int32 recompute when it may have saturated, as the score of (query q,
// sorted subject sidx).
__device__ __forceinline__ void p2_emit(const DbView& db, const SearchParams* __restrict__ P,
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

// Inclusive maximum of v over the lanes at or below this one that carry the
// same key (a query's strips occupy consecutive lanes).
__device__ __forceinline__ int p2_segmax(int key, int v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int ko = __shfl_up_sync(FULL, key, d);
    const int vo = __shfl_up_sync(FULL, v, d);
    if (lane >= d && ko == key) v = max(v, vo);
  }
  return v;
}

template <int G>
__global__ void __launch_bounds__(P2_WARPS * 32, 1)
pair2q_kernel(DbView db, const SearchParams* __restrict__ P, SearchState* st, Scratch scr) {
  constexpr int PQ = P2_QUARTERS;
  extern __shared__ __align__(16) uint8_t smem[];
  const int K = P->n_spairs2;
  const int64_t total = P->n_pair2_items;
  if (K <= 0 || total <= 0) return;  // uniform over the grid
  int8_t* sm = (int8_t*)smem;
  uint8_t* prof = smem + MATRIX_SMEM;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint8_t* ring = prof + P2_PROFILE + wib * P2_RING;
  unsigned long long* s_item = (unsigned long long*)(prof + P2_PROFILE + P2_WARPS * P2_RING);
  load_matrix(sm, P);
  // Every ring byte holds a residue code (<= PAD_CODE) from here on: slots a
  // lane reads before its first column (the ramp of each pass) then still
  // address a row of the profile.
  for (int i = lane; i < P2_RING; i += 32) ring[i] = PAD_CODE;
  __syncthreads();
  uint2* hb = scr.pair_border + ((int64_t)blockIdx.x * P2_WARPS + wib) * scr.pair_stride;
  uint32_t GO2, NGE2, MGO;  // (Go, Go), (-Ge, -Ge), -(Go, Go)
  gap_words<G>(P, GO2, NGE2, MGO);
  const uint32_t one = (uint32_t)P->one;
  const uint32_t lane_off = (uint32_t)(lane * P2_LANE_BYTES);
  // lane 0 takes its top border from the scratch row, the others from the
  // lane above: x * is0 + y * not0 picks one word exactly (a product by 0 or
  // 1), as two multiply-adds on the FMA pipe instead of a select on the
  // busier ALU pipe
  const uint32_t is0 = lane == 0 ? 1u : 0u, not0 = 1u - is0;
  for (;;) {
    if (threadIdx.x == 0) *s_item = atomicAdd(&st->pair2_work, 1ull);
    __syncthreads();
    const unsigned long long it = *s_item;
    __syncthreads();  // read by all before thread 0 writes the next item
    if ((int64_t)it >= total) break;  // uniform over the block
    const int g = (int)((int64_t)it / K);  // subject group, longest first
    const int k = (int)((int64_t)it - (int64_t)g * K);
    const int2 sp = P->spairs2[k];  // (first strip, strips) of this stream pair
    const int sidx = g * P2_WARPS + wib;
    const bool has = sidx < P->n_long;
    const int n = has ? db.clen[sidx] : 0;
    const uint8_t* __restrict__ d = db.cont + (has ? db.coff[sidx] : 0);
    const int orig = has ? db.perm[sidx] : -1;
    const int npass = (sp.y + 31) / 32;
    // residues of columns [128 b, 128 b + 128) into ring slot b % 3 (pad past the end)
    auto load_block = [&](int b) {
      const int c = 128 * b + 4 * lane;
      uint32_t w = 0;
#pragma unroll
      for (int i = 0; i < 4; i++) w |= (uint32_t)(c + i < n ? d[c + i] : PAD_CODE) << (8 * i);
      *(uint32_t*)(ring + c % P2_RING) = w;
    };
    uint32_t carry = GO2;  // per half: S' so far of the query that continues into the next pass
    for (int p = 0; p < npass; p++) {
      __syncthreads();  // every warp is done with the previous pass's profile
      p2_profile(prof, sm, P, sp, p);
      // this lane's strip
      int qa = -1, qb = -1;
      bool enda = false, endb = false;
      uint32_t keep = 0u;  // halves whose strip continues the query of the lane above
      if (32 * p + lane < sp.y) {
        const int4 si = P->strips2[sp.x + 32 * p + lane];
        qa = si.x;
        qb = si.z;
        enda = qa >= 0 && si.y < 0;
        endb = qb >= 0 && si.w < 0;
        if (qa >= 0 && (si.y & 0x7fffffff) != 0) keep |= 0x0000ffffu;
        if (qb >= 0 && (si.w & 0x7fffffff) != 0) keep |= 0xffff0000u;
      }
      const uint32_t gtop = GO2 & ~keep;  // (H', F') = (Go, 0) where a query starts
      if (n > 0) load_block(0);
      __syncthreads();
      uint32_t smax = GO2;
      if (n > 0) {  // uniform over the warp
        uint32_t Hp[32], E[32];
#pragma unroll
        for (int r = 0; r < 32; r++) {
          Hp[r] = GO2;  // H(i, 0) = 0
          E[r] = 0u;    // E(i, 1) = -Go
        }
        // quarter q's bottom-row H' one and two steps back, its F' one step back
        uint32_t qh1[PQ], qh2[PQ], qf1[PQ];
        // profile offset of the code read at each of the last four steps (slot
        // t mod 4): quarter q at step t scores the column read at step t - q
        uint32_t A[PQ];
#pragma unroll
        for (int q = 0; q < PQ; q++) {
          qh1[q] = GO2;
          qh2[q] = GO2;
          qf1[q] = 0u;
          A[q] = lane_off;
        }
        uint32_t hdiag = GO2, out_h = GO2, out_f = 0u;
        // steady state: lane 0's border of columns t .. t + 3, slot t mod 4
        uint2 bq[4] = {make_uint2(0u, 0u), make_uint2(0u, 0u), make_uint2(0u, 0u),
                       make_uint2(0u, 0u)};
        const bool last_pass = (p == npass - 1);
        const int steps = n + 32 * PQ - 1;
        // ring position of column t0 - PQ*lane; a multiple of 4, as is P2_RING
        int pos = (P2_RING - (PQ * lane) % P2_RING) % P2_RING;
        // one step of the wavefront.  CHECK: some quarter may lie outside the
        // columns (ramp and drain); RING: this step may start a 128-column
        // residue block (the steady state refills the ring before each block)
        // MASK: some lane's strip starts a query (the steady state of a pass
        // in which none does leaves the top borders as they come)
        auto step = [&](const int t, auto checked, auto slot, auto ringed, auto masked) {
          constexpr bool CHECK = decltype(checked)::value;
          constexpr int U = decltype(slot)::value;  // t mod 4
          if constexpr (U == 0 && decltype(ringed)::value) {
            if ((t & 127) == 0) {
              load_block((t >> 7) + 1);
              __syncwarp();
            }
          }
          uint32_t in_h = __shfl_up_sync(FULL, out_h, 1);
          uint32_t in_f = __shfl_up_sync(FULL, out_f, 1);
          // lane 0's top border, column t, from the previous pass: every lane
          // loads the same word (one broadcast, no branch).  In the steady
          // state it was loaded four steps earlier (its column is rewritten by
          // lane 31 only 127 steps after lane 0 reads it), and this step loads
          // column t + 4: t < n there, and the border rows have 4 columns of
          // slack past the longest subject
          uint2 bv;
          if constexpr (CHECK) {
            bv = hb[min(t, n - 1)];
          } else {
            bv = bq[U];
            bq[U] = hb[t + 4];
          }
          in_h = imad(bv.x, is0, imad(in_h, not0, 0u));
          in_f = imad(bv.y, is0, imad(in_f, not0, 0u));
          if constexpr (decltype(masked)::value) {
            in_h = (in_h & keep) | gtop;  // H(0, j) = 0 above a query's first row
            in_f &= keep;                 // F(1, j) = -Go
          }
          const int c0 = t - PQ * lane;  // quarter 0's column
          A[U] = lane_off + (uint32_t)ring[pos + U] * P2_CODE_BYTES;
          uint32_t nh[PQ], nf[PQ];
#pragma unroll
          for (int q = 0; q < PQ; q++) {
            const int col = c0 - q;
            bool active = true;
            if constexpr (CHECK) active = col >= 0 && col < n;
            nh[q] = qh1[q];
            nf[q] = qf1[q];
            if (active) {
              const uint8_t* pw = prof + A[(U - q) & 3] + 32 * q;
              const uint4 w0 = *(const uint4*)pw;
              const uint4 w1 = *(const uint4*)(pw + 16);
              const uint32_t w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
              uint32_t hd = q == 0 ? hdiag : qh2[q - 1];  // H' one row up, one column back
              uint32_t f = q == 0 ? in_f : qf1[q - 1];    // F' of this quarter's first row
              uint32_t hprev = 0;
#pragma unroll
              for (int i = 0; i < 8; i++) {
                const int r = 8 * q + i;
                uint32_t e = E[r];
                const uint32_t h = packed_cell<G>(hd, w[i], e, f, GO2, NGE2, MGO, one);
                hd = Hp[r];
                Hp[r] = h;
                E[r] = e;
                if (i & 1)
                  smax = __vimax3_s16x2(smax, hprev, h);
                else
                  hprev = h;
              }
              nh[q] = Hp[8 * q + 7];
              nf[q] = f;
              if (q == PQ - 1 && lane == 31 && !last_pass) hb[col] = make_uint2(nh[q], f);
            } else if (col < 0) {
              nh[q] = GO2;  // left of the matrix: H = 0
            }
          }
          hdiag = in_h;
          out_h = nh[PQ - 1];
          out_f = nf[PQ - 1];
#pragma unroll
          for (int q = 0; q < PQ; q++) {
            qh2[q] = qh1[q];
            qh1[q] = nh[q];
            qf1[q] = nf[q];
          }
        };
        auto block = [&](const int t0, auto checked, auto ringed, auto masked) {
          step(t0, checked, std::integral_constant<int, 0>{}, ringed, masked);
          step(t0 + 1, checked, std::integral_constant<int, 1>{}, ringed, masked);
          step(t0 + 2, checked, std::integral_constant<int, 2>{}, ringed, masked);
          step(t0 + 3, checked, std::integral_constant<int, 3>{}, ringed, masked);
          pos = pos + 4 == P2_RING ? 0 : pos + 4;
        };
        // ramp (every lane's quarters enter), steady state in whole 128-column
        // residue blocks with no test (every quarter of every lane is inside
        // the columns for 127 <= t < n), then the rest and the drain; the last
        // block may run past `steps`, where every quarter is outside
        static_assert(32 * PQ == 128, "the ramp must end on a residue block boundary");
        int t0 = 0;
        for (; t0 < 32 * PQ; t0 += 4)
          block(t0, std::true_type{}, std::true_type{}, std::true_type{});
        if (t0 + 128 <= n) {  // the first steady block's first four border words
#pragma unroll
          for (int u = 0; u < 4; u++) bq[u] = hb[t0 + u];
        }
        // no lane's strip starts a query in most passes of long streams
        const bool any_start = __any_sync(FULL, keep != 0xffffffffu);
#pragma unroll 1
        for (; t0 + 128 <= n; t0 += 128) {
          load_block((t0 >> 7) + 1);
          __syncwarp();
          if (any_start) {
#pragma unroll 1
            for (int b = 0; b < 128; b += 4)
              block(t0 + b, std::false_type{}, std::false_type{}, std::true_type{});
          } else {
#pragma unroll 1
            for (int b = 0; b < 128; b += 4)
              block(t0 + b, std::false_type{}, std::false_type{}, std::false_type{});
          }
        }
        for (; t0 < steps; t0 += 4)
          block(t0, std::true_type{}, std::true_type{}, std::true_type{});
      }
      // S' of each query over its lanes of this pass (and the previous passes)
      int va = (int)(int16_t)(smax & 0xffffu), vb = (int)(int16_t)(smax >> 16);
      if (lane == 0) {
        if (keep & 0x0000ffffu) va = max(va, (int)(int16_t)(carry & 0xffffu));
        if (keep & 0xffff0000u) vb = max(vb, (int)(int16_t)(carry >> 16));
      }
      va = p2_segmax(qa, va, lane);
      vb = p2_segmax(qb, vb, lane);
      if (has) {
        if (enda) p2_emit(db, P, st, scr, qa, sidx, orig, va);
        if (endb) p2_emit(db, P, st, scr, qb, sidx, orig, vb);
      }
      // what lane 31's queries carry into the next pass (nothing past an end)
      const int ca = __shfl_sync(FULL, (enda || qa < 0) ? (int)(int16_t)(GO2 & 0xffffu) : va, 31);
      const int cb = __shfl_sync(FULL, (endb || qb < 0) ? (int)(int16_t)(GO2 >> 16) : vb, 31);
      carry = (uint32_t)(uint16_t)(int16_t)ca | ((uint32_t)(uint16_t)(int16_t)cb << 16);
    }
  }
}

size_t pair2q_smem_bytes() { return (size_t)P2_SMEM; }
int pair2q_warps() { return P2_WARPS; }

typedef void (*Pair2qKernel)(DbView, const SearchParams*, SearchState*, Scratch);

static Pair2qKernel pick_pair2q(int gclass) {
  return gclass == 1 ? pair2q_kernel<1> : gclass == 2 ? pair2q_kernel<2> : pair2q_kernel<0>;
}

int pair2q_blocks_per_sm() {
  for (int g = 0; g < GAP_CLASSES; g++) {  // every variant the plan may launch
    if (cudaFuncSetAttribute(pick_pair2q(g), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             P2_SMEM) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pick_pair2q(0), P2_WARPS * 32,
                                                    (size_t)P2_SMEM) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

cudaError_t launch_pair2q(int gclass, int blocks, const DbView& db, const SearchParams* params,
                          SearchState* state, const Scratch& scr, cudaStream_t stream) {
  cudaGetLastError();  // a stale error must not be read as this launch's
  pick_pair2q(gclass)<<<blocks, P2_WARPS * 32, P2_SMEM, stream>>>(db, params, state, scr);
  return cudaGetLastError();
}

}  // namespace swgb
