// pair_kernel.cu -- the packed intra-task kernel of libswgb (long subjects).
//
// Two widths, launched one after the other: pair_kernel<16> (16 rows per
// lane, 512-row passes, 16 warps per SM) and pair_kernel<32> (32 rows per
// lane, 1024-row passes, 8 warps per SM).  The wider one halves the per-step
// overhead per cell (shuffles, residue and profile loads, loop control), so
// it is about 15% faster per cell, but pads a query to a multiple of 1024
// rows instead of 512.  The plan gives each query to the width with the
// smaller padded cost (api.cu).
#include <type_traits>

#include "device_common.cuh"

namespace swgb {

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
// quarter 0 loads the profile row of its column (16 bytes per 16 rows) and
// later quarters reuse its words.  Values carry the +Go bias of the inter-task kernel, and a
// pair half whose S' reaches the threshold is recomputed in int32 like any
// other saturated pair.
constexpr int PQ = 4;                      // quarters (independent chains) per lane
constexpr int PHALF = NCODES * 32 * 16;    // int8 [code][lane][16 rows]: one 16-row half
constexpr int PRING = 384;                 // residue ring per subject: 3 blocks of 128

// Warp slice: PR/16 profile halves (each in the conflict-free 16-byte row
// layout of lane_profile<16>), then the two residue rings.
template <int PR>
struct PairShape {
  static_assert(PR == 16 || PR == 32, "16 or 32 rows per lane");
  static constexpr int PQR = PR / PQ;               // rows per quarter
  static constexpr int PROFILE = (PR / 16) * PHALF;
  static constexpr int SLICE = PROFILE + 2 * PRING;
  static constexpr int MIN_BLOCKS = PR == 16 ? 4 : 2;  // 16 or 8 warps per SM
};

template <int PR, int G>
__global__ void __launch_bounds__(PAIR_WARPS * 32, PairShape<PR>::MIN_BLOCKS)
pair_kernel(DbView db, const SearchParams* __restrict__ P, SearchState* st, Scratch scr) {
  constexpr int PQR = PairShape<PR>::PQR;
  constexpr int PAIR_PROFILE = PairShape<PR>::PROFILE;
  constexpr int PAIR_SLICE = PairShape<PR>::SLICE;
  extern __shared__ __align__(16) uint8_t smem[];
  int8_t* sm = (int8_t*)smem;
  load_matrix(sm, P);
  __syncthreads();
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  uint8_t* prof = smem + MATRIX_SMEM + wib * PAIR_SLICE;
  uint8_t* ring0 = prof + PAIR_PROFILE;
  uint8_t* ring1 = ring0 + PRING;
  // Every ring byte holds a residue code (<= PAD_CODE) from here on: slots a
  // lane reads before its first column (the ramp of each pass) then still
  // address a row inside this warp's profile.
  for (int i = lane; i < 2 * PRING; i += 32) ring0[i] = PAD_CODE;
  __syncwarp();
  const int64_t warp_id = (int64_t)blockIdx.x * PAIR_WARPS + wib;
  // the two widths may run at the same time: the wide one has its own rows
  uint2* hb = scr.pair_border + ((PR == 32 ? scr.pair_rows16 : 0) + warp_id) * scr.pair_stride;
  // Items of this width (none when the packed path is off): the wide kernel
  // takes the pairs [0, n_wide_pairs) with the queries qpair[0, nq_pair32);
  // the narrow one takes those pairs with qpair[nq_pair32, nq_pair32 +
  // nq_pair16), then the other pairs with every query (qorder).
  const int npairs = P->pair_queries > 0 ? (P->n_long + 1) / 2 : 0;
  const int nwide = P->n_wide_pairs;
  const int64_t first = (int64_t)nwide * (PR == 32 ? P->nq_pair32 : P->nq_pair16);
  const int64_t total = PR == 32 ? first : first + (int64_t)(npairs - nwide) * P->pair_queries;
  if (total <= 0) return;  // uniform over the grid
  unsigned long long* counter = PR == 32 ? &st->pair_work32 : &st->pair_work;
  const int go = P->go;
  uint32_t GO2, NGE2, MGO;  // (Go, Go), (-Ge, -Ge), -(Go, Go)
  gap_words<G>(P, GO2, NGE2, MGO);
  const uint32_t one = (uint32_t)P->one;
  constexpr int ROWS = 32 * PR;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(counter, 1ull);
    it = __shfl_sync(FULL, it, 0);
    if ((int64_t)it >= total) break;
    int pair, q;
    if ((int64_t)it < first) {
      const int nqw = PR == 32 ? P->nq_pair32 : P->nq_pair16;
      pair = (int)((int64_t)it / nqw);
      q = P->qpair[(PR == 32 ? 0 : P->nq_pair32) + (int)((int64_t)it % nqw)];
    } else {
      const int64_t rest = (int64_t)it - first;
      pair = nwide + (int)(rest / P->pair_queries);
      q = P->qorder[rest % P->pair_queries];
    }
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
      // this lane's PR rows, 16 at a time
      lane_profile<16>(prof, sm, qr, m, p * ROWS + lane * PR, lane);
      if constexpr (PR == 32)
        lane_profile<16>(prof + PHALF, sm, qr, m, p * ROWS + lane * PR + 16, lane);
      load_block(0);
      if constexpr (PR == 32) {
        // the row above the matrix, for the first pass's steady-state steps
        // (lane 0 reads column j at step j; lane 31 rewrites it 127 steps later)
        if (p == 0)
          for (int j = lane; j < n0; j += 32) hb[j] = make_uint2(GO2, 0u);
      }
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
      // (with PR = 32 the second 16-row half in VA2 / VB2)
      uint4 VA[PQ], VB[PQ], VA2[PQ], VB2[PQ];
#pragma unroll
      for (int k = 0; k < PQ; k++) {
        VA[k] = make_uint4(0u, 0u, 0u, 0u);
        VB[k] = make_uint4(0u, 0u, 0u, 0u);
        VA2[k] = make_uint4(0u, 0u, 0u, 0u);
        VB2[k] = make_uint4(0u, 0u, 0u, 0u);
      }
      uint32_t hdiag = GO2, out_h = GO2, out_f = 0u;
      const bool last_pass = (p == npass - 1);
      const int steps = n0 + 32 * PQ - 1;
      // ring position of column t0 - PQ*lane; a multiple of 4, as is PRING
      int pos = (PRING - (PQ * lane) % PRING) % PRING;
      // one step of the wavefront; CHECK: some quarter may lie outside the
      // columns (ramp-up and drain); in the steady state every quarter of
      // every lane is inside, so the step needs no per-quarter test
      // CHECK: some quarter may lie outside the columns (ramp and drain);
      // RING: this step may start a 128-column residue block (the steady
      // state runs whole blocks and refills the ring before each)
      auto step = [&](const int t, auto checked, auto slot, auto ring) {
        constexpr bool CHECK = decltype(checked)::value;
        constexpr int U = decltype(slot)::value;  // t mod 4
        if constexpr (U == 0 && decltype(ring)::value) {
          if ((t & 127) == 0) {
            load_block((t >> 7) + 1);
            __syncwarp();
          }
        }
        uint32_t in_h = __shfl_up_sync(FULL, out_h, 1);
        uint32_t in_f = __shfl_up_sync(FULL, out_f, 1);
        const int c0 = t - PQ * lane;  // quarter 0's column
        if constexpr (PR == 32) {
          // lane 0's top border, column t, from the previous pass (unused on
          // the first): every lane loads the same (clamped, so in bounds)
          // word, so the load is one broadcast and no lane branches; in the
          // steady state t < n0 holds, so neither clamp nor test is needed
          if constexpr (CHECK) {
            const uint2 bv = hb[min(t, n0 - 1)];
            const bool from_scratch = p > 0 && t < n0;
            if (lane == 0) {
              in_h = from_scratch ? bv.x : GO2;  // else H(0, j) = 0
              in_f = from_scratch ? bv.y : 0u;   // else F(1, j) = -Go
            }
          } else {
            // the first pass's row holds (H', F') = (Go, 0) here (filled
            // before the pass), so the value needs no test either
            const uint2 bv = hb[t];
            if (lane == 0) {
              in_h = bv.x;
              in_f = bv.y;
            }
          }
        } else if (lane == 0) {
          if (p > 0 && c0 < n0) {
            const uint2 v = hb[c0];
            in_h = v.x;
            in_f = v.y;
          } else {
            in_h = GO2;  // H(0, j) = 0
            in_f = 0u;   // F(1, j) = -Go
          }
        }
        const int ra = ring0[pos + U];
        const int rb = ring1[pos + U];
        VA[U] = *(const uint4*)(prof + (ra * 32 + lane) * 16);
        VB[U] = *(const uint4*)(prof + (rb * 32 + lane) * 16);
        constexpr int U1 = (U + 3) & 3, U2 = (U + 2) & 3, U3 = (U + 1) & 3;
        // words of quarter k's rows, from the vector loaded k steps ago
        uint32_t wa[PQ][PQR / 4], wb[PQ][PQR / 4];
        if constexpr (PR == 16) {
          wa[0][0] = VA[U].x, wa[1][0] = VA[U1].y, wa[2][0] = VA[U2].z, wa[3][0] = VA[U3].w;
          wb[0][0] = VB[U].x, wb[1][0] = VB[U1].y, wb[2][0] = VB[U2].z, wb[3][0] = VB[U3].w;
        } else {
          VA2[U] = *(const uint4*)(prof + PHALF + (ra * 32 + lane) * 16);
          VB2[U] = *(const uint4*)(prof + PHALF + (rb * 32 + lane) * 16);
          wa[0][0] = VA[U].x, wa[0][1] = VA[U].y, wa[1][0] = VA[U1].z, wa[1][1] = VA[U1].w;
          wa[2][0] = VA2[U2].x, wa[2][1] = VA2[U2].y, wa[3][0] = VA2[U3].z, wa[3][1] = VA2[U3].w;
          wb[0][0] = VB[U].x, wb[0][1] = VB[U].y, wb[1][0] = VB[U1].z, wb[1][1] = VB[U1].w;
          wb[2][0] = VB2[U2].x, wb[2][1] = VB2[U2].y, wb[3][0] = VB2[U3].z, wb[3][1] = VB2[U3].w;
        }
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
              const uint32_t h = packed_cell<G>(hd, prmt(wa[k][i >> 2], wb[k][i >> 2],
                                                      sext_pair_sel(i & 3)), e, f, GO2, NGE2, MGO, one);
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
      auto block = [&](const int t0, auto checked, auto ring) {
        step(t0, checked, std::integral_constant<int, 0>{}, ring);
        step(t0 + 1, checked, std::integral_constant<int, 1>{}, ring);
        step(t0 + 2, checked, std::integral_constant<int, 2>{}, ring);
        step(t0 + 3, checked, std::integral_constant<int, 3>{}, ring);
        pos = pos + 4 == PRING ? 0 : pos + 4;
      };
      // every quarter of every lane is inside the columns for 32*PQ-1 <= t < n0;
      // the last block may run past `steps`, where every quarter is outside
      int t0 = 0;
      for (; t0 < 32 * PQ; t0 += 4) block(t0, std::true_type{}, std::true_type{});
      if constexpr (PR == 32) {
        // steady state in whole 128-column residue blocks (t0 is a multiple
        // of 128 here): refill the ring once, then 32 four-step blocks with
        // no test; the rest (under 128 steady steps, then the drain) runs the
        // checked step, so the step has two instantiations in all
        static_assert(32 * PQ == 128, "the ramp must end on a residue block boundary");
#pragma unroll 1
        for (; t0 + 128 <= n0; t0 += 128) {
          load_block((t0 >> 7) + 1);
          __syncwarp();
#pragma unroll 1
          for (int b = 0; b < 128; b += 4) block(t0 + b, std::false_type{}, std::false_type{});
        }
      } else {
#pragma unroll 1
        for (; t0 + 4 <= n0; t0 += 4) block(t0, std::false_type{}, std::true_type{});
      }
      for (; t0 < steps; t0 += 4) block(t0, std::true_type{}, std::true_type{});
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
          if ((int64_t)k < scr.flag_capacity)
            scr.flags[k] = make_int2(q, sidx);
          else  // the list is full: mark the pair for the host's next recompute round
            P->scores[(int64_t)q * db.n + orig] = FLAG_SENTINEL;
        } else {
          P->scores[(int64_t)q * db.n + orig] = sb - go;
        }
      }
    }
  }
}

size_t pair_smem_bytes(int rows) {
  const int slice = rows == 32 ? PairShape<32>::SLICE : PairShape<16>::SLICE;
  return (size_t)MATRIX_SMEM + (size_t)PAIR_WARPS * slice;
}

typedef void (*PairKernel)(DbView, const SearchParams*, SearchState*, Scratch);

// Both widths are compiled for each gap class.
static PairKernel pick_pair(int rows, int gclass) {
  if (rows == 32)
    return gclass == 1 ? pair_kernel<32, 1> : gclass == 2 ? pair_kernel<32, 2> : pair_kernel<32, 0>;
  if (rows == 16)
    return gclass == 1 ? pair_kernel<16, 1> : gclass == 2 ? pair_kernel<16, 2> : pair_kernel<16, 0>;
  return nullptr;
}

int pair_blocks_per_sm(int rows) {
  if (rows != 16 && rows != 32) return 0;
  PairKernel k = pick_pair(rows, 0);
  const size_t smem = pair_smem_bytes(rows);
  for (int g = 0; g < GAP_CLASSES; g++)  // every variant the plan may launch
    if (cudaFuncSetAttribute(pick_pair(rows, g), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, PAIR_WARPS * 32, smem) != cudaSuccess)
    return 0;
  return nb;
}

cudaError_t launch_pairs(int rows, int gclass, int blocks, const DbView& db,
                         const SearchParams* params, SearchState* state, const Scratch& scr,
                         cudaStream_t stream) {
  PairKernel k = pick_pair(rows, gclass);
  if (!k) return cudaErrorInvalidValue;
  cudaGetLastError();  // a stale error must not be read as this launch's
  k<<<blocks, PAIR_WARPS * 32, pair_smem_bytes(rows), stream>>>(db, params, state, scr);
  return cudaGetLastError();
}

}  // namespace swgb
