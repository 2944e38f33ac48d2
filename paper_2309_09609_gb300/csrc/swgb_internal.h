// swgb_internal.h -- types and helpers shared by the CUDA translation units
// of libswgb.  Nothing here is part of the public ABI (include/swgb.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/swgb.h"

namespace swgb {

// ---- alphabet and layout constants ------------------------------------------
constexpr int ALPHA = 24;        // BLOSUM62 symbols A R N D C Q E G H I L K M F P S T W Y V B Z X *
constexpr int PAD_CODE = 24;     // trailing padding residue (never in user input)
constexpr int NCODES = 25;       // ALPHA + PAD
constexpr int PAD_SCORE = -64;   // SM against PAD: trailing cells scoring <= 0 leave S unchanged
constexpr int GROUP = 64;        // subjects per inter-task group (32 lanes x 2 packed subjects)
constexpr int CHUNK = 8;         // residues per subject per interleaved chunk
constexpr int CHUNK_BYTES = GROUP * CHUNK;  // 512 bytes: one chunk of a whole group
constexpr int S16_LIMIT = 32767;
// Score written for a saturated pair that found the flag list full; no
// exact score is negative, so a later pass can find the pair by it.
constexpr int32_t FLAG_SENTINEL = -1;
// Default capacity of a plan's flag list (saturated pairs per search round).
constexpr int64_t DEFAULT_FLAG_CAPACITY = 1 << 20;

// ---- error reporting ----------------------------------------------------------
sw_status sw_set_error(sw_status st, const char* fmt, ...);
sw_status sw_set_cuda_error(cudaError_t err, const char* where);
void sw_clear_error();

#define CUDA_TRY(call)                                                       \
  do {                                                                       \
    cudaError_t _e = (call);                                                 \
    if (_e != cudaSuccess) return ::swgb::sw_set_cuda_error(_e, #call);      \
  } while (0)

// ---- device-resident database view (passed by value to kernels) -------------
struct DbView {
  const uint8_t* inter;  // interleaved groups: [group][chunk][lane][2 subjects][8 residues]
  const int64_t* goff;   // [G] byte offset of each group in `inter`
  const int32_t* glen;   // [G] group length padded to a multiple of CHUNK
  const uint8_t* cont;   // all subjects, sorted by length (descending), contiguous
  const int64_t* coff;   // [N] offset of sorted subject s in `cont`
  const int32_t* clen;   // [N] length of sorted subject s
  const int32_t* perm;   // [G * GROUP] sorted index -> caller index, -1 for padding slots
  int64_t n;             // subjects
  int32_t groups;        // G
  int32_t max_len;       // longest subject
};

// ---- per-search parameters, read by the kernels from device memory ----------
// Kept in device memory (not kernel arguments) so that one captured CUDA graph
// serves every batch: a new search only rewrites this block.
struct SearchParams {
  uint4 init_border;      // packed (H', F') of the row above the matrix: (Go, 0, Go, 0)
  const uint8_t* qres;    // concatenated query codes
  const int64_t* qoff;    // [nq]
  const int32_t* qlen;    // [nq]
  const int32_t* qorder;  // [nq] query indices, longest first
  const int32_t* qpair;   // [nq_pair32 + nq_pair16] query indices for the pair kernels:
                          // those of pair_kernel<32>, then those of pair_kernel<16>
  int32_t* scores;        // [nq x N] caller order
  // two queries per word (inter2q_kernel.cu): the strip table, per strip
  // (query of half 0, its first row | end bit 31, query of half 1, its first
  // row | end bit 31), query -1 for an empty half; and per stream pair its
  // first strip and strip count
  const int4* strips;
  const int2* spairs;
  int64_t n_inter2_items; // stream pairs x 2 x inter groups (0: the one-query kernel runs)
  // two queries per word for the long subjects (pair2q_kernel.cu): a strip
  // table of 32-row strips and its stream pairs, in the same format
  const int4* strips2;
  const int2* spairs2;
  int64_t n_pair2_items;  // stream pairs x groups of PAIR2_GROUP long subjects (0: pair_kernel runs)
  int64_t n_intra_items;  // n_long x nq  (int32 intra-task items, when the packed path is off)
  int64_t n_inter_items;  // inter groups x nq  (packed inter-task items)
  int32_t nq;
  int32_t n_spairs;       // stream pairs of the two-query kernel
  int32_t n_spairs2;      // stream pairs of the two-query intra-task kernel
  int32_t pair_queries;   // nq when the packed path scores the long subjects, else 0
  int32_t n_wide_pairs;   // subject pairs [0, n_wide_pairs) may go to pair_kernel<32> ...
  int32_t nq_pair32;      // ... with these queries (qpair[0, nq_pair32)); the narrow
  int32_t nq_pair16;      // kernel takes them with the others, and every other pair
  int32_t n_long;         // sorted subjects [0, n_long) go to the intra-task kernels
  int32_t g_first;        // first inter-task group (n_long / GROUP)
  int32_t go;             // Go = gap_open + gap_extend  (Eq. 2-3)
  int32_t ge;             // Ge = gap_extend
  int32_t sat_threshold;  // packed path: S + Go >= this (32767 - max SM) is recomputed in int32
  int32_t one;            // 1, read at run time so multiply-adds stay integer multiply-adds
  int8_t sm[NCODES * NCODES];  // SM(query code, subject code), PAD row/column = PAD_SCORE
};

// ---- per-search device state (zeroed before each search) --------------------
struct SearchState {
  unsigned long long work;        // next work item (inter-task kernel)
  unsigned long long n_flags;     // saturated pairs appended to the flag list
  unsigned long long recompute;   // next flagged pair (int32 intra-task kernel, per block)
  unsigned long long pair_work;   // next work item (pair_kernel<16>)
  unsigned long long pair_work32; // next work item (pair_kernel<32>)
  unsigned long long intra_work;  // next int32 intra-task item (per warp)
  unsigned long long work2;       // next work item (two-query inter-task kernel)
  unsigned long long pair2_work;  // next work item (two-query intra-task kernel, per block)
  unsigned int status;            // reserved: error bits raised on the device
  unsigned int pad;
};

// ---- scratch handed to the kernels --------------------------------------------
struct Scratch {
  uint4* inter_border;        // per warp: [chunk][4][lane] uint4 (H,F words of 2 columns)
  int64_t inter_stride_vec;   // uint4 per warp
  int2* intra_border;         // per warp: [column] (H, F) int32
  int64_t intra_stride;       // int2 per warp
  int2* flags;                // saturated pairs: (query index, sorted subject index)
  int64_t flag_capacity;
  uint2* pair_border;         // packed intra-task kernels, per warp: [column] (H', F') words;
                              // rows [0, pair_rows16) for pair_kernel<16>, the rest for <32>
  int64_t pair_stride;        // uint2 per warp
  int64_t pair_rows16;
};

// ---- gap classes ------------------------------------------------------------------
// The packed kernels are compiled for two common gap settings with the
// penalties as compile-time constants, besides the general form that reads
// them at run time:
//   class 1: gap_open 10, gap_extend 2 (Go = 12, Ge = 2), the paper's "10/2";
//   class 2: gap_open 11, gap_extend 1 (Go = 12, Ge = 1), BLAST's default.
template <int G> struct GapClass;
template <> struct GapClass<1> { static constexpr int GO = 12, GE = 2; };
template <> struct GapClass<2> { static constexpr int GO = 12, GE = 1; };
constexpr int GAP_CLASSES = 3;
inline int gap_class(int go, int ge) {
  if (go == GapClass<1>::GO && ge == GapClass<1>::GE) return 1;
  if (go == GapClass<2>::GO && ge == GapClass<2>::GE) return 2;
  return 0;
}

// ---- kernel launchers -----------------------------------------------------------
struct KernelConfig {
  int variant;     // inter: packed rows per thread (16/32); intra: int32 rows per lane (8/16)
  int cols;        // inter: columns per wavefront (4, or 8 with 32 rows)
  int warps;       // warps per block
  int blocks;      // grid size
  size_t smem;     // dynamic shared memory per block
};

// Inter-task kernel, packed 16-bit (inter_kernel.cu).
size_t inter_smem_bytes(int rows, int warps);
int inter_blocks_per_sm(int rows, int cols, int warps);  // resident blocks per SM, 0 if none
cudaError_t launch_inter(const KernelConfig& kc, int gclass, const DbView& db,
                         const SearchParams* params, SearchState* state, const Scratch& scr,
                         cudaStream_t stream);

// Inter-task kernel with two queries per word (inter2q_kernel.cu), 16, 24 or
// 32 rows per strip.
size_t inter2q_smem_bytes(int rows, int warps);
int inter2q_warps(int rows);  // warps per block (one block per SM)
int inter2q_blocks_per_sm(int rows, int warps);  // resident blocks per SM, 0 if none
cudaError_t launch_inter2q(const KernelConfig& kc, int gclass, const DbView& db,
                           const SearchParams* params, SearchState* state, const Scratch& scr,
                           cudaStream_t stream);

// Int32 intra-task kernel (intra_kernel.cu): int32 items one warp each, then
// flagged pairs one block each.  Scratch: one border row per warp.
constexpr int INTRA_WARPS = 16;  // warps per block
size_t intra_smem_bytes(int rows);
int intra_blocks_per_sm(int rows);
cudaError_t launch_intra(const KernelConfig& kc, const DbView& db, const SearchParams* params,
                         SearchState* state, const Scratch& scr, cudaStream_t stream);

// Flag-list overflow (intra_kernel.cu): appends every pair whose score in
// P->scores is FLAG_SENTINEL to the flag list (up to its capacity, counting
// all of them in state->n_flags), for a further round of the int32 kernel.
cudaError_t launch_collect(int blocks, const DbView& db, const SearchParams* params,
                           SearchState* state, const Scratch& scr, cudaStream_t stream);

// Packed intra-task kernel over subject pairs, long subjects (pair_kernel.cu),
// with 16 or 32 query rows per lane.
constexpr int PAIR_WARPS = 4;  // warps per block
int pair_blocks_per_sm(int rows);
size_t pair_smem_bytes(int rows);
cudaError_t launch_pairs(int rows, int gclass, int blocks, const DbView& db,
                         const SearchParams* params, SearchState* state, const Scratch& scr,
                         cudaStream_t stream);
// Packed intra-task kernel with two queries per word, long subjects
// (pair2q_kernel.cu): one block of pair2q_warps() warps per SM, one subject
// per warp, 32-row strips; scratch: the pair_border rows [0, blocks x warps).
constexpr int PAIR2_STRIP = 32;  // rows per strip of its strip table
constexpr int PAIR2_GROUP = 12;  // subjects per item (the warps of a block)
int pair2q_warps();
size_t pair2q_smem_bytes();
int pair2q_blocks_per_sm();
cudaError_t launch_pair2q(int gclass, int blocks, const DbView& db, const SearchParams* params,
                          SearchState* state, const Scratch& scr, cudaStream_t stream);
// pair_kernel<32> costs about 0.85 of pair_kernel<16> per cell it computes
// but pads a query to 1024-row passes instead of 512: a query of m residues
// goes to the wide kernel when 0.85 * ceil(m / 1024) * 1024 is below
// ceil(m / 512) * 512, i.e. 17 * ceil(m / 1024) < 10 * ceil(m / 512).
inline bool pair_wide(int32_t m) {
  const int64_t a = ((int64_t)m + 1023) / 1024, b = ((int64_t)m + 511) / 512;
  return m > 0 && 17 * a < 10 * b;
}

// Plain int32 baseline (Algorithm 1 per cell), one query per launch (plain_kernel.cu).
int plain_blocks_per_sm();
cudaError_t launch_plain(int blocks, const DbView& db, const SearchParams* params, int query,
                         int2* border, const int64_t* border_off, cudaStream_t stream);

// Optimal local alignments with traceback (align_kernel.cu).
struct AlignItem {
  int32_t q;          // query index (SearchParams::qres / qoff / qlen)
  int32_t s;          // sorted subject index
  int64_t bits_off;   // first uint32 of this pair's direction bits
  int64_t border_off; // first int2 of this pair's pass-border row
  int64_t ops_end;    // the transcript ends just before this byte of the ops buffer
};
struct AlignOut {
  int32_t score;
  int32_t i_end, j_end;      // 1-based cell of the score (0 when it is 0)
  int32_t q_begin, s_begin;  // 0-based first aligned residues
  int32_t n_ops;
  int64_t ops_offset;        // the transcript occupies [ops_offset, ops_offset + n_ops)
};
// uint32 words of direction bits for an m x n pair (4 bits per cell)
int64_t align_bits_words(int32_t m, int32_t n);
// block_mode: one block of 16 warps per pair (border: 16 rows of the subject's
// length per pair), else one warp per pair (one row per pair)
cudaError_t launch_align(const DbView& db, const SearchParams* params, const AlignItem* items,
                         int n_items, bool block_mode, uint32_t* bits, int2* border, AlignOut* out,
                         uint8_t* ops, cudaStream_t stream);
constexpr int ALIGN_BLOCK_ROWS = 16;  // border rows per pair in block mode

// Integer-pipe microbenchmark (intpeak.cu).
int intpeak_run(int op, int blocks_per_sm, int threads, int iters, double* lane_ops_per_clk_sm,
                double* clock_mhz, double* seconds);

}  // namespace swgb
