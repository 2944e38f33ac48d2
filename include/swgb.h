/*
 * swgb.h -- C ABI of libswgb: exact Smith-Waterman/Gotoh protein database
 * search on one NVIDIA GB300 (sm_103a).
 *
 * The library computes, for every (query, subject) pair, the optimal local
 * alignment score of arxiv 2309.09609, Section II-B, Eq. 1-3:
 *
 *   H(i,j) = max(0, H(i-1,j-1) + SM(Q[i], D[j]), E(i,j), F(i,j))
 *   E(i,j) = max(H(i,j-1) - Go, E(i,j-1) - Ge)
 *   F(i,j) = max(H(i-1,j) - Go, F(i-1,j) - Ge)
 *   score  = max over all cells of H  (H is 0 on row and column 0)
 *
 * in integer arithmetic, exactly (bit for bit) -- the database search of
 * Section III-A with BLOSUM62 and integer scores (Section IV-A).
 *
 * Conventions shared by every call:
 *   - Residues are codes 0..23 in the BLOSUM62 order
 *     A R N D C Q E G H I L K M F P S T W Y V B Z X *  (sw_encode maps text).
 *   - Gaps: (gap_open, gap_extend) with a gap of k residues costing
 *     gap_open + k * gap_extend, i.e. Go = gap_open + gap_extend and
 *     Ge = gap_extend in Eq. 2-3.  Both must be >= 0.  The paper's "10/2"
 *     (Section IV-A) is gap_open = 10, gap_extend = 2 here.
 *   - matrix: 24 x 24 int8, row-major, matrix[a * 24 + b] = SM(a, b) with a the
 *     query residue and b the subject residue; NULL selects BLOSUM62.
 *   - scores: int32, n_queries x n_subjects, row-major, subjects in the order
 *     given to sw_db_create.  Zero-length sequences score 0.
 *   - Pointers may be host or device memory unless stated; the library
 *     detects which.  Inputs are borrowed for the duration of the call only.
 *   - Every call returns a status; on failure sw_last_error() describes it.
 *     No call aborts the process, traps on the device or waits unboundedly.
 *   - Testing hook: with the environment variable SWGB_FAULT=alloc the device
 *     allocations of sw_db_create and sw_plan_create fail with SW_ENOMEM, and
 *     with SWGB_FAULT=copy a search's first copy fails with SW_ECUDA (read at
 *     every call; unset in normal use).
 */
#ifndef SWGB_H
#define SWGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SW_OK = 0,
  SW_EINVAL = 1,     /* bad argument: residue code >= 24, negative length, NULL ... */
  SW_ENOMEM = 2,     /* device or host allocation failed */
  SW_ECUDA = 3,      /* a CUDA runtime call failed */
  SW_ETIMEDOUT = 4,  /* sw_plan_wait: the search is still running when its host-side
                        time limit is up (no kernel of the library waits on the device) */
  SW_EBUSY = 5       /* the plan's capacity is exceeded or it is in use */
} sw_status;

/* Opaque handle: a protein database resident in device memory. */
typedef struct sw_db sw_db;

/* Opaque handle: a reusable search context (device buffers + CUDA graph). */
typedef struct sw_plan sw_plan;

/* Thread-local text of the last error on this thread ("" if none). */
const char* sw_last_error(void);

/* Maps n ASCII letters to residue codes (Section IV-A scores with BLOSUM62,
 * whose 24 symbols define the alphabet).  Lower case is folded; U, O, J and
 * any other byte map to X (code 22).  text and out are host memory. */
sw_status sw_encode(const char* text, int64_t n, uint8_t* out);

/* Copies the library's built-in BLOSUM62 (24 x 24 int8, row-major) to out
 * (host memory, 576 bytes). */
void sw_default_matrix(int8_t* out);

/* Builds the device database (Section III-A: the database is split by
 * length into an inter-task part of short subjects and an intra-task part of
 * long ones).
 *   residues: concatenated codes of all subjects, sum(lengths) bytes, host.
 *   lengths:  n_subjects int32 lengths (>= 0), host.
 *   device:   CUDA device ordinal.
 * The subjects are sorted by length and laid out twice on the device: in
 * groups of 64 subjects interleaved 8 residues at a time (inter-task kernel)
 * and contiguously (pair, int32 intra-task and alignment kernels).  Inputs are copied;
 * the handle owns all device memory until sw_db_destroy.
 * Errors: SW_EINVAL for a code >= 24, a negative length or n_subjects < 0;
 * SW_ENOMEM; SW_ECUDA. */
sw_status sw_db_create(const uint8_t* residues, const int32_t* lengths, int64_t n_subjects,
                       int device, sw_db** out);

/* Frees the database.  NULL-safe.  No plan of this database may be used after. */
void sw_db_destroy(sw_db* db);

/* Number of subjects / residues / the longest subject length. */
int64_t sw_db_subjects(const sw_db* db);
int64_t sw_db_residues(const sw_db* db);
int32_t sw_db_max_length(const sw_db* db);

/* Tuning of the exact search; every field has a safe default (zero-init and
 * call sw_options_default).  None of them changes a score. */
typedef struct {
  int32_t rows_per_thread;   /* query rows per thread in the packed inter-task kernel: 16 or 32 */
  int32_t warps_per_block;   /* 4 or 8 */
  int32_t long_cutoff;       /* subjects longer than this use the intra-task kernel */
  int32_t intra_rows;        /* query rows per lane in the int32 intra-task kernel: 8 or 16 */
  int32_t use_graph;         /* 1: capture the launch sequence in a CUDA graph */
  int32_t force_int32;       /* 1: all subjects through the int32 intra-task kernel */
  int32_t auto_cutoff;       /* 1: per search of >= 1e10 cells, also send to the intra-task
                                kernel every group whose (query, group) work item would
                                exceed a quarter of one warp's share of the search (load
                                balance for few long queries); default 0 */
  int32_t wide_min_len;      /* long subjects are scored 32 query rows per lane (1024-row
                                passes, fewer instructions per cell, half the warps) instead
                                of 16 (512-row passes) for queries of at least this many
                                residues whose padded cost is lower that way ... default 0 */
  int32_t wide_min_subject;  /* ... against subject pairs whose longer subject has at least
                                this many residues, or against every pair when the search
                                has fewer (pair, query) items than 16-row warps; default 4096 */
  int32_t inter_columns;     /* subject columns per wavefront in the packed inter-task kernel
                                with rows_per_thread 32: 4 or 8 (16 rows always use 4);
                                default 8 */
  int32_t overlap_kernels;   /* 1: the inter-task kernel runs alongside the pair kernels
                                instead of after them, so its blocks take the SMs that their
                                tails leave (lower latency for small searches); search_ms and
                                pair_ms then overlap, both from the start; default 0 */
  int32_t two_query;         /* inter-task scoring with two queries per 32-bit word against one
                                subject per lane (no per-cell byte merge, 4.5 instead of 5.5
                                ALU operations per word): 0 never, 1 when the plan's cost
                                model expects it to be faster (default), 2 whenever a search
                                has at least two queries */
  int32_t two_query_rows;    /* query rows per strip of that kernel: 16, 24 or 32 (default) */
  int32_t two_query_pairs;   /* stream pairs of the two-query layouts, inter- and intra-task
                                (0: the plan's choice, per layout; otherwise at most
                                n_queries / 2) */
  int32_t flag_capacity;     /* entries of the plan's list of saturated pairs (8 bytes each);
                                0: min(max_queries x subjects, 2^20).  More saturated pairs
                                than this in one search are still scored exactly, in further
                                rounds of the int32 kernel after the search (see
                                sw_stats.overflow_rounds) */
  int32_t two_query_long;    /* intra-task scoring of the long subjects with two queries per
                                32-bit word against one subject per warp (no per-cell byte
                                merge): 0 never, 1 when the plan's cost model expects it to be
                                faster (default), 2 whenever a search has at least two queries */
} sw_options;

void sw_options_default(sw_options* opt);

/* Statistics of the last search run through a plan. */
typedef struct {
  int64_t cells;             /* sum(query lengths) * sum(subject lengths) */
  int64_t inter_items;       /* (query, group of 64 subjects) work items of the two-subject
                                inter-task kernel (0 when the two-query kernel ran) */
  int64_t intra_items;       /* (query, long subject) work items */
  int64_t recomputed_pairs;  /* pairs whose 16-bit score saturated, redone in int32 */
  int32_t overflow_rounds;   /* extra rounds of the int32 kernel that the last search ran
                                because it had more saturated pairs than the plan's flag list
                                holds (0 normally); their time is not in recompute_ms */
  int32_t kernels_launched;  /* kernels of this library launched by the search */
  float search_ms;           /* device time of the inter-task search kernel (CUDA events) */
  float recompute_ms;        /* device time of the int32 intra-task kernel (CUDA events):
                                the recompute of saturated pairs, or every pair when the
                                packed path is off */
  float pair_ms;             /* device time of the packed intra-task kernels, both widths,
                                from their fork to their join (CUDA events) */
  int32_t pad_;
  int64_t inter_cells;       /* cells scored by the inter-task kernel */
  int64_t inter2_items;      /* (stream pair, half group) items of the two-query inter-task
                                kernel; 0 when the one-query kernel scored the short subjects */
  int64_t pair2_items;       /* (stream pair, group of 12 long subjects) items of the two-query
                                intra-task kernel; 0 when the subject-pair kernels scored the
                                long subjects */
} sw_stats;

/* Creates a search context for up to max_queries queries holding up to
 * max_query_residues residues in total, on the database's device.  The
 * device memory a search needs is allocated here, once: the query buffers,
 * the per-warp border scratch of each kernel (a fixed amount for the device
 * and database, about 2.2 GB on a GB300 for a database whose longest subject
 * has 35,000 residues, independent of the queries), the saturated-pair list
 * (opt.flag_capacity entries of 8 bytes, 8 MiB by default) and the work
 * counters.  One more buffer, max_queries x subjects int32, is allocated by
 * the first search whose scores go to host memory, and kept.  opt may be
 * NULL.
 * Errors: SW_EINVAL, SW_ENOMEM, SW_ECUDA. */
sw_status sw_plan_create(sw_db* db, int32_t max_queries, int64_t max_query_residues,
                         const sw_options* opt, sw_plan** out);

void sw_plan_destroy(sw_plan* plan);

/* Exact scores of every query against every subject (Eq. 1-3), the batched
 * path: six persistent launches, each taking its work longest first from its
 * own atomic counter.  First, for the subjects longer than opt.long_cutoff,
 * one of two packed intra-task layouts: two queries per 32-bit word against
 * one subject per warp, over (pair of query streams, group of 12 subjects)
 * items; or two subjects per word, over (pair of subjects, query) items, at
 * 32 and at 16 query rows per lane, two launches side by side on two streams
 * (opt.wide_min_len and opt.wide_min_subject split the items between them).
 * Then one of two packed inter-task layouts for the other subjects: two
 * queries per word against one subject per lane, over (pair of query
 * streams, half of a group of 64 subjects) items, or two subjects per word,
 * over (query, group of 64 subjects) items.  opt.two_query_long and
 * opt.two_query with a cost model choose each layout per search; a single
 * query always takes the two-subject ones; the kernels of the other layout
 * find no items.  Last the int32 intra-task kernel recomputes every pair
 * whose 16-bit score may have saturated (one block per pair; more saturated
 * pairs than opt.flag_capacity are recomputed in further rounds before the
 * call returns).  With gap penalties too large for 16 bits, or
 * opt.force_int32, every pair goes to the int32 kernel instead (one warp per
 * pair).  The packed kernels are compiled with the gap penalties as
 * constants for (10, 2) and (11, 1), and read them at run time otherwise.
 * The launch sequence is replayed from a CUDA graph (one per such gap
 * setting) when opt.use_graph is set.
 *   queries:   concatenated query codes (sum(q_lengths) bytes), host or device.
 *   q_lengths: n_queries int32, host or device.
 *   scores:    n_queries x n_subjects int32, host or device, written in full.
 *   stream:    cudaStream_t to run on (NULL: the legacy default stream).
 * The call returns after the scores are in `scores` (it synchronises the
 * stream).  One plan serves one call at a time (SW_EBUSY otherwise).
 * Errors: SW_EINVAL (bad code, length, gap or size), SW_EBUSY (capacity),
 * SW_ECUDA. */
sw_status sw_plan_search(sw_plan* plan, const uint8_t* queries, const int32_t* q_lengths,
                         int32_t n_queries, int32_t gap_open, int32_t gap_extend,
                         const int8_t* matrix, int32_t* scores, void* stream);

/* Like sw_plan_search but returns as soon as the work is queued on the
 * stream; queries/q_lengths must be host memory (copied before return) and
 * scores device memory; completion is observed with sw_plan_wait or any CUDA
 * stream/event query.  Used by the serving loop to overlap requests. */
sw_status sw_plan_search_async(sw_plan* plan, const uint8_t* queries, const int32_t* q_lengths,
                               int32_t n_queries, int32_t gap_open, int32_t gap_extend,
                               const int8_t* matrix, int32_t* scores, void* stream);

/* Waits for the plan's last asynchronous search, at most timeout_ms
 * milliseconds (0: only poll; negative: no bound); SW_ETIMEDOUT if it is
 * still running when the time is up. */
sw_status sw_plan_wait(sw_plan* plan, int32_t timeout_ms);

/* Statistics of the plan's last completed search. */
sw_status sw_plan_stats(const sw_plan* plan, sw_stats* out);

/* One-shot exact search: sw_plan_search through a plan that the database
 * keeps for these calls.  The first call creates it (default options, sized
 * for its batch), later calls reuse it, and a batch larger than it holds
 * replaces it with one sized for both; it is freed by sw_db_destroy.  Calls
 * on one database are serialized (they would share the GPU anyway).  Same
 * arguments and errors as sw_plan_search. */
sw_status sw_search(sw_db* db, const uint8_t* queries, const int32_t* q_lengths,
                    int32_t n_queries, int32_t gap_open, int32_t gap_extend,
                    const int8_t* matrix, int32_t* scores, void* stream);

/* The plain baseline of Algorithm 1: int32 cells, one thread per subject,
 * one kernel launch per query, no packing, no long-subject kernel.  Same
 * arguments, result and errors as sw_search. */
sw_status sw_search_plain(sw_db* db, const uint8_t* queries, const int32_t* q_lengths,
                          int32_t n_queries, int32_t gap_open, int32_t gap_extend,
                          const int8_t* matrix, int32_t* scores, void* stream);

/* One optimal local alignment (sw_align). */
typedef struct {
  int32_t score;             /* S, as sw_search returns it */
  int32_t q_begin, q_end;    /* aligned query residues [q_begin, q_end), 0-based */
  int32_t s_begin, s_end;    /* aligned subject residues [s_begin, s_end), 0-based */
  int32_t n_ops;             /* transcript length; 0 when score is 0 */
  int64_t ops_offset;        /* the transcript is ops[ops_offset, ops_offset + n_ops) */
} sw_alignment;

/* Optimal local alignments, with traceback, of selected (query, subject)
 * pairs: the alignment behind each score, recovered by the traceback of
 * Section II-B (the score kernels keep only S).  For pair k, query
 * pair_query[k] (an index into queries / q_lengths) against database
 * subject pair_subject[k] (caller order).
 * Which of several optimal alignments is returned: the one ending at the
 * first cell in row-major order (query position, then subject position)
 * whose H equals S; walking back, the diagonal term is preferred to E, and E
 * to F, when they tie, and a gap opens from H when that reaches the gap's
 * value.  Transcript, first column to last: 'M' (a query and a subject
 * residue), 'I' (a query residue against a gap), 'D' (a subject residue
 * against a gap).
 *   queries, q_lengths: as sw_search (host or device).
 *   pair_query, pair_subject: n_pairs entries each, host memory.
 *   out: n_pairs records, host memory.
 *   ops: host buffer of ops_capacity bytes; pair k's transcript lies in its
 *        own slot of q_len + s_len bytes (slots back to back in pair order),
 *        at its end.  Needs ops_capacity >= sum over pairs of q_len + s_len.
 * Device memory for the direction bits (4 bits per cell of every pair) is
 * allocated by the call and freed before it returns; pairs are processed in
 * chunks of at most 8 GiB of bits.  Synchronous on the stream.
 * Errors: SW_EINVAL (index out of range, short ops buffer, bad gaps or
 * codes), SW_ENOMEM, SW_ECUDA. */
sw_status sw_align(sw_db* db, const uint8_t* queries, const int32_t* q_lengths, int32_t n_queries,
                   const int32_t* pair_query, const int64_t* pair_subject, int32_t n_pairs,
                   int32_t gap_open, int32_t gap_extend, const int8_t* matrix, sw_alignment* out,
                   uint8_t* ops, int64_t ops_capacity, void* stream);

/* Exact scores of every (query, subject) pair without allocating any memory.
 * The paper has no counterpart: this entry point serves callers that cannot
 * let a library allocate -- a host framework that owns all device memory
 * through its own pool, or a service that must not allocate once it is
 * serving, so that its memory use stays fixed and no call can fail for lack
 * of memory.  Every other search entry point allocates (a database, a plan,
 * kernel scratch); this one calls no cudaMalloc, cudaFree or other allocating
 * routine.
 *   queries, subjects:     concatenated residue codes, device memory of the
 *                          current device; may be NULL when every length on
 *                          that side is 0.
 *   q_offsets, s_offsets:  int64 start of each sequence, device memory.
 *   q_lengths, s_lengths:  int32 lengths, device memory; subjects may be at
 *                          most 4096 residues long, queries any length.
 *   matrix:                24 x 24 int8 SM(query, subject), HOST memory
 *                          (NULL = BLOSUM62).
 *   scores:                n_queries x n_subjects int32, device memory.
 * Every device buffer must belong to the current device (or be managed
 * memory); the call checks this before any launch.
 * Same gap convention and the same scores as sw_search.  The kernel's
 * scratch (one border row per warp, a work counter, a status word) is a
 * file-scope device array of ~16 MiB that every GPU loading the library holds
 * until the process exits; the counter and status are cleared at the start of
 * every call.  The first call on a device looks the array's address up on
 * that device (the device must be current); make that first call before any
 * stream capture.  All calls share the one array, so calls whose work
 * overlaps on the GPU (other streams, other threads) race: serialize them.
 * The call returns after the scores are written (it synchronizes the stream).
 * Errors: SW_EINVAL for negative counts or gaps, a NULL buffer, a buffer
 * that is not memory of the current device, a negative length, a subject
 * longer than 4096 residues, a NULL residue buffer with a positive length, or
 * a code >= 24.  Pairs with a bad length or code are not scored: their
 * entries of `scores` keep what they held; every other pair is scored.
 * SW_ECUDA. */
sw_status sw_search_pairs_noalloc(const uint8_t* queries, const int64_t* q_offsets,
                                  const int32_t* q_lengths, int32_t n_queries,
                                  const uint8_t* subjects, const int64_t* s_offsets,
                                  const int32_t* s_lengths, int32_t n_subjects,
                                  int32_t gap_open, int32_t gap_extend, const int8_t* matrix,
                                  int32_t* scores, void* stream);

/* The query streams of the two-query kernels, for inspection and tests (host
 * only, no device work).  Deals n_queries queries (lengths q_lengths, host)
 * longest first, each to the stream with the fewest strips so far, to
 * 2 x n_pairs streams of `rows`-row strips (each query padded to whole
 * strips, at least one); streams 2k and 2k + 1 form pair k, and the queries
 * of each pair are then split between its two streams so that the longer
 * one is as short as possible.  This is the layout sw_plan_search uses once
 * it has chosen the number of pairs (the batching of Section III-A with two
 * queries per 32-bit word).
 *   strips:   4 int32 per strip, for at most strip_capacity strips: the query
 *             of half 0, its first row | 0x80000000 when the strip is that
 *             query's last; the same for half 1 (query -1: an empty half);
 *   pairs:    2 int32 per stream pair (n_pairs pairs): first strip, strips;
 *   n_strips: the table's length.
 * Errors: SW_EINVAL (rows not 16, 24 or 32; n_pairs outside 1..n_queries/2;
 * a negative length; a NULL buffer), SW_EBUSY (more than strip_capacity
 * strips). */
sw_status sw_query_streams(const int32_t* q_lengths, int32_t n_queries, int32_t rows,
                           int32_t n_pairs, int32_t* strips, int64_t strip_capacity,
                           int32_t* pairs, int64_t* n_strips);

/* Integer-pipe microbenchmark (Section III-B, Eq. 4: the throughput term,
 * measured instead of looked up).  op selects an instruction kind (0 iadd,
 * 1 imax, 2 viaddmax_s32, 3 viaddmax_s16x2, 4 viaddmax_s16x2_relu,
 * 5 vimax3_s16x2, 6 vmaxs2, 7 vsub2, 8 vaddss2, 9 prmt, 10 packed cell pair,
 * 11 packed cell pair + prmt, 12 int32 cell, 13 imad, 14 the biased packed
 * cell pair of the search kernel, 15 vadd4, 16 vmaxu4, 17 vmaxs4, 18 vaddus4,
 * 19 vsubus4, 20 an unsigned biased 8x4 cell update of four cells, 10 ops);
 * results (host memory):
 * out[0] lane-operations per SM clock, out[1] SM clock in MHz, out[2] seconds. */
sw_status sw_intpeak(int32_t op, int32_t blocks_per_sm, int32_t threads, int32_t iters,
                     double* out);

#ifdef __cplusplus
}
#endif

#endif /* SWGB_H */
