/*
 * sw_oracle.c -- plain, slow, scalar int32 reference for Smith-Waterman local
 * alignment scores with Gotoh affine gaps.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path
 * (the CUDA library) never calls it, and the two share no code.
 *
 * What it computes (Section II-B, Eq. 1-3 of arxiv 2309.09609):
 *
 *   H[i][j] = max(0, H[i-1][j-1] + SM(Q[i], D[j]), E[i][j], F[i][j])   (Eq. 1)
 *   E[i][j] = max(H[i][j-1] - Go, E[i][j-1] - Ge)                       (Eq. 2)
 *   F[i][j] = max(H[i-1][j] - Go, F[i-1][j] - Ge)                       (Eq. 3)
 *
 * for 1 <= i <= m, 1 <= j <= n; H is 0 on row 0 and column 0; the score S is
 * the largest H over the whole matrix (Section II-B, text after Eq. 3).
 * Go and Ge are used exactly as in Eq. 2-3: a gap of k residues costs
 * Go + (k-1)*Ge.  The mapping from the library's (gap_open, gap_extend)
 * convention lives in the Python wrapper.
 *
 * Reading of the boundary: the paper initialises E and F with 0 on row 0 and
 * column 0.  oracle_sw_gotoh uses minus infinity there (the textbook Gotoh
 * start); oracle_sw_gotoh_zero_init follows the paper literally.  Both give
 * the same H and S whenever Go, Ge >= 0, and a test checks that.
 *
 * Linear space (Section II-B, last paragraph): only one row of H and F is
 * kept, because only the score is needed.
 *
 * Everything is scalar int32 C; the pair loop is spread over POSIX threads.
 * Nothing is blocked, fused, reordered or vectorised by hand.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* minus infinity for E and F: far below any reachable value, yet safe to
 * subtract a gap penalty from without wrapping int32 */
#define NEG_INF (INT32_MIN / 4)

static int32_t max2(int32_t a, int32_t b) { return a > b ? a : b; }

/* Eq. 1-3 with E and F starting at minus infinity on the borders. */
static int32_t gotoh(const uint8_t *q, int32_t m, const uint8_t *d, int32_t n,
                     const int32_t *sm, int32_t alpha, int32_t go, int32_t ge,
                     int zero_init, int32_t *Hrow, int32_t *Frow) {
  int32_t border_gap = zero_init ? 0 : NEG_INF;
  int32_t best = 0;
  int32_t i, j;
  /* row 0: H = 0, F = border value */
  for (j = 0; j <= n; j++) {
    Hrow[j] = 0;
    Frow[j] = border_gap;
  }
  for (i = 1; i <= m; i++) {
    const int32_t *smrow = sm + (int64_t)q[i - 1] * alpha;
    int32_t h_diag = Hrow[0];  /* H[i-1][0] */
    int32_t h_left = 0;        /* H[i][0]   */
    int32_t e = border_gap;    /* E[i][0]   */
    Hrow[0] = 0;
    for (j = 1; j <= n; j++) {
      int32_t h_up = Hrow[j];  /* H[i-1][j] */
      int32_t f_up = Frow[j];  /* F[i-1][j] */
      int32_t e_ij = max2(h_left - go, e - ge);         /* Eq. 2 */
      int32_t f_ij = max2(h_up - go, f_up - ge);        /* Eq. 3 */
      int32_t h_ij = h_diag + smrow[d[j - 1]];          /* Eq. 1 */
      h_ij = max2(h_ij, e_ij);
      h_ij = max2(h_ij, f_ij);
      h_ij = max2(h_ij, 0);
      if (h_ij > best) best = h_ij;                     /* S = max H */
      h_diag = h_up;
      Hrow[j] = h_ij;
      Frow[j] = f_ij;
      h_left = h_ij;
      e = e_ij;
    }
  }
  return best;
}

static int32_t run_one(const uint8_t *q, int32_t m, const uint8_t *d, int32_t n,
                       const int32_t *sm, int32_t alpha, int32_t go, int32_t ge,
                       int zero_init) {
  int32_t *buf;
  int32_t s;
  if (m <= 0 || n <= 0) return 0;
  buf = (int32_t *)malloc(sizeof(int32_t) * 2 * ((size_t)n + 1));
  if (!buf) return -1;
  s = gotoh(q, m, d, n, sm, alpha, go, ge, zero_init, buf, buf + n + 1);
  free(buf);
  return s;
}

/* One pair; E/F start at minus infinity.  Returns -1 on allocation failure. */
int32_t oracle_sw_gotoh(const uint8_t *q, int32_t m, const uint8_t *d, int32_t n,
                        const int32_t *sm, int32_t alpha, int32_t go, int32_t ge) {
  return run_one(q, m, d, n, sm, alpha, go, ge, 0);
}

/* One pair; E/F start at 0 exactly as the paper states (Section II-B). */
int32_t oracle_sw_gotoh_zero_init(const uint8_t *q, int32_t m, const uint8_t *d,
                                  int32_t n, const int32_t *sm, int32_t alpha,
                                  int32_t go, int32_t ge) {
  return run_one(q, m, d, n, sm, alpha, go, ge, 1);
}

/* ---- many pairs over POSIX threads ------------------------------------- */

typedef struct {
  const uint8_t *qres; const int64_t *qoff; const int32_t *qlen;
  const uint8_t *dres; const int64_t *doff; const int32_t *dlen;
  const int32_t *pair_q; const int64_t *pair_d; int64_t npairs;
  const int32_t *sm; int32_t alpha, go, ge;
  int32_t *out;
  int64_t next;           /* next pair to take, guarded by lock */
  pthread_mutex_t lock;
  int failed;
} job_t;

static void *worker(void *arg) {
  job_t *jb = (job_t *)arg;
  int32_t *buf = NULL;
  int64_t cap = 0;
  for (;;) {
    int64_t lo, hi, k;
    pthread_mutex_lock(&jb->lock);
    lo = jb->next;
    hi = lo + 64;
    if (hi > jb->npairs) hi = jb->npairs;
    jb->next = hi;
    pthread_mutex_unlock(&jb->lock);
    if (lo >= jb->npairs) break;
    for (k = lo; k < hi; k++) {
      int32_t qi = jb->pair_q[k];
      int64_t di = jb->pair_d[k];
      int32_t m = jb->qlen[qi], n = jb->dlen[di];
      if (m <= 0 || n <= 0) { jb->out[k] = 0; continue; }
      if ((int64_t)n + 1 > cap) {
        free(buf);
        cap = 2 * ((int64_t)n + 1);
        buf = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)cap);
        if (!buf) { jb->failed = 1; return NULL; }
      }
      jb->out[k] = gotoh(jb->qres + jb->qoff[qi], m, jb->dres + jb->doff[di], n,
                         jb->sm, jb->alpha, jb->go, jb->ge, 0, buf, buf + n + 1);
    }
  }
  free(buf);
  return NULL;
}

/* Scores of an explicit list of (query, subject) pairs.
 * qres/qoff/qlen: concatenated query codes, start offsets, lengths.
 * dres/doff/dlen: the same for subjects.  out[k] = S(pair_q[k], pair_d[k]).
 * Returns 0, or -1 if a worker could not allocate. */
int32_t oracle_pairs(const uint8_t *qres, const int64_t *qoff, const int32_t *qlen,
                     const uint8_t *dres, const int64_t *doff, const int32_t *dlen,
                     const int32_t *pair_q, const int64_t *pair_d, int64_t npairs,
                     const int32_t *sm, int32_t alpha, int32_t go, int32_t ge,
                     int32_t *out, int32_t nthreads) {
  job_t jb;
  pthread_t *tids;
  int32_t t;
  if (nthreads < 1) nthreads = 1;
  memset(&jb, 0, sizeof jb);
  jb.qres = qres; jb.qoff = qoff; jb.qlen = qlen;
  jb.dres = dres; jb.doff = doff; jb.dlen = dlen;
  jb.pair_q = pair_q; jb.pair_d = pair_d; jb.npairs = npairs;
  jb.sm = sm; jb.alpha = alpha; jb.go = go; jb.ge = ge; jb.out = out;
  pthread_mutex_init(&jb.lock, NULL);
  tids = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
  if (!tids) return -1;
  for (t = 0; t < nthreads; t++) pthread_create(&tids[t], NULL, worker, &jb);
  for (t = 0; t < nthreads; t++) pthread_join(tids[t], NULL);
  free(tids);
  pthread_mutex_destroy(&jb.lock);
  return jb.failed ? -1 : 0;
}

/* ---- BLOSUM62 ------------------------------------------------------------
 * The paper scores with BLOSUM62 (Section IV-A) but does not print it.  This
 * is the public NCBI BLOSUM62 table (Henikoff & Henikoff 1992, half-bit
 * units), in the residue order A R N D C Q E G H I L K M F P S T W Y V B Z X *,
 * typed in for this oracle.  The tests pin it by its structure (symmetry,
 * diagonal, extremes) and by the published Karlin-Altschul parameters of
 * BLOSUM62 under the Robinson & Robinson background frequencies. */
static const int8_t BLOSUM62[24 * 24] = {
/*        A   R   N   D   C   Q   E   G   H   I   L   K   M   F   P   S   T   W   Y   V   B   Z   X   * */
/* A */   4, -1, -2, -2,  0, -1, -1,  0, -2, -1, -1, -1, -1, -2, -1,  1,  0, -3, -2,  0, -2, -1,  0, -4,
/* R */  -1,  5,  0, -2, -3,  1,  0, -2,  0, -3, -2,  2, -1, -3, -2, -1, -1, -3, -2, -3, -1,  0, -1, -4,
/* N */  -2,  0,  6,  1, -3,  0,  0,  0,  1, -3, -3,  0, -2, -3, -2,  1,  0, -4, -2, -3,  3,  0, -1, -4,
/* D */  -2, -2,  1,  6, -3,  0,  2, -1, -1, -3, -4, -1, -3, -3, -1,  0, -1, -4, -3, -3,  4,  1, -1, -4,
/* C */   0, -3, -3, -3,  9, -3, -4, -3, -3, -1, -1, -3, -1, -2, -3, -1, -1, -2, -2, -1, -3, -3, -2, -4,
/* Q */  -1,  1,  0,  0, -3,  5,  2, -2,  0, -3, -2,  1,  0, -3, -1,  0, -1, -2, -1, -2,  0,  3, -1, -4,
/* E */  -1,  0,  0,  2, -4,  2,  5, -2,  0, -3, -3,  1, -2, -3, -1,  0, -1, -3, -2, -2,  1,  4, -1, -4,
/* G */   0, -2,  0, -1, -3, -2, -2,  6, -2, -4, -4, -2, -3, -3, -2,  0, -2, -2, -3, -3, -1, -2, -1, -4,
/* H */  -2,  0,  1, -1, -3,  0,  0, -2,  8, -3, -3, -1, -2, -1, -2, -1, -2, -2,  2, -3,  0,  0, -1, -4,
/* I */  -1, -3, -3, -3, -1, -3, -3, -4, -3,  4,  2, -3,  1,  0, -3, -2, -1, -3, -1,  3, -3, -3, -1, -4,
/* L */  -1, -2, -3, -4, -1, -2, -3, -4, -3,  2,  4, -2,  2,  0, -3, -2, -1, -2, -1,  1, -4, -3, -1, -4,
/* K */  -1,  2,  0, -1, -3,  1,  1, -2, -1, -3, -2,  5, -1, -3, -1,  0, -1, -3, -2, -2,  0,  1, -1, -4,
/* M */  -1, -1, -2, -3, -1,  0, -2, -3, -2,  1,  2, -1,  5,  0, -2, -1, -1, -1, -1,  1, -3, -1, -1, -4,
/* F */  -2, -3, -3, -3, -2, -3, -3, -3, -1,  0,  0, -3,  0,  6, -4, -2, -2,  1,  3, -1, -3, -3, -1, -4,
/* P */  -1, -2, -2, -1, -3, -1, -1, -2, -2, -3, -3, -1, -2, -4,  7, -1, -1, -4, -3, -2, -2, -1, -2, -4,
/* S */   1, -1,  1,  0, -1,  0,  0,  0, -1, -2, -2,  0, -1, -2, -1,  4,  1, -3, -2, -2,  0,  0,  0, -4,
/* T */   0, -1,  0, -1, -1, -1, -1, -2, -2, -1, -1, -1, -1, -2, -1,  1,  5, -2, -2,  0, -1, -1,  0, -4,
/* W */  -3, -3, -4, -4, -2, -2, -3, -2, -2, -3, -2, -3, -1,  1, -4, -3, -2, 11,  2, -3, -4, -3, -2, -4,
/* Y */  -2, -2, -2, -3, -2, -1, -2, -3,  2, -1, -1, -2, -1,  3, -3, -2, -2,  2,  7, -1, -3, -2, -1, -4,
/* V */   0, -3, -3, -3, -1, -2, -2, -3, -3,  3,  1, -2,  1, -1, -2, -2,  0, -3, -1,  4, -3, -2, -1, -4,
/* B */  -2, -1,  3,  4, -3,  0,  1, -1,  0, -3, -4,  0, -3, -3, -2,  0, -1, -4, -3, -3,  4,  1, -1, -4,
/* Z */  -1,  0,  0,  1, -3,  3,  4, -2,  0, -3, -3,  1, -1, -3, -1,  0, -1, -3, -2, -2,  1,  4, -1, -4,
/* X */   0, -1, -1, -1, -2, -1, -1, -1, -1, -1, -1, -1, -1, -1, -2,  0,  0, -2, -1, -1, -1, -1, -1, -4,
/* * */  -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4, -4,  1,
};

/* Copies the oracle's BLOSUM62 (24 x 24, row-major) into out. */
void oracle_blosum62(int8_t *out) { memcpy(out, BLOSUM62, sizeof BLOSUM62); }
