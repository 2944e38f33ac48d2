/*
 * sw_align_oracle.c -- plain, slow reference for the optimal local alignment
 * itself (its end points and its column-by-column transcript), not only its
 * score.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite and the benchmark's CPU leg
 * may load this library.  The product path never calls it, and the two share
 * no code.
 *
 * It fills the full (m+1) x (n+1) matrices of Eq. 1-3 (Section II-B) in
 * int32, E and F starting at minus infinity on row 0 and column 0:
 *
 *   E[i][j] = max(H[i][j-1] - Go, E[i][j-1] - Ge)                       (Eq. 2)
 *   F[i][j] = max(H[i-1][j] - Go, F[i-1][j] - Ge)                       (Eq. 3)
 *   H[i][j] = max(0, H[i-1][j-1] + SM(Q[i], D[j]), E[i][j], F[i][j])   (Eq. 1)
 *
 * and walks back from the cell holding the score S (the traceback that the
 * paper names for recovering the alignment, Section II-B).  Several
 * alignments can reach S; the paper does not say which one to return, so
 * this reference fixes one, and the CUDA path follows the same rules:
 *
 *   1. the alignment ends at the first cell (i, j) in row-major order
 *      (smallest i, then smallest j) whose H equals S;
 *   2. walking back in state H (always at a cell with H > 0): the diagonal
 *      term H[i-1][j-1] + SM first, then E[i][j], then F[i][j], whichever
 *      equals H[i][j];
 *   3. in state E (F) at (i, j): the gap was opened from H[i][j-1]
 *      (H[i-1][j]) when E[i][j] (F[i][j]) equals that minus Go, otherwise it
 *      extends E[i][j-1] (F[i-1][j]);
 *   4. the walk ends with the diagonal step into a cell whose H is 0.
 *
 * Transcript, first column to last: 'M' aligns Q[i] with D[j], 'I' aligns
 * Q[i] with a gap (a step up), 'D' aligns D[j] with a gap (a step left).
 * The aligned residues are Q[qb..qe) and D[sb..se), 0-based.
 *
 * O(mn) memory: for test sizes only.
 */
#include <stdint.h>
#include <stdlib.h>

#define NEG_INF (INT32_MIN / 4)

static int32_t max2(int32_t a, int32_t b) { return a > b ? a : b; }

/* Returns S (>= 0); -1 when memory runs out, -2 when ops_cap < m + n. */
int32_t oracle_sw_align(const uint8_t *q, int32_t m, const uint8_t *d, int32_t n,
                        const int32_t *sm, int32_t alpha, int32_t go, int32_t ge,
                        int32_t *qb, int32_t *qe, int32_t *sb, int32_t *se,
                        char *ops, int64_t ops_cap, int64_t *n_ops) {
  int32_t *H, *E, *F;
  char *rev;
  int64_t W, k, t;
  int32_t i, j, best = 0, bi = 0, bj = 0, state;
  *qb = *qe = *sb = *se = 0;
  *n_ops = 0;
  if (m <= 0 || n <= 0) return 0;
  if (ops_cap < (int64_t)m + n) return -2;
  W = (int64_t)n + 1;
  H = (int32_t *)malloc(sizeof(int32_t) * (size_t)((m + 1) * W));
  E = (int32_t *)malloc(sizeof(int32_t) * (size_t)((m + 1) * W));
  F = (int32_t *)malloc(sizeof(int32_t) * (size_t)((m + 1) * W));
  rev = (char *)malloc((size_t)m + (size_t)n);
  if (!H || !E || !F || !rev) {
    free(H); free(E); free(F); free(rev);
    return -1;
  }
#define AT(X, r, c) X[(int64_t)(r) * W + (c)]
  for (j = 0; j <= n; j++) {
    AT(H, 0, j) = 0;
    AT(E, 0, j) = NEG_INF;
    AT(F, 0, j) = NEG_INF;
  }
  for (i = 1; i <= m; i++) {
    AT(H, i, 0) = 0;
    AT(E, i, 0) = NEG_INF;
    AT(F, i, 0) = NEG_INF;
    for (j = 1; j <= n; j++) {
      int32_t e = max2(AT(H, i, j - 1) - go, AT(E, i, j - 1) - ge);   /* Eq. 2 */
      int32_t f = max2(AT(H, i - 1, j) - go, AT(F, i - 1, j) - ge);   /* Eq. 3 */
      int32_t h = AT(H, i - 1, j - 1) + sm[(int64_t)q[i - 1] * alpha + d[j - 1]];
      h = max2(max2(h, e), max2(f, 0));                                /* Eq. 1 */
      AT(E, i, j) = e;
      AT(F, i, j) = f;
      AT(H, i, j) = h;
      if (h > best) {  /* strictly greater: the first such cell in row-major order */
        best = h;
        bi = i;
        bj = j;
      }
    }
  }
  if (best > 0) {
    /* rule 2-4: walk back from (bi, bj) in state H (0 = H, 1 = E, 2 = F) */
    i = bi;
    j = bj;
    state = 0;
    k = 0;
    for (;;) {
      if (state == 0) {
        const int32_t v = AT(H, i, j);
        const int32_t diag = AT(H, i - 1, j - 1) + sm[(int64_t)q[i - 1] * alpha + d[j - 1]];
        if (v == diag) {
          rev[k++] = 'M';
          i--;
          j--;
          if (AT(H, i, j) == 0) break;
        } else if (v == AT(E, i, j)) {
          state = 1;
        } else {
          state = 2;
        }
      } else if (state == 1) {
        rev[k++] = 'D';
        state = AT(E, i, j) == AT(H, i, j - 1) - go ? 0 : 1;
        j--;
      } else {
        rev[k++] = 'I';
        state = AT(F, i, j) == AT(H, i - 1, j) - go ? 0 : 2;
        i--;
      }
    }
    for (t = 0; t < k; t++) ops[t] = rev[k - 1 - t];
    *n_ops = k;
    *qb = i;
    *sb = j;
    *qe = bi;
    *se = bj;
  }
#undef AT
  free(H); free(E); free(F); free(rev);
  return best;
}
