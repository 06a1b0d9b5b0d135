/*
 * Plain CPU oracle for min-max (MMA) decoding of non-binary LDPC codes over
 * GF(2^p) (Alg. 2 of "In-Memory Non-Binary LDPC Decoding").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline of the benchmark load this file; the decoder library never does.
 * It shares no code, header, table or constant with the CUDA decoder.
 *
 * Written for obviousness, not speed: every step follows the algorithm in the
 * paper's order and notation, with int arithmetic throughout.  Readings of
 * points where the paper is silent are marked "reading:".
 *
 *  - Field (Sec. 2.1): elements 0, 1, x, ..., x^(q-2); x = 2 is primitive for
 *    the given primitive polynomial; addition is XOR; multiplication through
 *    exponent/logarithm tables (Sec. 2.3, "implemented in LUTs").
 *  - Messages: gamma, alpha, beta are non-negative integer reliabilities
 *    relative to the most likely symbol (Alg. 2, initialization).
 *    reading: messages are 8-bit; the only saturation is min(255, .) applied
 *    after the variable-node normalization; alpha^(0) = gamma unchanged.
 *  - Schedule: flooding (all check nodes, then all variable nodes).
 *  - reading: hard decisions take the lowest symbol on ties; the stop test on
 *    c^(k-1) comes before iteration k; "iterations" counts completed
 *    check+variable passes.
 *
 * parity pins: field axioms, brute-force check update, binary min-sum at
 * q = 2, zero syndrome, noiseless recovery, edge-order invariance (tests/).
 */
#include "oracle_common.h"

/* ---- exported field helpers (for the field-axiom pins) ---------------- */
int orc_gf_tables(int q, unsigned poly, int32_t *exp_out, int32_t *log_out) {
  gf_t g;
  if (gf_build(&g, q, poly)) return -1;
  for (int i = 0; i < q - 1; i++) exp_out[i] = g.exp[i];
  log_out[0] = -1;
  for (int a = 1; a < q; a++) log_out[a] = g.log[a];
  return 0;
}

int orc_gf_mul_all(int q, unsigned poly, int32_t *mul_out /* q*q */, int32_t *inv_out /* q */) {
  gf_t g;
  if (gf_build(&g, q, poly)) return -1;
  for (int a = 0; a < q; a++)
    for (int b = 0; b < q; b++) mul_out[a * q + b] = gf_mul(&g, a, b);
  inv_out[0] = 0;
  for (int a = 1; a < q; a++) inv_out[a] = gf_inv(&g, a);
  return 0;
}

/* ---- check-node processing (Alg. 2, "CNP, F & B matrices" and "beta") ----
 *
 * One check node with d edges, coefficients h[0..d-1] and incoming messages
 * alpha[j][x] (variable order x).  Edge order is the order given.
 *
 *   F_0(x)   = alpha_0(h_0^-1 x)
 *   F_n(x)   = min over (x', x'') with x' + h_n x'' = x of max(F_{n-1}(x'), alpha_n(x''))
 *   B_{d-1}(x) = alpha_{d-1}(h_{d-1}^-1 x)
 *   B_{n-1}(x) = min over x' + h_{n-1} x'' = x of max(B_n(x'), alpha_{n-1}(x''))
 *   beta_0(x)     = B_1(h_0 x)
 *   beta_{d-1}(x) = F_{d-2}(h_{d-1} x)
 *   beta_n(x)     = min over x' + h_n x = x'' of max(F_{n-1}(x''), B_{n+1}(x'))
 *
 * Each "min over pairs" visits every pair (x', x'') once and lets it bid for
 * the one output symbol it constrains.                                      */
#define BIG 0x7fffffff

/* pairs (optional, [3]): pairs (x', x'') visited by the F, B and beta
 * "remaining edges" blocks, counted row by row as they run (the work that
 * Table 1 tabulates per block). */
static void cnp_one_check(const gf_t *g, int d, const int *h, int *const *alpha, int *const *beta,
                          int *F /* d*q */, int *B /* d*q */, long long *pairs) {
  const int q = g->q;
  /* F & B: first edges */
  const int hinv_first = gf_inv(g, h[0]), hinv_last = gf_inv(g, h[d - 1]);
  for (int x = 0; x < q; x++) {
    F[0 * q + x] = alpha[0][gf_mul(g, hinv_first, x)];
    B[(d - 1) * q + x] = alpha[d - 1][gf_mul(g, hinv_last, x)];
  }
  /* F: remaining edges, n = 1..d-2 (F_{d-1} is never used) */
  for (int n = 1; n <= d - 2; n++) {
    for (int x = 0; x < q; x++) F[n * q + x] = BIG;
    for (int x1 = 0; x1 < q; x1++) {        /* x'  */
      if (pairs) pairs[0] += q;
      for (int x2 = 0; x2 < q; x2++) {      /* x'' */
        int x = x1 ^ gf_mul(g, h[n], x2);
        int v = F[(n - 1) * q + x1] > alpha[n][x2] ? F[(n - 1) * q + x1] : alpha[n][x2];
        if (v < F[n * q + x]) F[n * q + x] = v;
      }
    }
  }
  /* B: remaining edges, B_{n-1} from B_n for n = d-1 down to 2 (B_0 unused) */
  for (int n = d - 1; n >= 2; n--) {
    for (int x = 0; x < q; x++) B[(n - 1) * q + x] = BIG;
    for (int x1 = 0; x1 < q; x1++) {
      if (pairs) pairs[1] += q;
      for (int x2 = 0; x2 < q; x2++) {
        int x = x1 ^ gf_mul(g, h[n - 1], x2);
        int v = B[n * q + x1] > alpha[n - 1][x2] ? B[n * q + x1] : alpha[n - 1][x2];
        if (v < B[(n - 1) * q + x]) B[(n - 1) * q + x] = v;
      }
    }
  }
  /* beta: first and last edge */
  for (int x = 0; x < q; x++) {
    beta[0][x] = B[1 * q + gf_mul(g, h[0], x)];
    beta[d - 1][x] = F[(d - 2) * q + gf_mul(g, h[d - 1], x)];
  }
  /* beta: remaining edges */
  for (int n = 1; n <= d - 2; n++) {
    const int hinv = gf_inv(g, h[n]);
    for (int x = 0; x < q; x++) beta[n][x] = BIG;
    for (int x1 = 0; x1 < q; x1++) {        /* x'  */
      if (pairs) pairs[2] += q;
      for (int x3 = 0; x3 < q; x3++) {      /* x'' */
        /* x' + h_n x = x''  <=>  x = h_n^-1 (x' + x'') */
        int x = gf_mul(g, hinv, x1 ^ x3);
        int v = F[(n - 1) * q + x3] > B[(n + 1) * q + x1] ? F[(n - 1) * q + x3] : B[(n + 1) * q + x1];
        if (v < beta[n][x]) beta[n][x] = v;
      }
    }
  }
}

/* Exported single-check update (for the brute-force pin); pairs (optional,
 * [3]) receives the pairs visited by the F, B and beta remaining-edge blocks. */
int orc_check_update_counted(int q, unsigned poly, int d, const int32_t *h, const uint8_t *alpha_in /* d*q */,
                             uint8_t *beta_out /* d*q */, long long *pairs) {
  gf_t g;
  if (gf_build(&g, q, poly) || d < 2) return -1;
  for (int j = 0; j < d; j++)
    if (h[j] <= 0 || h[j] >= q) return -1;
  int *a = malloc(sizeof(int) * d * q), *b = malloc(sizeof(int) * d * q);
  int *F = malloc(sizeof(int) * d * q), *B = malloc(sizeof(int) * d * q);
  int **ap = malloc(sizeof(int *) * d), **bp = malloc(sizeof(int *) * d);
  int hh[256];
  for (int j = 0; j < d; j++) {
    hh[j] = h[j];
    ap[j] = a + j * q;
    bp[j] = b + j * q;
    for (int x = 0; x < q; x++) a[j * q + x] = alpha_in[j * q + x];
  }
  if (pairs) pairs[0] = pairs[1] = pairs[2] = 0;
  cnp_one_check(&g, d, hh, ap, bp, F, B, pairs);
  for (int i = 0; i < d * q; i++) beta_out[i] = (uint8_t)b[i];
  free(a); free(b); free(F); free(B); free(ap); free(bp);
  return 0;
}

int orc_check_update(int q, unsigned poly, int d, const int32_t *h, const uint8_t *alpha_in /* d*q */,
                     uint8_t *beta_out /* d*q */) {
  return orc_check_update_counted(q, poly, d, h, alpha_in, beta_out, NULL);
}

/* ---- decoder --------------------------------------------------------- */

/*
 * Decode `frames` frames.  gamma: [frames][n][q] (symbol value is the index).
 * Outputs: out_sym [frames][n], out_iters [frames], out_ok [frames].
 * cap: the saturation of the variable-node messages (255 for the 8-bit
 * messages of the main reading; 65535 for the 16-bit-message comparison).
 * Returns 0, or -1 on invalid arguments (nothing written).
 */
/* Messages of the last iteration run, for tests (orc_decode_trace). */
typedef struct {
  int32_t *beta;   /* [E][q] check-node outputs */
  int32_t *s;      /* [n][q] a-posteriori sums */
  int32_t *alpha;  /* [E][q] variable-node outputs */
} trace_t;

static int decode_frames(int q, unsigned poly, int n, int m, const int32_t *row_ptr, const int32_t *col_idx,
                         const int32_t *coef, const uint8_t *gamma, int frames, int max_iters, int early_stop,
                         int cap, uint8_t *out_sym, int32_t *out_iters, uint8_t *out_ok, const trace_t *tr) {
  gf_t g;
  if (gf_build(&g, q, poly) || frames < 0 || max_iters < 0 || cap < 1) return -1;
  if (check_code(q, n, m, row_ptr, col_idx, coef)) return -1;
  const int E = row_ptr[m];

  /* variable-node view: for each column, the edges (CSR positions) on it */
  int *vdeg = calloc((size_t)n, sizeof(int));
  for (int e = 0; e < E; e++) vdeg[col_idx[e]]++;
  int *vptr = malloc(sizeof(int) * (size_t)(n + 1));
  vptr[0] = 0;
  for (int c = 0; c < n; c++) vptr[c + 1] = vptr[c] + vdeg[c];
  int *vfill = calloc((size_t)n, sizeof(int));
  int *vedge = malloc(sizeof(int) * (size_t)E);
  for (int e = 0; e < E; e++) {
    int c = col_idx[e];
    vedge[vptr[c] + vfill[c]++] = e;
  }

  int dmax = 0;
  for (int r = 0; r < m; r++)
    if (row_ptr[r + 1] - row_ptr[r] > dmax) dmax = row_ptr[r + 1] - row_ptr[r];

  int *alpha = malloc(sizeof(int) * (size_t)E * q);   /* VN -> CN */
  int *beta = malloc(sizeof(int) * (size_t)E * q);    /* CN -> VN */
  int *F = malloc(sizeof(int) * (size_t)dmax * q);
  int *B = malloc(sizeof(int) * (size_t)dmax * q);
  int **ap = malloc(sizeof(int *) * (size_t)dmax), **bp = malloc(sizeof(int *) * (size_t)dmax);
  int *hrow = malloc(sizeof(int) * (size_t)dmax);
  int *chat = malloc(sizeof(int) * (size_t)n);
  int *ap_sum = malloc(sizeof(int) * (size_t)q);

  for (int f = 0; f < frames; f++) {
    const uint8_t *gam = gamma + (size_t)f * n * q;
    /* Initialization: alpha^(0)_{m,n} = gamma_n */
    for (int e = 0; e < E; e++)
      for (int x = 0; x < q; x++) alpha[(size_t)e * q + x] = gam[(size_t)col_idx[e] * q + x];
    /* c^(0) = argmin gamma (lowest symbol on ties) */
    for (int c = 0; c < n; c++) {
      int best = 0;
      for (int x = 1; x < q; x++)
        if (gam[(size_t)c * q + x] < gam[(size_t)c * q + best]) best = x;
      chat[c] = best;
    }
    int ok = syndrome_ok(&g, m, row_ptr, col_idx, coef, chat);
    int iters = 0;
    if (!(early_stop && ok)) {
      for (int k = 1; k <= max_iters; k++) {
        /* CNP for every check node */
        for (int r = 0; r < m; r++) {
          int d = row_ptr[r + 1] - row_ptr[r];
          for (int j = 0; j < d; j++) {
            int e = row_ptr[r] + j;
            hrow[j] = coef[e];
            ap[j] = alpha + (size_t)e * q;
            bp[j] = beta + (size_t)e * q;
          }
          cnp_one_check(&g, d, hrow, ap, bp, F, B, NULL);
        }
        if (tr && k == max_iters)
          for (size_t i = 0; i < (size_t)E * q; i++) tr->beta[i] = beta[i];
        /* VNP for every variable node:
         *   alpha'_{m,n}(x) = gamma_n(x) + sum over i in S_c(n)\m of beta_{i,n}(x)
         *   alpha_{m,n}(x)  = alpha'(x) - min_x alpha'(x), saturated at cap   */
        for (int c = 0; c < n; c++) {
          for (int a = vptr[c]; a < vptr[c + 1]; a++) {
            int e = vedge[a];
            int mn = BIG;
            for (int x = 0; x < q; x++) {
              int s = gam[(size_t)c * q + x];
              for (int b = vptr[c]; b < vptr[c + 1]; b++)
                if (b != a) s += beta[(size_t)vedge[b] * q + x];
              alpha[(size_t)e * q + x] = s;
              if (s < mn) mn = s;
            }
            for (int x = 0; x < q; x++) {
              int v = alpha[(size_t)e * q + x] - mn;
              alpha[(size_t)e * q + x] = v > cap ? cap : v;
            }
          }
          /* a posteriori information and hard decision */
          for (int x = 0; x < q; x++) {
            int s = gam[(size_t)c * q + x];
            for (int b = vptr[c]; b < vptr[c + 1]; b++) s += beta[(size_t)vedge[b] * q + x];
            ap_sum[x] = s;
            if (tr && k == max_iters) tr->s[(size_t)c * q + x] = s;
          }
          int best = 0;
          for (int x = 1; x < q; x++)
            if (ap_sum[x] < ap_sum[best]) best = x;
          chat[c] = best;
        }
        if (tr && k == max_iters)
          for (size_t i = 0; i < (size_t)E * q; i++) tr->alpha[i] = alpha[i];
        iters = k;
        ok = syndrome_ok(&g, m, row_ptr, col_idx, coef, chat);
        if (early_stop && ok) break;
      }
    }
    for (int c = 0; c < n; c++) out_sym[(size_t)f * n + c] = (uint8_t)chat[c];
    out_iters[f] = iters;
    out_ok[f] = (uint8_t)ok;
  }
  free(vdeg); free(vptr); free(vfill); free(vedge); free(alpha); free(beta);
  free(F); free(B); free(ap); free(bp); free(hrow); free(chat); free(ap_sum);
  return 0;
}

int orc_decode_cap(int q, unsigned poly, int n, int m, const int32_t *row_ptr, const int32_t *col_idx,
                   const int32_t *coef, const uint8_t *gamma, int frames, int max_iters, int early_stop,
                   int cap, uint8_t *out_sym, int32_t *out_iters, uint8_t *out_ok) {
  return decode_frames(q, poly, n, m, row_ptr, col_idx, coef, gamma, frames, max_iters, early_stop, cap, out_sym,
                       out_iters, out_ok, NULL);
}

/*
 * One frame decoded for exactly `iters` >= 1 iterations without early stop,
 * returning, besides the decision, the messages of the last iteration: the
 * check-node outputs beta [E][q], the a-posteriori sums S [n][q] of the
 * decision and the variable-node outputs alpha [E][q] (edges in CSR order).
 * The same loop as orc_decode_cap, which it shares; only the copies out are
 * added.  Test helper for hand-worked iterations.
 */
int orc_decode_trace(int q, unsigned poly, int n, int m, const int32_t *row_ptr, const int32_t *col_idx,
                     const int32_t *coef, const uint8_t *gamma, int iters, int cap, int32_t *beta_out,
                     int32_t *s_out, int32_t *alpha_out, uint8_t *out_sym) {
  if (iters < 1) return -1;
  trace_t tr = {beta_out, s_out, alpha_out};
  int32_t its = 0;
  uint8_t ok = 0;
  return decode_frames(q, poly, n, m, row_ptr, col_idx, coef, gamma, 1, iters, 0, cap, out_sym, &its, &ok, &tr);
}

/* The main reading: 8-bit messages, saturation at 255. */
int orc_decode(int q, unsigned poly, int n, int m, const int32_t *row_ptr, const int32_t *col_idx,
               const int32_t *coef, const uint8_t *gamma, int frames, int max_iters, int early_stop,
               uint8_t *out_sym, int32_t *out_iters, uint8_t *out_ok) {
  return orc_decode_cap(q, poly, n, m, row_ptr, col_idx, coef, gamma, frames, max_iters, early_stop, 255,
                        out_sym, out_iters, out_ok);
}

/* Syndrome check of given words (for tests). */
int orc_syndrome_ok(int q, unsigned poly, int n, int m, const int32_t *row_ptr, const int32_t *col_idx,
                    const int32_t *coef, const uint8_t *words, int frames, uint8_t *out_ok) {
  gf_t g;
  if (gf_build(&g, q, poly)) return -1;
  int *c = malloc(sizeof(int) * (size_t)n);
  for (int f = 0; f < frames; f++) {
    for (int i = 0; i < n; i++) c[i] = words[(size_t)f * n + i];
    out_ok[f] = (uint8_t)syndrome_ok(&g, m, row_ptr, col_idx, coef, c);
  }
  free(c);
  return 0;
}
