/*
 * Field arithmetic, syndrome and code validation shared by the two oracle
 * decoders (min-max, Alg. 2; FFT-SPA, Alg. 1).  TEST INFRASTRUCTURE ONLY,
 * like the decoders that include it; it shares nothing with the CUDA decoder.
 *
 * Field (Sec. 2.1): elements 0, 1, x, ..., x^(q-2); x = 2 is primitive for
 * the given primitive polynomial; addition is XOR; multiplication through
 * exponent/logarithm tables.
 */
#ifndef NBLDPC_ORACLE_COMMON_H
#define NBLDPC_ORACLE_COMMON_H

#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int q;          /* field order */
  int exp[256];   /* exp[i] = x^i, i = 0..q-2 */
  int log[256];   /* log[exp[i]] = i; log[0] unused */
} gf_t;

/* Build exp/log tables by repeated multiplication by x modulo the primitive
 * polynomial.  Returns 0, or -1 when x does not generate all q-1 non-zero
 * elements (polynomial not primitive / wrong degree). */
static inline int gf_build(gf_t *g, int q, unsigned poly) {
  int p = 0;
  if (q < 2 || q > 256 || (q & (q - 1))) return -1;
  while ((1 << p) < q) p++;
  if ((int)(poly >> p) != 1) return -1; /* degree must be exactly p */
  g->q = q;
  for (int i = 0; i < 256; i++) g->log[i] = -1;
  int v = 1;
  for (int i = 0; i < q - 1; i++) {
    if (g->log[v] != -1) return -1; /* x^i repeated before q-1 steps */
    g->exp[i] = v;
    g->log[v] = i;
    v <<= 1;
    if (v & q) v ^= (int)poly;
  }
  if (v != 1) return -1;
  return 0;
}

static inline int gf_mul(const gf_t *g, int a, int b) {
  if (a == 0 || b == 0) return 0;
  return g->exp[(g->log[a] + g->log[b]) % (g->q - 1)];
}

static inline int gf_inv(const gf_t *g, int a) {
  return g->exp[(g->q - 1 - g->log[a]) % (g->q - 1)];
}

/* syndrome c H^T == 0 ? */
static inline int syndrome_ok(const gf_t *g, int m, const int32_t *row_ptr, const int32_t *col_idx,
                       const int32_t *coef, const int *c) {
  for (int r = 0; r < m; r++) {
    int s = 0;
    for (int e = row_ptr[r]; e < row_ptr[r + 1]; e++) s ^= gf_mul(g, coef[e], c[col_idx[e]]);
    if (s) return 0;
  }
  return 1;
}

/* Validate H: rows of degree >= 2 (max 256), columns in range, no column twice
 * in one row, coefficients 1..q-1, every column used at least once. */
static inline int check_code(int q, int n, int m, const int32_t *row_ptr, const int32_t *col_idx,
                      const int32_t *coef) {
  if (n <= 0 || m <= 0 || row_ptr[0] != 0) return -1;
  int *seen = calloc((size_t)n, sizeof(int));
  int *last = malloc(sizeof(int) * (size_t)n);
  for (int i = 0; i < n; i++) last[i] = -1;
  int bad = 0;
  for (int r = 0; r < m && !bad; r++) {
    int d = row_ptr[r + 1] - row_ptr[r];
    if (d < 2 || d > 256) bad = 1;
    for (int e = row_ptr[r]; e < row_ptr[r + 1] && !bad; e++) {
      int c = col_idx[e];
      if (c < 0 || c >= n || coef[e] <= 0 || coef[e] >= q || last[c] == r) bad = 1;
      else { last[c] = r; seen[c]++; }
    }
  }
  for (int c = 0; c < n && !bad; c++)
    if (!seen[c]) bad = 1;
  free(seen); free(last);
  return bad ? -1 : 0;
}

#endif
