/*
 * Plain CPU oracle for FFT-based sum-product (FFT-SPA) decoding of
 * non-binary LDPC codes over GF(2^p) (Alg. 1 of "In-Memory Non-Binary LDPC
 * Decoding").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite and the CPU leg of the
 * benchmark load this file; the decoder library never does.  It shares no
 * code, header, table or constant with the CUDA decoder.
 *
 * Arithmetic is IEEE double throughout (the decoder computes in float); the
 * steps follow Alg. 1 in the paper's order:
 *
 *   initialization   u^(0)_{m,n}(x) = p_n(x), the channel probabilities
 *   stop test        c^(k-1) H^T = 0 before iteration k (when enabled)
 *   permutation      u'_{m,n}(h_{m,n} x) = u_{m,n}(x)
 *   check node       v_{m,n} = FFT^-1( prod over j in S_v(m)\n of FFT(u'_{m,j}) )
 *   depermutation    v'_{m,n}(x) = v_{m,n}(h_{m,n} x)
 *   variable node    z_{m,n}(x) = p_n(x) prod over i in S_c(n)\m of v'_{i,n}(x),
 *                    u_{m,n} = z_{m,n} / sum_x z_{m,n}(x)
 *   decision         z'_n(x) = p_n(x) prod over i in S_c(n) of v'_{i,n}(x),
 *                    c_n = argmax_x z'_n(x)
 *
 * "FFT" is the radix-2 transform over (Z_2)^p (Sec. 4, FFT-SPA blocks):
 * W(s) = sum_x (-1)^popcount(s & x) u(x), the Walsh-Hadamard transform, which
 * turns the XOR convolution of the check node into a product.  Its inverse is
 * the same transform divided by q.
 *
 * Readings where the paper is silent or garbled:
 *  - the permutation multiplies the symbol index by h (the printed
 *    "h^-1 . u(x)" and "h . v(x^-1)" are index maps; in GF(2^p) every element
 *    is its own additive inverse, so x^-1 in the depermutation is x);
 *  - the decision multiplies the incoming check messages v' (the printed
 *    product over u is read as v', which makes z' the a-posteriori
 *    probability of the symbol);
 *  - a check-node output below zero (rounding of the transform) is set to 0;
 *  - a normalization whose sum is not positive gives the uniform vector 1/q;
 *  - ties in the decision take the lowest symbol; "iterations" counts
 *    completed check+variable passes, as in the min-max oracle.
 *
 * parity pins: transform against its definition, brute-force check update,
 * exact marginals on a cycle-free graph, binary belief propagation at q = 2
 * (tests/).
 */
#include "oracle_common.h"

/* Radix-2 Walsh-Hadamard transform in place: for each bit b = 0..p-1, the
 * butterfly (a, b) -> (a + b, a - b) over the pairs (x, x + 2^b), x without
 * bit b. */
static void wht(double *v, int q) {
  for (int h = 1; h < q; h <<= 1)
    for (int i = 0; i < q; i += 2 * h)
      for (int x = i; x < i + h; x++) {
        double a = v[x], b = v[x + h];
        v[x] = a + b;
        v[x + h] = a - b;
      }
}

/* Exported transform (for the definition pin). */
void orc_wht(int q, double *v) { wht(v, q); }

/* Normalize z[q] to sum 1 (uniform when the sum is not positive). */
static void normalize(double *z, int q) {
  double s = 0.0;
  for (int x = 0; x < q; x++) s += z[x];
  for (int x = 0; x < q; x++) z[x] = s > 0.0 ? z[x] / s : 1.0 / q;
}

/* ---- check-node processing (Alg. 1: permutation, FFT, product, inverse FFT,
 * depermutation) for one check with d edges, coefficients h[j], incoming
 * messages u[j][x] and outgoing messages v'[j][x].  W and T are d*q and q
 * scratch. */
static void cnp_one_check(const gf_t *g, int d, const int *h, double *const *u, double *const *vout,
                          double *W, double *T) {
  int q = g->q;
  for (int j = 0; j < d; j++) {
    /* permutation: u'_j(h_j x) = u_j(x) */
    for (int x = 0; x < q; x++) W[j * q + gf_mul(g, h[j], x)] = u[j][x];
    /* FFT */
    wht(W + j * q, q);
  }
  for (int n = 0; n < d; n++) {
    /* product over the other edges in the transform domain */
    for (int s = 0; s < q; s++) {
      double pr = 1.0;
      for (int j = 0; j < d; j++)
        if (j != n) pr *= W[j * q + s];
      T[s] = pr;
    }
    /* inverse FFT: the same transform, divided by q; negative rounding -> 0 */
    wht(T, q);
    for (int y = 0; y < q; y++) {
      T[y] /= q;
      if (T[y] < 0.0) T[y] = 0.0;
    }
    /* depermutation: v'_n(x) = v_n(h_n x) */
    for (int x = 0; x < q; x++) vout[n][x] = T[gf_mul(g, h[n], x)];
  }
}

/* Exported single-check update (for the brute-force pin). */
int orc_fft_check_update(int q, unsigned poly, int d, const int32_t *h, const double *u_in /* d*q */,
                         double *v_out /* d*q */) {
  gf_t g;
  if (gf_build(&g, q, poly) || d < 2) return -1;
  for (int j = 0; j < d; j++)
    if (h[j] <= 0 || h[j] >= q) return -1;
  double *u = malloc(sizeof(double) * (size_t)d * q);
  double **up = malloc(sizeof(double *) * (size_t)d), **vp = malloc(sizeof(double *) * (size_t)d);
  double *W = malloc(sizeof(double) * (size_t)d * q), *T = malloc(sizeof(double) * (size_t)q);
  int *hh = malloc(sizeof(int) * (size_t)d);
  for (int j = 0; j < d; j++) {
    hh[j] = h[j];
    up[j] = u + (size_t)j * q;
    vp[j] = v_out + (size_t)j * q;
    for (int x = 0; x < q; x++) up[j][x] = u_in[(size_t)j * q + x];
  }
  cnp_one_check(&g, d, hh, up, vp, W, T);
  free(u); free(up); free(vp); free(W); free(T); free(hh);
  return 0;
}

/*
 * Decode `frames` frames.  prob: [frames][n][q] channel probabilities p_n(x)
 * (float, as the decoder receives them; symbol value is the index).
 * Outputs: out_sym [frames][n], out_iters [frames], out_ok [frames] and, when
 * out_app is not NULL, the normalized a-posteriori vectors z'_n / sum z'_n of
 * the last decision ([frames][n][q]; p_n normalized when no iteration ran).
 * Returns 0, or -1 on invalid arguments (nothing written).
 */
int orc_fftspa_decode(int q, unsigned poly, int n, int m, const int32_t *row_ptr, const int32_t *col_idx,
                      const int32_t *coef, const float *prob, int frames, int max_iters, int early_stop,
                      uint8_t *out_sym, int32_t *out_iters, uint8_t *out_ok, double *out_app) {
  gf_t g;
  if (gf_build(&g, q, poly) || frames < 0 || max_iters < 0) return -1;
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

  double *p = malloc(sizeof(double) * (size_t)n * q);
  double *u = malloc(sizeof(double) * (size_t)E * q);    /* VN -> CN */
  double *v = malloc(sizeof(double) * (size_t)E * q);    /* CN -> VN (depermuted) */
  double *W = malloc(sizeof(double) * (size_t)dmax * q);
  double *T = malloc(sizeof(double) * (size_t)q);
  double *z = malloc(sizeof(double) * (size_t)q);
  double **up = malloc(sizeof(double *) * (size_t)dmax), **vp = malloc(sizeof(double *) * (size_t)dmax);
  int *hrow = malloc(sizeof(int) * (size_t)dmax);
  int *chat = malloc(sizeof(int) * (size_t)n);

  for (int f = 0; f < frames; f++) {
    double *app = out_app ? out_app + (size_t)f * n * q : NULL;
    for (int i = 0; i < n * q; i++) p[i] = (double)prob[(size_t)f * n * q + i];
    /* Initialization: u^(0)_{m,n} = p_n */
    for (int e = 0; e < E; e++)
      for (int x = 0; x < q; x++) u[(size_t)e * q + x] = p[(size_t)col_idx[e] * q + x];
    /* c^(0) = argmax p_n (lowest symbol on ties) */
    for (int c = 0; c < n; c++) {
      int best = 0;
      for (int x = 1; x < q; x++)
        if (p[(size_t)c * q + x] > p[(size_t)c * q + best]) best = x;
      chat[c] = best;
      if (app) {
        for (int x = 0; x < q; x++) z[x] = p[(size_t)c * q + x];
        normalize(z, q);
        for (int x = 0; x < q; x++) app[(size_t)c * q + x] = z[x];
      }
    }
    int ok = syndrome_ok(&g, m, row_ptr, col_idx, coef, chat);
    int iters = 0;
    if (!(early_stop && ok)) {
      for (int k = 1; k <= max_iters; k++) {
        /* permutation, CNP, depermutation for every check node */
        for (int r = 0; r < m; r++) {
          int d = row_ptr[r + 1] - row_ptr[r];
          for (int j = 0; j < d; j++) {
            int e = row_ptr[r] + j;
            hrow[j] = coef[e];
            up[j] = u + (size_t)e * q;
            vp[j] = v + (size_t)e * q;
          }
          cnp_one_check(&g, d, hrow, up, vp, W, T);
        }
        /* VNP for every variable node, then the a-posteriori decision */
        for (int c = 0; c < n; c++) {
          for (int a = vptr[c]; a < vptr[c + 1]; a++) {
            for (int x = 0; x < q; x++) {
              double s = p[(size_t)c * q + x];
              for (int b = vptr[c]; b < vptr[c + 1]; b++)
                if (b != a) s *= v[(size_t)vedge[b] * q + x];
              z[x] = s;
            }
            normalize(z, q);
            for (int x = 0; x < q; x++) u[(size_t)vedge[a] * q + x] = z[x];
          }
          for (int x = 0; x < q; x++) {
            double s = p[(size_t)c * q + x];
            for (int b = vptr[c]; b < vptr[c + 1]; b++) s *= v[(size_t)vedge[b] * q + x];
            z[x] = s;
          }
          int best = 0;
          for (int x = 1; x < q; x++)
            if (z[x] > z[best]) best = x;
          chat[c] = best;
          if (app) {
            normalize(z, q);
            for (int x = 0; x < q; x++) app[(size_t)c * q + x] = z[x];
          }
        }
        iters = k;
        ok = syndrome_ok(&g, m, row_ptr, col_idx, coef, chat);
        if (early_stop && ok) break;
      }
    }
    for (int c = 0; c < n; c++) out_sym[(size_t)f * n + c] = (uint8_t)chat[c];
    out_iters[f] = iters;
    out_ok[f] = (uint8_t)ok;
  }
  free(vdeg); free(vptr); free(vfill); free(vedge); free(p); free(u); free(v); free(W); free(T); free(z);
  free(up); free(vp); free(hrow); free(chat);
  return 0;
}
