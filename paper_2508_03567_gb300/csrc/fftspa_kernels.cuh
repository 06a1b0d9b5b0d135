// FFT-based sum-product (FFT-SPA, Alg. 1) decoding of non-binary LDPC codes
// over GF(2^p): device code for sm_103a, float arithmetic.  One persistent
// block per SM decodes one frame at a time with the flooding schedule of
// Alg. 1 (check-node pass: permutation, transform, product, inverse
// transform, depermutation; variable-node pass: product with the channel
// probabilities, normalization, decision; syndrome), then takes the next
// frame from a global counter.
//
// Messages are q floats per Tanner-graph edge in a per-block global slot
// (resident in L2), updated in place: the check-node pass reads u (variable
// to check) and writes v' (check to variable) over it, the variable-node pass
// the reverse.
//
// The transform over (Z_2)^p is the radix-2 Walsh-Hadamard transform,
//     W(s) = sum_x (-1)^popcount(s & x) u(x),
// whose inverse is the same transform divided by q.  The check-node pass has
// two forms.  Distributed (q >= 8, check degree <= 8): a check vector is
// spread over G lanes of R elements each (element y = lane * R + r);
// butterflies on the bits of r run in registers, those on the lane bits
// through select-free half exchanges between partner lanes (one shuffle per
// two butterfly inputs, one FMA per output; see wht_sf).  Lane per edge
// (q <= 4, or a check of degree 9..32): one lane holds a whole vector and the
// permutation moves into the transform domain (see cnp_lane).
//
// Multiplication by a field constant is linear over GF(2), so the permuted
// index h^-1 (y0 ^ r) of a lane's R elements is h^-1 y0 ^ h^-1 r, and
// h^-1 r is the XOR of h^-1 2^b = x^(log h^-1 + b) over the bits b of r:
// log2(R) + 1 table reads per edge give all R gather (and scatter) indices.
#pragma once

#include <type_traits>

#include "mma_kernels.cuh"   // CodeBlob, ilog2, group_mask

namespace nbldpc {

// One code and the frames to decode with it.
struct FftJob {
  const unsigned char* blob;  // code description (device)
  CodeBlob off;
  const float* prob;          // [frames][n][q] channel probabilities p_n(x)
  uint8_t* out_sym;           // [frames][n]
  int32_t* out_iters;         // [frames]
  uint8_t* out_ok;            // [frames]
  float* out_app;             // [frames][n][q] normalized a-posteriori vectors, or null
  int q, n, m, frames, max_iters, early_stop;
  int ntasks;                 // warp tasks of the q <= 64 check-node pass (blob task_c0)
};

struct FftParams {
  FftJob job;
  unsigned int* counter;      // next frame
  float* msg;                 // message slots, one per block: [nnz][q] floats
  size_t slot_floats;
  int blob_cap, n_cap;        // shared-memory layout: blob, decisions, control word,
  int w_off;                  // then (q <= 64, 256-byte aligned) the transformed vectors, 32 * q floats per warp
};

// Elements per lane and block size of the distributed check-node form at
// q = 64 and q = 128, and the largest q with select-based half-exchange lane
// stages where the select-free form is switched off (compile-time tuning
// knobs; the defaults are the measured best on GB300, with select-based lane
// stages: GF(64) (2,4) N=576: 4 elements / 768 threads 1.19 Gbit/s, 8 / 768
// 0.97, 16 / 512 0.72, 2 / 1024 1.05, 4 / 896 1.08; GF(128) (2,4) N=256: 4
// elements 0.81, 8 elements 0.71).
#ifndef NBLDPC_FFT_R64
#define NBLDPC_FFT_R64 4
#endif
#ifndef NBLDPC_FFT_T64
#define NBLDPC_FFT_T64 768
#endif
#ifndef NBLDPC_FFT_R128
#define NBLDPC_FFT_R128 4
#endif
#ifndef NBLDPC_FFT_HALF_MAXQ
#define NBLDPC_FFT_HALF_MAXQ 64
#endif

template <int Q_> struct FftGeo {
  static constexpr int Q = Q_;
  static constexpr int LQ = ilog2(Q);                 // p
  static constexpr int PB = LQ > 0 ? LQ : 1;          // basis images per coefficient
  static constexpr int R = Q < 8 ? (Q < 4 ? Q : 4)
                                  : (Q <= 64 ? NBLDPC_FFT_R64 : (Q == 128 ? NBLDPC_FFT_R128 : 8));   // elements per lane
  static constexpr int RB = ilog2(R);
  static constexpr int G = Q / R;                     // lanes per check vector (1..32)
};

// Variable-node lanes: RV elements of a vector per lane, VG lanes per vector
// (1..32).  8-element lanes for q >= 64 shorten the shuffle reductions
// (decision, normalization) by one stage; column degree 2 only (with 4 the
// register arrays of the pass no longer fit 80 registers).
template <int Q, int DV> struct VnpGeo {
  static constexpr int Q_ = Q;
  static constexpr int RV = Q <= 4 ? Q : ((Q >= 64 && DV <= 2) ? 8 : (Q / 32 > 4 ? Q / 32 : 4));
  static constexpr int VG = Q / RV;
};

// Walsh-Hadamard butterflies over the R register elements: the pair (a, b)
// at register indices (r, r + h) becomes (a + b, a - b).
template <class g>
__device__ __forceinline__ void wht_regs(float (&v)[g::R]) {
#pragma unroll
  for (int h = 1; h < g::R; h <<= 1) {
#pragma unroll
    for (int r = 0; r < g::R; ++r) {
      if (!(r & h)) {
        const float a = v[r], b = v[r + h];
        v[r] = a + b;
        v[r + h] = a - b;
      }
    }
  }
}

// Select-based lane stages (lane_stage, lane_stage_full, wht_fwd, wht_inv):
// the forms for field orders above NBLDPC_FFT_SELECT_FREE_MAXQ, a tuning knob
// that by default gives every field the select-free form.
//
// Butterfly over lane bit k by half exchanges: the lanes of a pair (gl, gl ^ 2^k)
// hold the same register indices of the two elements of each butterfly; the
// lower lane keeps registers with bit c = 2^(k mod RB) clear and sends the
// others, the upper lane the reverse, so one shuffle moves two butterfly
// inputs and each lane then computes both outputs of the butterflies it
// holds: low = keep + recv (a + b), high = +-(keep - recv) (a - b, exact).
// Afterwards register bit c carries the element's lane bit k and lane bit k the
// element's register bit c; applying the stages k = 0..K-1 and later
// K-1..0 restores the layout (the products between the transforms are
// element-wise, so they see the same layout for every edge).
template <class g>
__device__ __forceinline__ void lane_stage(float (&v)[g::R], int k, int gl, unsigned gmask) {
  const int o = 1 << k;
  const int c = 1 << (k % g::RB);
  const bool up = (gl & o) != 0;
  const float sg = up ? -1.f : 1.f;
#pragma unroll
  for (int r = 0; r < g::R; ++r) {
    if (r & c) continue;
    const float send = up ? v[r] : v[r | c];
    const float keep = up ? v[r | c] : v[r];
    const float recv = __shfl_xor_sync(gmask, send, o);
    v[r] = keep + recv;
    v[r | c] = sg * (keep - recv);
  }
}

// Butterfly over lane bit k with every element shuffled: the upper lane of
// the pair computes partner - own, the lower own + partner (layout unchanged).
// Taken above NBLDPC_FFT_HALF_MAXQ: at q >= 128 the selects of the
// select-based half exchange cost more than the shuffles they save (measured
// on GB300: GF(256) -8 % with half exchanges; GF(16) +7 %, GF(8) / GF(64)
// +1 %, GF(32) -1 %).  The select-free form beats both (GF(128) 811 -> 887
// Mbit/s, GF(256) 550 -> 556 against this one).
template <class g>
__device__ __forceinline__ void lane_stage_full(float (&v)[g::R], int k, int gl, unsigned gmask) {
  const int o = 1 << k;
  const float sg = (gl & o) ? -1.f : 1.f;
#pragma unroll
  for (int r = 0; r < g::R; ++r) {
    const float t = __shfl_xor_sync(gmask, v[r], o);
    v[r] = fmaf(sg, v[r], t);
  }
}

template <class g> struct HalfExchange { static constexpr bool v = g::Q <= NBLDPC_FFT_HALF_MAXQ; };

// forward transform: register bits, then lane bits 0..K-1 (natural layout in,
// exchanged layout out)
template <class g>
__device__ __forceinline__ void wht_fwd(float (&v)[g::R], int gl, unsigned gmask) {
  wht_regs<g>(v);
#pragma unroll
  for (int k = 0; (1 << k) < g::G; ++k) {
    if constexpr (HalfExchange<g>::v) lane_stage<g>(v, k, gl, gmask);
    else lane_stage_full<g>(v, k, gl, gmask);
  }
}

// inverse (unnormalized) transform: register bits, then lane bits K-1..0
// (exchanged layout in, natural layout out)
template <class g>
__device__ __forceinline__ void wht_inv(float (&v)[g::R], int gl, unsigned gmask) {
  wht_regs<g>(v);
#pragma unroll
  for (int k = g::LQ - g::RB - 1; k >= 0; --k) {
    if constexpr (HalfExchange<g>::v) lane_stage<g>(v, k, gl, gmask);
    else lane_stage_full<g>(v, k, gl, gmask);
  }
}

// ---- select-free butterflies (half exchanges for q >= 8, R = 4 or 8)
// Every butterfly is computed as
//     out_lo = recv + x * keep,   out_hi = recv - x * keep        (one FMA each)
// into registers (r, r | c), with x = +-1 a per-lane constant of the stage.
// In a lane stage both lanes of a pair keep register r and send register
// r | c: the upper lane holds its elements with register bit c relabelled, so
// the half exchange needs no selects.  A stored value is then a sign times
// the transform element at some index; which output gets the sum (the sign
// of x) is chosen per lane so that each stage leaves the relabelling the next
// stage on the same register bit needs, and the signs follow.  Layout and
// signs depend on the field order only, so a compile-time run of the stages
// (make_fft_signs) gives the lanes whose coefficient is -1 at every stage
// and the signs of the inverse outputs (folded into the final 1/q scale).
// The inverse starts from the forward signs raised to the number of factors of
// the product, odd here (check-degree buckets 4 and 8), i.e. the forward
// signs themselves; its outputs are back in natural order (element
// lane * R + r in register r).
struct FftSigns {
  uint32_t fwd[8];   // forward stage s (RB register stages, then lane stages 0..K-1): bit gl = coefficient -1
  uint32_t inv[8];   // inverse stage s (RB register stages, then lane stages K-1..0)
  uint32_t out[8];   // register r: bit gl = the inverse output in register r of lane gl is the negated element
  bool ok;           // every stage paired single-bit index pairs, coefficients independent of r, natural order out
};

// One butterfly on (keep, recv) = (sign, index) pairs with the sum placed in
// out_lo when eps = +1, in out_hi when eps = -1; returns x = eps * s_recv * s_keep.
__host__ __device__ constexpr int sf_bfly(int ik, int sk, int ir, int sr, int eps, int& ilo, int& slo, int& ihi,
                                          int& shi, bool& ok) {
  const int t = ik ^ ir;
  if (t == 0 || (t & (t - 1)) != 0) ok = false;
  const int lo = ik < ir ? ik : ir, hi = lo | t;
  // recv + e * x * keep carries sign s_recv; it is the sum for e = eps, the
  // difference (index hi) for e = -eps, negated when recv is the upper element
  const bool recv_lo = ir == lo;
  ilo = lo; slo = sr;                                 // e = eps: the sum
  ihi = hi; shi = recv_lo ? sr : -sr;                 // e = -eps: the difference
  if (eps < 0) {                                      // sum into out_hi
    const int ti = ilo, ts = slo;
    ilo = ihi; slo = shi; ihi = ti; shi = ts;
  }
  return eps * sr * sk;
}

template <int Q, int R> __host__ __device__ constexpr FftSigns make_fft_signs() {
  constexpr int G = Q / R;
  int RB = 0, LQ = 0;
  while ((1 << RB) < R) ++RB;
  while ((1 << LQ) < Q) ++LQ;
  const int K = LQ - RB;
  FftSigns T{};
  T.ok = G >= 2 && K >= 1 && RB + K <= 8;
  int idx[Q] = {}, sg[Q] = {}, ni[Q] = {}, ns[Q] = {};
  int m0[G] = {};           // initial relabelling: bit c_k of lane gl is bit k of gl, k < RB
  for (int gl = 0; gl < G; ++gl)
    for (int k = 0; k < K && k < RB; ++k) m0[gl] |= ((gl >> k) & 1) << (k % RB);
  for (int gl = 0; gl < G; ++gl)
    for (int p = 0; p < R; ++p) { idx[gl * R + p] = (gl << RB) | (p ^ m0[gl]); sg[gl * R + p] = 1; }
  // one stage: register stage (lane_stage false, bit b) or lane stage (bit k);
  // the eps rule picks, per lane, where the sum goes
  for (int pass = 0; pass < 2; ++pass) {
    for (int st = 0; st < RB + K; ++st) {
      const bool lane_st = st >= RB;
      const int b = st;                                         // register stage bit
      const int k = !lane_st ? 0 : (pass == 0 ? st - RB : K - 1 - (st - RB));   // lane stage lane bit
      const int c = lane_st ? 1 << (k % RB) : 1 << b;
      uint32_t& mask = pass == 0 ? T.fwd[st] : T.inv[st];
      for (int i = 0; i < Q; ++i) { ni[i] = idx[i]; ns[i] = sg[i]; }
      for (int gl = 0; gl < G; ++gl) {
        int xl = 0;
        for (int r = 0; r < R; ++r) {
          if (r & c) continue;
          const int kp = gl * R + r;
          const int rp = lane_st ? (gl ^ (1 << k)) * R + (r | c) : gl * R + (r | c);
          int eps = 1;
          if (!lane_st) {
            // keep the relabelling: the sum goes to the slot of the lower index
            eps = idx[kp] < idx[rp] ? 1 : -1;
          } else if (pass == 0) {
            // relabel register bit c for its next use: lane stage k + RB, else the inverse's stage k
            const int nxt = k + RB < K ? k + RB : k;
            eps = ((gl >> nxt) & 1) ? -1 : 1;
          } else {
            // inverse: relabel for lane stage k - RB, natural order after the last use
            eps = (k - RB >= 0 && ((gl >> (k - RB)) & 1)) ? -1 : 1;
          }
          int ilo = 0, slo = 0, ihi = 0, shi = 0;
          const int x = sf_bfly(idx[kp], sg[kp], idx[rp], sg[rp], eps, ilo, slo, ihi, shi, T.ok);
          if (xl == 0) xl = x;
          else if (xl != x) T.ok = false;
          ni[kp] = ilo; ns[kp] = slo;
          ni[gl * R + (r | c)] = ihi; ns[gl * R + (r | c)] = shi;
        }
        if (xl < 0) mask |= 1u << gl;
      }
      for (int i = 0; i < Q; ++i) { idx[i] = ni[i]; sg[i] = ns[i]; }
    }
  }
  for (int i = 0; i < Q; ++i) {
    if (idx[i] != i) T.ok = false;
    if (sg[i] < 0) T.out[i % R] |= 1u << (i / R);
  }
  return T;
}

// Largest field order with select-free butterflies (compile-time knob; above
// it, q <= NBLDPC_FFT_HALF_MAXQ takes the select-based half exchange and larger
// fields one shuffle per element).
#ifndef NBLDPC_FFT_SELECT_FREE_MAXQ
#define NBLDPC_FFT_SELECT_FREE_MAXQ 256
#endif
template <class g> struct SelectFree {
  static constexpr bool v = (g::R == 4 || g::R == 8) && g::Q >= 8 && g::Q <= NBLDPC_FFT_SELECT_FREE_MAXQ;
  static constexpr FftSigns T = make_fft_signs<(v ? g::Q : 8), (v ? g::R : 4)>();
  static_assert(!v || T.ok, "select-free butterfly schedule");
};

template <int I, int N, class F> __device__ __forceinline__ void static_for(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>{});
    static_for<I + 1, N>(f);
  }
}

// +-1 for this lane from a mask of lanes (bit gl set: -1), a constant when
// every lane agrees.  A mask and its complement give the same value up to a
// sign (a free operand negation), so the value is formed from the member of
// the pair with lane 0 clear and equal classes share one register.
template <uint32_t MASK, int G> __device__ __forceinline__ float sf_coef(int gl) {
  constexpr uint32_t all = G >= 32 ? 0xFFFFFFFFu : (1u << G) - 1;
  constexpr uint32_t m = MASK & all, base = (m & 1u) ? (m ^ all) : m;
  constexpr float sign = (m & 1u) ? -1.f : 1.f;
  if constexpr (base == 0) return sign;
  else return sign * (((base >> gl) & 1) ? -1.f : 1.f);
}

template <class g, bool INV>
__device__ __forceinline__ void wht_sf(float (&v)[g::R], int gl, unsigned gmask) {
  constexpr FftSigns T = SelectFree<g>::T;
  constexpr int RB = g::RB, K = g::LQ - g::RB;
  static_for<0, RB>([&](auto S) {
    constexpr int b = decltype(S)::value, h = 1 << b;
    const float x = sf_coef<INV ? T.inv[b] : T.fwd[b], g::G>(gl);
#pragma unroll
    for (int r = 0; r < g::R; ++r) {
      if (r & h) continue;
      const float keep = v[r], recv = v[r | h];
      v[r] = fmaf(x, keep, recv);
      v[r | h] = fmaf(-x, keep, recv);
    }
  });
  static_for<0, K>([&](auto S) {
    constexpr int s = decltype(S)::value;
    constexpr int k = INV ? K - 1 - s : s, c = 1 << (k % RB);
    const float x = sf_coef<INV ? T.inv[RB + s] : T.fwd[RB + s], g::G>(gl);
#pragma unroll
    for (int r = 0; r < g::R; ++r) {
      if (r & c) continue;
      const float keep = v[r];
      const float recv = __shfl_xor_sync(gmask, v[r | c], 1 << k);
      v[r] = fmaf(x, keep, recv);
      v[r | c] = fmaf(-x, keep, recv);
    }
  });
}

// idx[r] = h^-1 (y0 ^ r) for the lane's elements y0 ^ r (y0 = lane * R), from
// log h^-1 (lhinv) and log y0 (ly0, unused when y0 = 0).
template <class g>
__device__ __forceinline__ void perm_index(int (&idx)[g::R], const uint8_t* exp2, int lhinv, int ly0, bool y0nz) {
  idx[0] = y0nz ? exp2[ly0 + lhinv] : 0;
#pragma unroll
  for (int b = 0; b < g::RB; ++b) {
    const int hb = exp2[lhinv + b];                  // h^-1 x^b
#pragma unroll
    for (int r = 0; r < (1 << b); ++r) idx[(1 << b) + r] = idx[r] ^ hb;
  }
}

template <int N> __device__ __forceinline__ void load_vec(const float* p, float (&v)[N]) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int i = 0; i < N / 4; ++i) {
      const float4 t = reinterpret_cast<const float4*>(p)[i];
      v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
    }
  } else if constexpr (N == 2) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x; v[1] = t.y;
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = p[i];
  }
}

template <int N> __device__ __forceinline__ void store_vec(float* p, const float (&v)[N]) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int i = 0; i < N / 4; ++i)
      reinterpret_cast<float4*>(p)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
  } else if constexpr (N == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) p[i] = v[i];
  }
}

// z / sum(z) over the VG lanes of a variable vector; the uniform vector 1/q
// when the sum is not positive.  Every lane sees the same sum (the shuffle
// tree adds the same pairs on every lane, in commuted order).
template <class g>
__device__ __forceinline__ void normalize_vec(float (&z)[g::RV], unsigned vmask) {
  static_assert(g::Q_ >= 2, "variable-node geometry");
  float s = 0.f;
#pragma unroll
  for (int r = 0; r < g::RV; ++r) s += z[r];
#pragma unroll
  for (int o = 1; o < g::VG; o <<= 1) s += __shfl_xor_sync(vmask, s, o);
  if (s > 0.f) {
    const float inv = __frcp_rn(s);
    if (isfinite(inv)) {
#pragma unroll
      for (int r = 0; r < g::RV; ++r) z[r] *= inv;
    } else {          // sum below the reciprocal's range: divide
#pragma unroll
      for (int r = 0; r < g::RV; ++r) z[r] = __fdiv_rn(z[r], s);
    }
  } else {
#pragma unroll
    for (int r = 0; r < g::RV; ++r) z[r] = 1.f / g::Q_;
  }
}


// ---------------------------------------------------------------- q <= 64: one lane per edge
// The lane-per-edge check-node pass (q <= 64) keeps a whole message vector in one lane's
// registers, so both transforms run without shuffles, and applies the
// coefficient permutations in the transform domain.  With M_c the GF(2)-linear
// map "multiply by c" (column k = c x^k), the transform of a permuted vector
// is the permuted transform:
//     WHT(u o M_c^-1)(s) = WHT(u)(M_c^T s),
// so with W_j = WHT(u_j) (natural order) the check node's output is
//     v'_n = WHT^-1(P_n),  P_n(s) = prod over j != n of W_j(M_{h_j / h_n}^T s).
// M_c^T s is the XOR of the basis images M_c^T e_i over the bits i of s
// (at_log[log c][i]); walking s in Gray-code order updates the index with one
// XOR per element.  W_j sits in shared memory (one 256-byte row per lane for
// q = 64, 16-byte chunks XOR-swizzled by the lane against bank conflicts),
// the message rows in global memory are read and written whole.
__host__ __device__ constexpr int ctz_c(int k) {
  int b = 0;
  while (k > 1 && !(k & 1)) { k >>= 1; ++b; }
  return b;
}

// all p butterfly stages in registers
template <int Q> __device__ __forceinline__ void wht_full(float (&v)[Q]) {
#pragma unroll
  for (int h = 1; h < Q; h <<= 1) {
#pragma unroll
    for (int r = 0; r < Q; ++r) {
      if (!(r & h)) {
        const float a = v[r], b = v[r + h];
        v[r] = a + b;
        v[r + h] = a - b;
      }
    }
  }
}

// 16-byte-chunk swizzle of a lane's row (element positions XOR swz)
template <int Q> __device__ __forceinline__ int row_swz(int lane) {
  if constexpr (Q >= 8) return (lane & (Q / 4 - 1)) << 2;
  else return 0;
}

// The block's dynamic shared memory (code blob, decisions, control word,
// transformed vectors), addressed by byte offset.
extern __shared__ __align__(16) unsigned char fft_smem[];

// acc[s] (=|*=) row[(M s) ^ swz] for s = 0..Q-1 in Gray-code order: step K
// visits s = K ^ (K >> 1), which differs from the previous s in bit ctz(K),
// so the element's byte offset changes by XOR with a4[ctz(K)] = 4 M e_ctz(K).
// `cur` starts at the row's byte offset XOR 4 swz (rows are aligned to their
// length, so XOR within the row is addition).
template <int Q, bool FIRST, int K = 0>
__device__ __forceinline__ void gray_gather(float (&acc)[Q], const int (&a4)[ilog2(Q) > 0 ? ilog2(Q) : 1], int cur) {
  if constexpr (K > 0) {
    constexpr int b = ctz_c(K);
    cur ^= a4[b];
  }
  constexpr int sk = K ^ (K >> 1);
  const float x = *reinterpret_cast<const float*>(fft_smem + cur);
  if constexpr (FIRST) acc[sk] = x; else acc[sk] *= x;
  if constexpr (K + 1 < Q) gray_gather<Q, FIRST, K + 1>(acc, a4, cur);
}

// ---------------------------------------------------------------- one frame
// DC >= every check degree (register arrays of the distributed check-node
// pass), or DC = 0: the lane-per-edge check-node pass (q <= 64, check degree
// <= 32); DV >= every column degree.
template <class g, int DC, int DV>
__device__ __forceinline__ void fft_decode_frame(const FftJob& job, int frame, float* X, const unsigned char* sblob,
                                                 uint8_t* chat, float* wsm) {
  using vg = VnpGeo<g::Q, DV>;
  constexpr int Q = g::Q, R = g::R, RV = vg::RV;
  const uint8_t* exp2 = sblob + job.off.exp2;        // x^(i mod (q-1)), i < 2(q-1)
  const uint8_t* glog = sblob + job.off.log;         // log_x(v), v >= 1
  const uint16_t* row_ptr = reinterpret_cast<const uint16_t*>(sblob + job.off.row_ptr);
  const uint16_t* edge_col = reinterpret_cast<const uint16_t*>(sblob + job.off.edge_col);
  const uint8_t* edge_lh = sblob + job.off.edge_lh;    // log_x(h) of each edge
  const uint8_t* edge_lhi = sblob + job.off.edge_lhi;  // log_x(h^-1) of each edge
  const uint16_t* vn_ptr = reinterpret_cast<const uint16_t*>(sblob + job.off.vn_ptr);
  const uint16_t* vn_edge = reinterpret_cast<const uint16_t*>(sblob + job.off.vn_edge);
  const uint16_t* edge_row = reinterpret_cast<const uint16_t*>(sblob + job.off.edge_row);
  const uint16_t* task_c0 = reinterpret_cast<const uint16_t*>(sblob + job.off.task_c0);
  const uint8_t* at_log = sblob + job.off.at_log;

  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
  const int grp = tid / g::G, ngroups = nthr / g::G, gl = tid % g::G;
  const unsigned gmask = group_mask<g::G>(lane);
  const int y0 = gl * R;
  const bool y0nz = y0 != 0;
  const int ly0 = y0nz ? glog[y0] : 0;
  const int vgrp = tid / vg::VG, nvgroups = nthr / vg::VG, vgl = tid % vg::VG;
  const unsigned vmask = group_mask<vg::VG>(lane);
  const float* pf = job.prob + (size_t)frame * job.n * Q;
  float* app = job.out_app ? job.out_app + (size_t)frame * job.n * Q : nullptr;

  // ---- variable-node pass (Alg. 1, VNP and decision):
  //   z_e(x) = p(x) prod over the other edges of v'(x), u_e = z_e / sum z_e
  //   c = argmax_x p(x) prod over all edges of v'(x)   (lowest symbol on ties)
  auto vnp = [&](bool first, bool want_u) {
    for (int vn = vgrp; vn < job.n; vn += nvgroups) {
      float pv[RV], T[RV];
      load_vec<RV>(pf + (size_t)vn * Q + vgl * RV, pv);
#pragma unroll
      for (int r = 0; r < RV; ++r) T[r] = pv[r];
      const int k0 = vn_ptr[vn], dv = vn_ptr[vn + 1] - k0;
      float V[DV][RV];
#pragma unroll
      for (int a = 0; a < DV; ++a) {
        if (!first && a < dv) {
          load_vec<RV>(X + (size_t)vn_edge[k0 + a] * Q + vgl * RV, V[a]);
#pragma unroll
          for (int r = 0; r < RV; ++r) T[r] *= V[a][r];
        } else {
#pragma unroll
          for (int r = 0; r < RV; ++r) V[a][r] = 1.f;
        }
      }
      float bv = T[0];
      int bi = vgl * RV;
#pragma unroll
      for (int r = 1; r < RV; ++r)
        if (T[r] > bv) { bv = T[r]; bi = vgl * RV + r; }
#pragma unroll
      for (int o = 1; o < vg::VG; o <<= 1) {
        const float ov = __shfl_xor_sync(vmask, bv, o);
        const int oi = __shfl_xor_sync(vmask, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
      }
      if (vgl == 0) chat[vn] = (uint8_t)bi;
      if (app) {
        normalize_vec<vg>(T, vmask);
        store_vec<RV>(app + (size_t)vn * Q + vgl * RV, T);
      }
      if (!first && want_u) {
#pragma unroll
        for (int a = 0; a < DV; ++a) {
          if (a < dv) {
            float z[RV];
#pragma unroll
            for (int r = 0; r < RV; ++r) {
              float t = pv[r];
#pragma unroll
              for (int b = 0; b < DV; ++b)
                if (b != a) t *= V[b][r];
              z[r] = t;
            }
            normalize_vec<vg>(z, vmask);
            store_vec<RV>(X + (size_t)vn_edge[k0 + a] * Q + vgl * RV, z);
          }
        }
      }
    }
  };

  // ---- syndrome of chat over all checks (block-wide)
  auto syndrome_ok = [&]() -> bool {
    int bad = 0;
    for (int r = tid; r < job.m; r += nthr) {
      int sy = 0;
      for (int e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
        const int c = chat[edge_col[e]];
        if (c) sy ^= exp2[glog[c] + edge_lh[e]];
      }
      bad |= sy;
    }
    return __syncthreads_or(bad) == 0;
  };


  // ---- check-node pass for q <= 64 (Alg. 1: permutation, FFT, product,
  // inverse FFT, depermutation), one lane per edge, warp tasks of whole checks
  auto cnp_lane = [&](bool first) {
    if constexpr (DC == 0 && Q <= 64) {
    constexpr int P = g::PB;
    const int warp = tid >> 5, nwarps = nthr >> 5;
    const int w_row0 = (int)(reinterpret_cast<unsigned char*>(wsm) - fft_smem);   // byte offset, 256-aligned
    float* wrow = wsm + ((size_t)warp * 32 + lane) * Q;        // this lane's transformed vector
    const int swz = row_swz<Q>(lane);
    for (int t = warp; t < job.ntasks; t += nwarps) {
      const int eb = row_ptr[task_c0[t]], ee = row_ptr[task_c0[t + 1]];
      const int e = eb + lane;
      const bool valid = e < ee;
      if (valid) {
        float v[Q];
        load_vec<Q>(first ? pf + (size_t)edge_col[e] * Q : X + (size_t)e * Q, v);   // u^(0) = p
        wht_full<Q>(v);                                                            // W_e = FFT(u_e)
        if constexpr (Q >= 4) {
#pragma unroll
          for (int c = 0; c < Q / 4; ++c)
            reinterpret_cast<float4*>(wrow)[c ^ (swz >> 2)] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
        } else {
#pragma unroll
          for (int i = 0; i < Q; ++i) wrow[i] = v[i];
        }
      }
      __syncwarp();
      if (valid) {
        const int r = edge_row[e], e0 = row_ptr[r], d = row_ptr[r + 1] - e0, n = e - e0;
        const int lhn = edge_lh[e];
        // basis images (byte offsets) of M^T for c = h_j / h_n, and the start offset of lane j's row
        auto setup = [&](int j, int (&a4)[P]) {
          int lc = edge_lh[e0 + j] - lhn;
          if (lc < 0) lc += Q - 1;
#pragma unroll
          for (int b = 0; b < P; ++b) a4[b] = 4 * at_log[lc * g::LQ + b];
          const int lj = lane - n + j;
          return (w_row0 + (warp * 32 + lj) * Q * 4) ^ (4 * row_swz<Q>(lj));
        };
        float acc[Q];
        const int jfirst = n == 0 ? 1 : 0;
        {
          int a4[P];
          const int cur = setup(jfirst, a4);
          gray_gather<Q, true>(acc, a4, cur);
        }
        for (int j = jfirst + 1; j < d; ++j) {
          if (j == n) continue;
          int a4[P];
          const int cur = setup(j, a4);
          gray_gather<Q, false>(acc, a4, cur);
        }
        wht_full<Q>(acc);                                                          // inverse FFT (times q)
#pragma unroll
        for (int i = 0; i < Q; ++i) acc[i] = fmaxf(acc[i] * (1.f / Q), 0.f);       // v'_e, rounding below 0 -> 0
        store_vec<Q>(X + (size_t)e * Q, acc);
      }
      __syncwarp();
    }
    }
  };

  // ---- check-node pass (Alg. 1: permutation, FFT, product, inverse FFT,
  // depermutation), one group of G lanes per check
  auto cnp = [&](bool first) {
    if constexpr (DC > 0) {
    constexpr bool SF = SelectFree<g>::v;
    constexpr FftSigns T = SelectFree<g>::T;
    static_assert(!SF || DC % 2 == 0, "the select-free inverse expects an odd number of product factors");
    // select-free form: the lane gathers its elements with the initial relabelling
    // (register bit k carries lane bit k, k < RB) and scales its outputs by +-1/q
    constexpr int RL = (g::LQ - g::RB) < g::RB ? (g::LQ - g::RB) : g::RB;
    const int y0s = SF ? (y0 ^ (gl & ((1 << RL) - 1))) : y0;
    const bool y0snz = y0s != 0;
    const int ly0s = y0snz ? glog[y0s] : 0;
    for (int r = grp; r < job.m; r += ngroups) {
      const int e0 = row_ptr[r], d = row_ptr[r + 1] - e0;
      float W[DC][R];
      // absent edges (d < DC) enter the product as the transform of the unit
      // vector at 0, all ones; in the select-free form an odd number of them
      // must carry the forward output signs (one such factor, the others 1)
      float pad[R];
#pragma unroll
      for (int i = 0; i < R; ++i) pad[i] = 1.f;
      if constexpr (SF) {
        if (d < DC && ((DC - d) & 1)) {
#pragma unroll
          for (int i = 0; i < R; ++i) pad[i] = (y0s == 0 && i == 0) ? 1.f : 0.f;
          wht_sf<g, false>(pad, gl, gmask);
        }
      }
#pragma unroll
      for (int j = 0; j < DC; ++j) {
        if (j < d) {
          const int e = e0 + j;
          int idx[R];
          perm_index<g>(idx, exp2, edge_lhi[e], ly0s, y0snz);
          // u'_j(y) = u_j(h_j^-1 y); u^(0) = p on the first pass
          const float* src = first ? pf + (size_t)edge_col[e] * Q : X + (size_t)e * Q;
#pragma unroll
          for (int i = 0; i < R; ++i) W[j][i] = src[idx[i]];
          if constexpr (SF) wht_sf<g, false>(W[j], gl, gmask);
          else wht_fwd<g>(W[j], gl, gmask);
        } else {
#pragma unroll
          for (int i = 0; i < R; ++i) W[j][i] = j == d ? pad[i] : 1.f;
        }
      }
#pragma unroll
      for (int j = 0; j < DC; ++j) {
        if (j < d) {
          float v[R];
#pragma unroll
          for (int i = 0; i < R; ++i) {
            float t = 1.f;
#pragma unroll
            for (int k = 0; k < DC; ++k)
              if (k != j) t *= W[k][i];
            v[i] = t;
          }
          if constexpr (SF) wht_sf<g, true>(v, gl, gmask);
          else wht_inv<g>(v, gl, gmask);
          const int e = e0 + j;
          int idx[R];
          perm_index<g>(idx, exp2, edge_lhi[e], ly0, y0nz);
          // v'_j(h_j^-1 y) = v_j(y): inverse transform / q, negative rounding -> 0
          float* dst = X + (size_t)e * Q;
          static_for<0, R>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const float t = SF ? v[i] * sf_coef<T.out[i], g::G>(gl) : v[i];
            dst[idx[i]] = fmaxf(t * (1.f / Q), 0.f);
          });
        }
      }
    }
    }
  };

  // ---- decode one frame
  vnp(true, false);                                  // c^(0) = argmax p
  __syncthreads();
  bool ok = syndrome_ok();
  int iters = 0;
  if (!(job.early_stop && ok)) {
    for (int k = 1; k <= job.max_iters; ++k) {
      if constexpr (DC == 0) cnp_lane(k == 1); else cnp(k == 1);
      __syncthreads();
      vnp(false, k < job.max_iters);
      __syncthreads();
      iters = k;
      ok = syndrome_ok();
      if (job.early_stop && ok) break;
    }
  }
  for (int i = tid; i < job.n; i += nthr) job.out_sym[(size_t)frame * job.n + i] = chat[i];
  if (tid == 0) {
    job.out_iters[frame] = iters;
    job.out_ok[frame] = ok ? 1 : 0;
  }
}

// ---------------------------------------------------------------- the kernel
// Threads of one block: one frame per SM, as many warps as the register
// arrays allow (80 registers per thread: 24 warps; 128: 16 warps; q = 64
// holds two 64-float vectors per lane).  A single
// frame's message slot per SM (nnz * q floats, 295 KB for GF(64) N=576) keeps
// the resident message state of the whole GPU inside L2.
template <int Q, int DC, int DV> struct FftThreads {
  static constexpr int v = DC == 0 ? (Q == 64 ? 512 : 768)
                                   : (Q == 64 ? NBLDPC_FFT_T64 : ((DC <= 4 && Q < 256) ? 768 : 512));
};

// Persistent blocks, one frame at a time; DC / DV bound the check and column
// degrees of the code (register arrays of the two passes).
template <int Q, int DC, int DV>
__global__ void __launch_bounds__(FftThreads<Q, DC, DV>::v, 1) fftspa_decode_kernel(const __grid_constant__ FftParams p) {
  unsigned char* smem = fft_smem;
  unsigned char* sblob = smem;
  uint8_t* chat = smem + p.blob_cap;
  volatile int* ctl = reinterpret_cast<volatile int*>(smem + p.blob_cap + p.n_cap);
  const FftJob& job = p.job;
  float* X = p.msg + (size_t)blockIdx.x * p.slot_floats;
  float* wsm = reinterpret_cast<float*>(smem + p.w_off);
  for (int i = threadIdx.x; i < job.off.fft_bytes / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(sblob)[i] = reinterpret_cast<const uint4*>(job.blob)[i];
  for (;;) {
    if (threadIdx.x == 0) ctl[0] = (int)atomicAdd(p.counter, 1u);
    __syncthreads();
    const int frame = ctl[0];
    if (frame >= job.frames) break;
    fft_decode_frame<FftGeo<Q>, DC, DV>(job, frame, X, sblob, chat, wsm);
    __syncthreads();
  }
}

}  // namespace nbldpc
