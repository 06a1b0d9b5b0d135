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
// through half exchanges between partner lanes (q <= 64: one shuffle per two
// butterfly inputs) or one shuffle per element (q >= 128).  Lane per edge
// (q <= 4, or a check of degree 9..32): one lane holds a whole vector and the
// permutation moves into the transform domain (see cnp_lane).
//
// Multiplication by a field constant is linear over GF(2), so the permuted
// index h^-1 (y0 ^ r) of a lane's R elements is h^-1 y0 ^ h^-1 r, and
// h^-1 r is the XOR of h^-1 2^b = x^(log h^-1 + b) over the bits b of r:
// log2(R) + 1 table reads per edge give all R gather (and scatter) indices.
#pragma once

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
// q = 64 and q = 128, and the largest q with half-exchange lane stages
// (compile-time tuning knobs; the defaults are the measured best on GB300:
// GF(64) (2,4) N=576: 4 elements / 768 threads 1.19 Gbit/s, 8 / 768 0.97,
// 16 / 512 0.72, 2 / 1024 1.05, 4 / 896 1.08; GF(128) (2,4) N=256: 4
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
// Used for q >= 128, where the selects of the half exchange cost more than
// the shuffles they save (measured on GB300: GF(256) -8 % with half
// exchanges; GF(16) +7 %, GF(8) / GF(64) +1 %, GF(32) -1 %).
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
    for (int r = grp; r < job.m; r += ngroups) {
      const int e0 = row_ptr[r], d = row_ptr[r + 1] - e0;
      float W[DC][R];
#pragma unroll
      for (int j = 0; j < DC; ++j) {
        if (j < d) {
          const int e = e0 + j;
          int idx[R];
          perm_index<g>(idx, exp2, edge_lhi[e], ly0, y0nz);
          // u'_j(y) = u_j(h_j^-1 y); u^(0) = p on the first pass
          const float* src = first ? pf + (size_t)edge_col[e] * Q : X + (size_t)e * Q;
#pragma unroll
          for (int i = 0; i < R; ++i) W[j][i] = src[idx[i]];
          wht_fwd<g>(W[j], gl, gmask);
        } else {
#pragma unroll
          for (int i = 0; i < R; ++i) W[j][i] = 1.f;   // transform of the unit vector at 0
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
          wht_inv<g>(v, gl, gmask);
          const int e = e0 + j;
          int idx[R];
          perm_index<g>(idx, exp2, edge_lhi[e], ly0, y0nz);
          // v'_j(h_j^-1 y) = v_j(y): inverse transform / q, negative rounding -> 0
          float* dst = X + (size_t)e * Q;
#pragma unroll
          for (int i = 0; i < R; ++i) dst[idx[i]] = fmaxf(v[i] * (1.f / Q), 0.f);
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
