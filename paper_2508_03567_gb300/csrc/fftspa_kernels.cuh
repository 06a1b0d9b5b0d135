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
// whose inverse is the same transform divided by q.  A check vector is spread
// over G lanes of R elements each (element y = lane * R + r): butterflies on
// the bits of r run in registers, those on the lane bits through shuffles.
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
};

struct FftParams {
  FftJob job;
  unsigned int* counter;      // next frame
  float* msg;                 // message slots, one per block: [nnz][q] floats
  size_t slot_floats;
  int blob_cap, n_cap;        // shared-memory layout: blob, decisions, control word
};

template <int Q_> struct FftGeo {
  static constexpr int Q = Q_;
  static constexpr int R = Q < 8 ? Q : 8;             // check-vector elements per lane
  static constexpr int RB = ilog2(R);
  static constexpr int G = Q / R;                     // lanes per check vector (1..32)
  static constexpr int RV = Q <= 4 ? Q : (Q / 32 > 4 ? Q / 32 : 4);   // variable-vector elements per lane
  static constexpr int VG = Q / RV;                   // lanes per variable vector (1..32)
};

// Walsh-Hadamard butterflies over the R register elements (index bits
// 0..RB-1) then the G lanes of the group (bits RB..p-1): the pair
// (a, b) at indices (x, x + 2^k) becomes (a + b, a - b).
template <class g>
__device__ __forceinline__ void wht(float (&v)[g::R], int gl, unsigned gmask) {
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
#pragma unroll
  for (int o = 1; o < g::G; o <<= 1) {
    const float sg = (gl & o) ? -1.f : 1.f;   // upper index: partner - own
#pragma unroll
    for (int r = 0; r < g::R; ++r) {
      const float t = __shfl_xor_sync(gmask, v[r], o);
      v[r] = fmaf(sg, v[r], t);
    }
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
    for (int r = 0; r < g::RV; ++r) z[r] = 1.f / g::Q;
  }
}

// ---------------------------------------------------------------- one frame
// DC >= every check degree, DV >= every column degree (register arrays).
template <class g, int DC, int DV>
__device__ __forceinline__ void fft_decode_frame(const FftJob& job, int frame, float* X, const unsigned char* sblob,
                                                 uint8_t* chat) {
  constexpr int Q = g::Q, R = g::R, RV = g::RV;
  const uint8_t* exp2 = sblob + job.off.exp2;        // x^(i mod (q-1)), i < 2(q-1)
  const uint8_t* glog = sblob + job.off.log;         // log_x(v), v >= 1
  const uint16_t* row_ptr = reinterpret_cast<const uint16_t*>(sblob + job.off.row_ptr);
  const uint16_t* edge_col = reinterpret_cast<const uint16_t*>(sblob + job.off.edge_col);
  const uint8_t* edge_lh = sblob + job.off.edge_lh;    // log_x(h) of each edge
  const uint8_t* edge_lhi = sblob + job.off.edge_lhi;  // log_x(h^-1) of each edge
  const uint16_t* vn_ptr = reinterpret_cast<const uint16_t*>(sblob + job.off.vn_ptr);
  const uint16_t* vn_edge = reinterpret_cast<const uint16_t*>(sblob + job.off.vn_edge);

  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
  const int grp = tid / g::G, ngroups = nthr / g::G, gl = tid % g::G;
  const unsigned gmask = group_mask<g::G>(lane);
  const int y0 = gl * R;
  const bool y0nz = y0 != 0;
  const int ly0 = y0nz ? glog[y0] : 0;
  const int vgrp = tid / g::VG, nvgroups = nthr / g::VG, vgl = tid % g::VG;
  const unsigned vmask = group_mask<g::VG>(lane);
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
      for (int o = 1; o < g::VG; o <<= 1) {
        const float ov = __shfl_xor_sync(vmask, bv, o);
        const int oi = __shfl_xor_sync(vmask, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
      }
      if (vgl == 0) chat[vn] = (uint8_t)bi;
      if (app) {
        normalize_vec<g>(T, vmask);
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
            normalize_vec<g>(z, vmask);
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

  // ---- check-node pass (Alg. 1: permutation, FFT, product, inverse FFT,
  // depermutation), one group of G lanes per check
  auto cnp = [&](bool first) {
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
          wht<g>(W[j], gl, gmask);
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
          wht<g>(v, gl, gmask);
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
  };

  // ---- decode one frame
  vnp(true, false);                                  // c^(0) = argmax p
  __syncthreads();
  bool ok = syndrome_ok();
  int iters = 0;
  if (!(job.early_stop && ok)) {
    for (int k = 1; k <= job.max_iters; ++k) {
      cnp(k == 1);
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
// arrays allow (80 registers per thread: 24 warps; 128: 16 warps).  A single
// frame's message slot per SM (nnz * q floats, 295 KB for GF(64) N=576) keeps
// the resident message state of the whole GPU inside L2.
template <int Q, int DC, int DV> struct FftThreads {
  static constexpr int v = (DC <= 4 && Q < 256) ? 768 : 512;
};

// Persistent blocks, one frame at a time; DC / DV bound the check and column
// degrees of the code (register arrays of the two passes).
template <int Q, int DC, int DV>
__global__ void __launch_bounds__(FftThreads<Q, DC, DV>::v, 1) fftspa_decode_kernel(const __grid_constant__ FftParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* sblob = smem;
  uint8_t* chat = smem + p.blob_cap;
  volatile int* ctl = reinterpret_cast<volatile int*>(smem + p.blob_cap + p.n_cap);
  const FftJob& job = p.job;
  float* X = p.msg + (size_t)blockIdx.x * p.slot_floats;
  for (int i = threadIdx.x; i < job.off.bytes / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(sblob)[i] = reinterpret_cast<const uint4*>(job.blob)[i];
  for (;;) {
    if (threadIdx.x == 0) ctl[0] = (int)atomicAdd(p.counter, 1u);
    __syncthreads();
    const int frame = ctl[0];
    if (frame >= job.frames) break;
    fft_decode_frame<FftGeo<Q>, DC, DV>(job, frame, X, sblob, chat);
    __syncthreads();
  }
}

}  // namespace nbldpc
