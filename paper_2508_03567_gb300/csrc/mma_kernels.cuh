// Min-max (MMA) decoding of non-binary LDPC codes over GF(2^p): device code
// for sm_103a.  One persistent block decodes one frame at a time, running the
// flooding schedule of Alg. 2 (check-node F/B/beta pass, variable-node pass,
// decision and syndrome) until the syndrome is zero or I_max is reached, then
// takes the next frame from a global counter.
//
// Message vectors (q reliabilities in 0..255) travel between the passes as q
// bytes per Tanner-graph edge in a per-block global slot that stays resident
// in L1/L2.  Inside the check-node pass a vector lives in shared memory as q
// 16-bit lanes packed two per 32-bit word ("pair layout", below), so that the
// min-max convolution runs on packed max.u16x2 / min.u16x2 instructions.
//
// Min-max convolution (Alg. 2, F/B/beta equations, with the coefficient
// permutation applied to the inputs):
//     C(x) = min over y of max(A(y), B(x ^ y)),   x, y in GF(2^p).
// A group of G lanes computes one convolution.  With x = xh*DN + l and
// y = yh*DN + (l ^ d), the lane-offset d runs over DN = 2^LB values and each
// lane keeps XN = 2^XB outputs in registers; A values reach lane l from lane
// l^d through shfl.xor, and the B values a lane needs for offset d are
// B(j*DN + d), j = xh ^ yh, held in registers, so no dynamic register
// indexing is needed.  SB high lane bits split the y range further; their
// partial minima are combined by a shuffle reduce-scatter at the end.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace nbldpc {

// ---------------------------------------------------------------- primitives
__device__ __forceinline__ uint32_t vmax2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ uint32_t vmin2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}
__device__ __forceinline__ uint32_t swap16(uint32_t a) { return __byte_perm(a, 0, 0x1032); }

// ---------------------------------------------------------------- geometry
// LB: lane bits of the shuffle offset d; SB: lane bits splitting y.
template <int Q> struct Layout;
template <> struct Layout<2>   { static constexpr int LB = 0, SB = 0; };
template <> struct Layout<4>   { static constexpr int LB = 1, SB = 0; };
template <> struct Layout<8>   { static constexpr int LB = 1, SB = 1; };
template <> struct Layout<16>  { static constexpr int LB = 2, SB = 1; };
template <> struct Layout<32>  { static constexpr int LB = 2, SB = 2; };
template <> struct Layout<64>  { static constexpr int LB = 3, SB = 2; };
template <> struct Layout<128> { static constexpr int LB = 4, SB = 1; };
template <> struct Layout<256> { static constexpr int LB = 5, SB = 0; };

constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }

template <int Q> struct Geo {
  static constexpr int P = ilog2(Q);
  static constexpr int LB = Layout<Q>::LB, SB = Layout<Q>::SB;
  static constexpr int XB = P - LB;             // register bits of x
  static constexpr int TB = XB - SB;            // register bits of y
  static constexpr int G = 1 << (LB + SB);      // lanes per group
  static constexpr int DN = 1 << LB;            // shuffle offsets
  static constexpr int XN = 1 << XB;            // accumulators per lane
  static constexpr int AW = 1 << (TB - 1);      // packed A words per lane
  static constexpr int KW = XN / 2;             // packed B words per offset
  static constexpr int DC = (DN * KW <= 32) ? DN : 32 / KW;  // offsets per B chunk
  static constexpr int W = Q / 2;               // packed words per vector
  static constexpr int BPL = Q / G;             // bytes per lane in byte-wise passes
  static constexpr int VB = (2 * Q + 15) / 16 * 16;  // bytes per packed vector in smem
  static_assert(TB >= 1 && XB == SB + TB, "layout");
  static_assert(AW * G == W, "own words cover the vector");
  static_assert(BPL == 2 || BPL == 4 || BPL == 8, "byte lanes");
};

// Pair layout: word w = kk*DN + vl holds v0 = 2*kk*DN + vl (low 16 bits) and
// v0 + DN (high 16 bits).  Index of value v as a 16-bit element:
template <int Q> __device__ __forceinline__ int pair_index(int v) {
  using g = Geo<Q>;
  const int word = ((v >> (g::LB + 1)) << g::LB) | (v & (g::DN - 1));
  return 2 * word + ((v >> g::LB) & 1);
}

// ---------------------------------------------------------------- convolution
// C = A (*) B in pair layout; s, l: lane coordinates inside the group.
// Inputs and output must not alias.  Caller syncs the group afterwards.
template <int Q>
__device__ __forceinline__ void mm_conv(const uint32_t* __restrict__ A, const uint32_t* __restrict__ B,
                                        uint32_t* __restrict__ C, int s, int l, unsigned gmask) {
  using g = Geo<Q>;
  uint32_t aown[g::AW];
#pragma unroll
  for (int u = 0; u < g::AW; ++u) aown[u] = A[(s * g::AW + u) * g::DN + l];
  uint32_t acc[g::XN];
#pragma unroll
  for (int x = 0; x < g::XN; ++x) acc[x] = 0xFFFFFFFFu;

#pragma unroll
  for (int c0 = 0; c0 < g::DN; c0 += g::DC) {
    uint32_t bl[g::DC][g::KW];
#pragma unroll
    for (int k = 0; k < g::KW; ++k) {
      const uint32_t* row = B + (k ^ (s * g::AW)) * g::DN + c0;
      if constexpr (g::DC % 4 == 0) {
#pragma unroll
        for (int dd = 0; dd < g::DC; dd += 4) {
          const uint4 v = *reinterpret_cast<const uint4*>(row + dd);
          bl[dd][k] = v.x; bl[dd + 1][k] = v.y; bl[dd + 2][k] = v.z; bl[dd + 3][k] = v.w;
        }
      } else if constexpr (g::DC % 2 == 0) {
#pragma unroll
        for (int dd = 0; dd < g::DC; dd += 2) {
          const uint2 v = *reinterpret_cast<const uint2*>(row + dd);
          bl[dd][k] = v.x; bl[dd + 1][k] = v.y;
        }
      } else {
#pragma unroll
        for (int dd = 0; dd < g::DC; ++dd) bl[dd][k] = row[dd];
      }
    }
#pragma unroll
    for (int dd = 0; dd < g::DC; ++dd) {
      const int d = c0 + dd;
      uint32_t a[g::AW], as[g::AW];
#pragma unroll
      for (int u = 0; u < g::AW; ++u) {
        a[u] = (d == 0) ? aown[u] : __shfl_xor_sync(gmask, aown[u], d);
        as[u] = swap16(a[u]);
      }
#pragma unroll
      for (int xh = 0; xh < g::XN; ++xh)
#pragma unroll
        for (int u = 0; u < g::AW; ++u)
          acc[xh] = vmin2(acc[xh], vmax2((xh & 1) ? as[u] : a[u], bl[dd][(xh >> 1) ^ u]));
    }
  }
  // Reduce-scatter over the SB lane bits: afterwards slot r holds x-block
  // xh = s * 2^TB + r.
#pragma unroll
  for (int b = g::SB - 1; b >= 0; --b) {
    const int c = g::TB + b;
    const bool sb = (s >> b) & 1;
#pragma unroll
    for (int x0 = 0; x0 < (1 << c); ++x0) {
      const uint32_t send = sb ? acc[x0] : acc[x0 + (1 << c)];
      const uint32_t keep = sb ? acc[x0 + (1 << c)] : acc[x0];
      const uint32_t recv = __shfl_xor_sync(gmask, send, 1 << (g::LB + b));
      acc[x0] = vmin2(keep, recv);
    }
  }
#pragma unroll
  for (int r = 0; r < g::AW; ++r) {
    const uint32_t e = acc[2 * r], o = acc[2 * r + 1];
    C[(s * g::AW + r) * g::DN + l] = vmin2(__byte_perm(e, o, 0x5410), __byte_perm(e, o, 0x7632));
  }
}

// ---------------------------------------------------------------- parameters
struct CodeBlob {           // offsets (bytes) into the code blob
  int exp2, log, row_ptr, edge_col, edge_lh, vn_ptr, vn_edge, bytes;
};

struct DecodeParams {
  const uint8_t* gamma;     // [frames][n][q]
  uint8_t* out_sym;         // [frames][n]
  int32_t* out_iters;       // [frames]
  uint8_t* out_ok;          // [frames]
  uint8_t* msg;             // per-block message slots
  unsigned int* counter;    // next frame
  const unsigned char* blob;
  CodeBlob off;
  size_t slot_bytes;
  int n, m, nnz, dmax;
  int frames, max_iters, early_stop;
  int group_bytes;          // per-group shared scratch
};

template <int Q> __host__ __device__ constexpr int group_scratch_bytes(int dmax) {
  return ((dmax * Q + 15) / 16) * 16 + (2 * dmax + 3) * Geo<Q>::VB;
}

template <int BPL> __device__ __forceinline__ void load_bytes(const uint8_t* p, int (&v)[BPL]) {
  if constexpr (BPL == 2) {
    const uint32_t w = *reinterpret_cast<const uint16_t*>(p);
    v[0] = w & 0xFF; v[1] = w >> 8;
  } else if constexpr (BPL == 4) {
    const uint32_t w = *reinterpret_cast<const uint32_t*>(p);
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = (w >> (8 * i)) & 0xFF;
  } else {
    const uint2 w = *reinterpret_cast<const uint2*>(p);
#pragma unroll
    for (int i = 0; i < 4; ++i) { v[i] = (w.x >> (8 * i)) & 0xFF; v[i + 4] = (w.y >> (8 * i)) & 0xFF; }
  }
}

template <int BPL> __device__ __forceinline__ void store_bytes(uint8_t* p, const int (&v)[BPL]) {
  if constexpr (BPL == 2) {
    *reinterpret_cast<uint16_t*>(p) = (uint16_t)(v[0] | (v[1] << 8));
  } else if constexpr (BPL == 4) {
    *reinterpret_cast<uint32_t*>(p) = (uint32_t)(v[0] | (v[1] << 8) | (v[2] << 16) | (v[3] << 24));
  } else {
    uint2 w;
    w.x = (uint32_t)(v[0] | (v[1] << 8) | (v[2] << 16) | (v[3] << 24));
    w.y = (uint32_t)(v[4] | (v[5] << 8) | (v[6] << 16) | (v[7] << 24));
    *reinterpret_cast<uint2*>(p) = w;
  }
}

template <int G> __device__ __forceinline__ int group_min(int v, unsigned gmask) {
#pragma unroll
  for (int o = 1; o < G; o <<= 1) v = min(v, __shfl_xor_sync(gmask, v, o));
  return v;
}

template <int G> __device__ __forceinline__ void group_sync(unsigned gmask) {
  if constexpr (G > 1) __syncwarp(gmask);
}

// ---------------------------------------------------------------- the kernel
template <int Q>
__global__ void __launch_bounds__(256) mma_decode_kernel(const DecodeParams p) {
  using g = Geo<Q>;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* sblob = smem;
  uint8_t* chat = smem + p.off.bytes;                                    // [n]
  __shared__ unsigned int s_frame;
  unsigned char* scratch_base = smem + p.off.bytes + ((p.n + 15) / 16) * 16;

  // stage the code description (GF tables, H, variable-node view)
  for (int i = threadIdx.x; i < p.off.bytes / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(sblob)[i] = reinterpret_cast<const uint4*>(p.blob)[i];
  __syncthreads();
  const uint8_t* exp2 = sblob + p.off.exp2;        // x^(i mod (q-1)), i < 2(q-1)
  const uint8_t* glog = sblob + p.off.log;         // log_x(v), v >= 1
  const uint16_t* row_ptr = reinterpret_cast<const uint16_t*>(sblob + p.off.row_ptr);
  const uint16_t* edge_col = reinterpret_cast<const uint16_t*>(sblob + p.off.edge_col);
  const uint8_t* edge_lh = sblob + p.off.edge_lh;  // log_x(h) of each edge
  const uint16_t* vn_ptr = reinterpret_cast<const uint16_t*>(sblob + p.off.vn_ptr);
  const uint16_t* vn_edge = reinterpret_cast<const uint16_t*>(sblob + p.off.vn_edge);

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int grp = tid / g::G, ngroups = blockDim.x / g::G;
  const int gl = tid % g::G;
  const unsigned gmask = (g::G == 32) ? 0xFFFFFFFFu : (((1u << g::G) - 1u) << (lane & ~(g::G - 1)));
  const int s = gl >> g::LB, l = gl & (g::DN - 1);

  unsigned char* gs = scratch_base + (size_t)grp * p.group_bytes;
  uint8_t* stage = gs;                                                   // [dmax][q] bytes
  unsigned char* vecs = gs + ((p.dmax * Q + 15) / 16) * 16;
  auto vec = [&](int i) { return reinterpret_cast<uint32_t*>(vecs + (size_t)i * g::VB); };
  // vectors: P_j = vec(j), F_j = vec(dmax + j), Bv[2] = vec(2dmax), vec(2dmax+1), R = vec(2dmax+2)
  uint8_t* X = p.msg + (size_t)blockIdx.x * p.slot_bytes;

  const int qm1 = Q - 1;

  for (;;) {
    if (tid == 0) s_frame = atomicAdd(p.counter, 1u);
    __syncthreads();
    const int frame = (int)s_frame;
    if (frame >= p.frames) break;
    const uint8_t* gam = p.gamma + (size_t)frame * p.n * Q;

    // ---- variable-node pass: S = gamma + sum beta, decision, alpha = sat(S - beta - min)
    auto vnp = [&](bool first, bool want_alpha) {
      for (int vn = grp; vn < p.n; vn += ngroups) {
        int S[g::BPL];
        load_bytes<g::BPL>(gam + (size_t)vn * Q + gl * g::BPL, S);
        const int k0 = vn_ptr[vn], k1 = vn_ptr[vn + 1];
        if (!first) {
          for (int k = k0; k < k1; ++k) {
            int b[g::BPL];
            load_bytes<g::BPL>(X + (size_t)vn_edge[k] * Q + gl * g::BPL, b);
#pragma unroll
            for (int i = 0; i < g::BPL; ++i) S[i] += b[i];
          }
        }
        int key = 0x7FFFFFFF;
#pragma unroll
        for (int i = 0; i < g::BPL; ++i) key = min(key, (S[i] << 8) | (gl * g::BPL + i));
        key = group_min<g::G>(key, gmask);
        if (gl == 0) chat[vn] = (uint8_t)(key & 0xFF);
        if (!first && want_alpha) {
          for (int k = k0; k < k1; ++k) {
            uint8_t* row = X + (size_t)vn_edge[k] * Q + gl * g::BPL;
            int t[g::BPL];
            load_bytes<g::BPL>(row, t);
            int mn = 0x7FFFFFFF;
#pragma unroll
            for (int i = 0; i < g::BPL; ++i) { t[i] = S[i] - t[i]; mn = min(mn, t[i]); }
            mn = group_min<g::G>(mn, gmask);
#pragma unroll
            for (int i = 0; i < g::BPL; ++i) t[i] = min(255, t[i] - mn);
            store_bytes<g::BPL>(row, t);
          }
        }
      }
    };

    // ---- syndrome of chat over all checks (block-wide)
    auto syndrome_ok = [&]() -> bool {
      int bad = 0;
      for (int r = tid; r < p.m; r += blockDim.x) {
        int sy = 0;
        for (int e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
          const int c = chat[edge_col[e]];
          if (c) sy ^= exp2[glog[c] + edge_lh[e]];
        }
        bad |= sy;
      }
      return __syncthreads_or(bad) == 0;
    };

    // ---- check-node pass (F, B, beta) for every check, one group per check
    auto cnp = [&](bool first) {
      for (int r = grp; r < p.m; r += ngroups) {
        const int e0 = row_ptr[r], d = row_ptr[r + 1] - e0;
        // stage incoming alpha rows (alpha^(0) = gamma on the first pass)
        if constexpr (Q >= 16) {
          constexpr int CH = Q / 16;
          for (int i = gl; i < d * CH; i += g::G) {
            const int j = i / CH, c = i % CH;
            const uint8_t* src = first ? gam + (size_t)edge_col[e0 + j] * Q : X + (size_t)(e0 + j) * Q;
            reinterpret_cast<uint4*>(stage + j * Q)[c] = reinterpret_cast<const uint4*>(src)[c];
          }
        } else {
          for (int i = gl; i < d * Q; i += g::G) {
            const int j = i / Q, c = i % Q;
            const uint8_t* src = first ? gam + (size_t)edge_col[e0 + j] * Q : X + (size_t)(e0 + j) * Q;
            stage[i] = src[c];
          }
        }
        group_sync<g::G>(gmask);
        // permutation: P_j(y) = alpha_j(h_j^-1 y), stored in pair layout
        for (int j = 0; j < d; ++j) {
          const int lhinv = (qm1 - edge_lh[e0 + j]) % qm1;
          const uint8_t* a = stage + j * Q;
          uint32_t* P = vec(j);
#pragma unroll
          for (int u = 0; u < g::AW; ++u) {
            const int w = gl + u * g::G;
            const int kk = w >> g::LB, vl = w & (g::DN - 1);
            const int v0 = (kk << (g::LB + 1)) | vl, v1 = v0 | g::DN;
            const int s0 = v0 ? exp2[glog[v0] + lhinv] : 0;
            const int s1 = exp2[glog[v1] + lhinv];
            P[w] = (uint32_t)a[s0] | ((uint32_t)a[s1] << 16);
          }
        }
        group_sync<g::G>(gmask);
        // beta_j(a) = R_j(h_j a), written over the edge's message row
        auto depermute = [&](const uint32_t* Rv, int e) {
          const uint16_t* R16 = reinterpret_cast<const uint16_t*>(Rv);
          const int lh = edge_lh[e];
          int out[g::BPL];
#pragma unroll
          for (int i = 0; i < g::BPL; ++i) {
            const int a = gl * g::BPL + i;
            const int v = a ? exp2[glog[a] + lh] : 0;
            out[i] = R16[pair_index<Q>(v)];
          }
          store_bytes<g::BPL>(X + (size_t)e * Q + gl * g::BPL, out);
        };
        // forward: F_0 = P_0, F_j = F_{j-1} (*) P_j
        const uint32_t* Fprev = vec(0);
        for (int j = 1; j <= d - 2; ++j) {
          mm_conv<Q>(Fprev, vec(j), vec(p.dmax + j), s, l, gmask);
          group_sync<g::G>(gmask);
          Fprev = vec(p.dmax + j);
        }
        depermute(Fprev, e0 + d - 1);                      // beta_{d-1} from F_{d-2}
        // backward: B_{d-1} = P_{d-1}; beta_j from F_{j-1} (*) B_{j+1}; B_j = B_{j+1} (*) P_j
        const uint32_t* Bcur = vec(d - 1);
        int pp = 0;
        for (int j = d - 2; j >= 1; --j) {
          const uint32_t* Fj = (j == 1) ? vec(0) : vec(p.dmax + j - 1);
          uint32_t* R = vec(2 * p.dmax + 2);
          mm_conv<Q>(Fj, Bcur, R, s, l, gmask);
          group_sync<g::G>(gmask);
          depermute(R, e0 + j);
          uint32_t* Bn = vec(2 * p.dmax + pp);
          mm_conv<Q>(Bcur, vec(j), Bn, s, l, gmask);
          group_sync<g::G>(gmask);
          Bcur = Bn;
          pp ^= 1;
        }
        depermute(Bcur, e0);                               // beta_0 from B_1
        group_sync<g::G>(gmask);
      }
    };

    // ---- decode one frame
    vnp(true, false);                // c^(0) = argmin gamma
    __syncthreads();
    bool ok = syndrome_ok();
    int iters = 0;
    if (!(p.early_stop && ok)) {
      for (int k = 1; k <= p.max_iters; ++k) {
        cnp(k == 1);
        __syncthreads();
        vnp(false, k < p.max_iters);
        __syncthreads();
        iters = k;
        ok = syndrome_ok();
        if (p.early_stop && ok) break;
      }
    }
    for (int i = tid; i < p.n; i += blockDim.x) p.out_sym[(size_t)frame * p.n + i] = chat[i];
    if (tid == 0) {
      p.out_iters[frame] = iters;
      p.out_ok[frame] = ok ? 1 : 0;
    }
    __syncthreads();
  }
}

}  // namespace nbldpc
