// Min-max (MMA) decoding of non-binary LDPC codes over GF(2^p): device code
// for sm_103a.  One persistent block decodes one frame at a time, running the
// flooding schedule of Alg. 2 (check-node F/B/beta pass, variable-node pass,
// decision and syndrome) until the syndrome is zero or I_max is reached, then
// takes the next frame from a global counter.
//
// Message vectors (q reliabilities in 0..255) travel between the passes as q
// bytes per Tanner-graph edge in a per-block global slot that stays resident
// in L1/L2.  Inside the check-node pass a vector lives in shared memory as q
// 16-bit values, so that the min-max convolution (see mm_conv) runs on packed
// max.u16x2 / min.u16x2 instructions, two symbols per instruction; the
// variable-node pass also works on 16-bit pairs held in 32-bit registers.
//
// Min-max convolution (Alg. 2, F/B/beta equations, with the coefficient
// permutation applied to the inputs):
//     C(x) = min over y of max(A(y), B(x ^ y)),   x, y in GF(2^p).
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

// max of two packed pairs on the FMA pipe instead of the ALU pipe:
// max(a, b) = b + relu(a - b).  The operands are 16-bit integers 0..255; read
// as fp16 they are subnormal numbers (k * 2^-24), whose differences and sums
// below 2^11 are exact in fp16, so the result is the integer maximum bit for
// bit.  Used for part of the maxima so the two pipes share the work.
__device__ __forceinline__ uint32_t vmax2_fma(uint32_t a, uint32_t b) {
  uint32_t t, d;
  const uint32_t neg1 = 0xBC00BC00u;   // (-1.0, -1.0) in f16x2
  asm("fma.rn.relu.f16x2 %0, %1, %2, %3;" : "=r"(t) : "r"(b), "r"(neg1), "r"(a));
  asm("add.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(t), "r"(b));
  return d;
}

// ---------------------------------------------------------------- geometry
// Bytes of one variable node's q-byte rows that each lane of the variable-node
// pass handles (q / VBPL lanes per node).  Wide lanes put several nodes in
// flight per warp and shorten the shuffle reductions; measured on GB300 the
// 4-byte lanes of GF(64) left that pass latency-bound (8 bytes: +10 %, 16
// bytes: +3 % more).
#ifndef NBLDPC_VBPL_64
#define NBLDPC_VBPL_64 16
#endif
#ifndef NBLDPC_VBPL_256
#define NBLDPC_VBPL_256 16
#endif
template <int Q> struct VnpBytes {
  static constexpr int v = Q == 2 ? 2 : Q == 4 ? 4 : Q == 8 ? 8 : Q == 64 ? NBLDPC_VBPL_64
                         : Q == 256 ? NBLDPC_VBPL_256 : 8;
};

// LB: lane bits of x (the shuffle offset d runs over them); SB: lane bits that
// split the register part of y between lanes.  XB = p - LB register bits of x
// per lane, TB = XB - SB register bits of y per lane.  Each field order has
// two layouts (variant 0 and 1: two ways of splitting the q x q work between
// the lanes of a group and their registers); the autotuner picks one per code.
template <int Q, int V> struct Layout;
template <> struct Layout<2, 0>   { static constexpr int LB = 1, SB = 0; };
template <> struct Layout<2, 1>   { static constexpr int LB = 1, SB = 0; };
template <> struct Layout<4, 0>   { static constexpr int LB = 1, SB = 0; };
template <> struct Layout<4, 1>   { static constexpr int LB = 2, SB = 0; };
template <> struct Layout<8, 0>   { static constexpr int LB = 1, SB = 1; };
template <> struct Layout<8, 1>   { static constexpr int LB = 2, SB = 0; };
template <> struct Layout<16, 0>  { static constexpr int LB = 2, SB = 1; };
template <> struct Layout<16, 1>  { static constexpr int LB = 3, SB = 0; };
template <> struct Layout<32, 0>  { static constexpr int LB = 2, SB = 2; };
template <> struct Layout<32, 1>  { static constexpr int LB = 3, SB = 1; };
template <> struct Layout<64, 0>  { static constexpr int LB = 3, SB = 2; };
template <> struct Layout<64, 1>  { static constexpr int LB = 3, SB = 1; };
template <> struct Layout<128, 0> { static constexpr int LB = 4, SB = 1; };
template <> struct Layout<128, 1> { static constexpr int LB = 5, SB = 0; };
template <> struct Layout<256, 0> { static constexpr int LB = 5, SB = 0; };
template <> struct Layout<256, 1> { static constexpr int LB = 4, SB = 1; };

constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }

// bytes of one 16-bit message vector in shared memory (NBLDPC_VPAD: padding
// that shifts consecutive vectors to other banks)
#ifndef NBLDPC_VPAD
#define NBLDPC_VPAD 0
#endif
template <int Q> __host__ __device__ constexpr int vec_bytes() { return (2 * Q + 15) / 16 * 16 + NBLDPC_VPAD; }

template <int Q_, int V_> struct Geo {
  static constexpr int Q = Q_, V = V_;
  static constexpr int P = ilog2(Q);
  static constexpr int LB = Layout<Q, V>::LB, SB = Layout<Q, V>::SB;
  static constexpr int XB = P - LB;             // register bits of x
  static constexpr int TB = XB - SB;            // register bits of y
  static constexpr int G = 1 << (LB + SB);      // lanes per convolution group
  static constexpr int DN = 1 << LB;            // x values per register slot (lane part)
  static constexpr int DS = DN / 2;             // shuffle steps (even offsets d = 2*ds)
  static constexpr int XN = 1 << XB;            // accumulators per lane
  static constexpr int AWN = 1 << TB;           // packed A words per lane
  static constexpr int DC = (DS * XN <= 32) ? DS : (32 / XN >= 1 ? 32 / XN : 1);  // steps per B chunk
  static constexpr int OPL = 1 << TB;           // outputs per lane
  static constexpr int W = Q / 2;               // 32-bit words per vector
  static constexpr int PW = (W + G - 1) / G;    // permutation words per lane
  static constexpr int BPL = Q / G;             // bytes per lane when a group writes q bytes
  static constexpr int VB = vec_bytes<Q>();     // bytes per 16-bit vector in smem
  // variable-node pass: VG lanes per variable node, VBPL bytes (VBPL/2 packed words) each
  static constexpr int VBPL = VnpBytes<Q>::v;
  static constexpr int VG = Q / VBPL;
  static constexpr int VW = VBPL / 2;
  static_assert(LB >= 1 && TB >= 0 && XB == SB + TB, "layout");
  static_assert(G <= 32 && G * OPL == Q, "group covers the field");
  static_assert(DS % DC == 0, "chunking");
  static_assert(BPL == 1 || BPL == 2 || BPL == 4 || BPL == 8, "byte lanes");
};

// Of the XN * AWN maxima of one shuffle step, FmaEighths eighths use
// vmax2_fma (the rest the ALU pipe, which also takes every minimum).  Measured
// on GB300: 3/8 is best for q <= 64 (GF(64) step: 5/16 435.6, 6/16 437.5,
// 7/16 434.9, 8/16 430.4 Mbit/s; again with the current frame decoder: 2/8
// and 4/8 2-3 % slower than 3/8); 3/8 for q >= 128 too since the
// convolution's chunk loop is rolled (GF(256) (2,6) N=384, layout 0: 0 to
// 5/8 at 162.2, 150.2, 145.0, 142.5, 148.7, 167.5 ms; before the loop was
// rolled 1/8 was best).
#ifndef NBLDPC_FMA_EIGHTHS
#define NBLDPC_FMA_EIGHTHS 3
#endif
#ifndef NBLDPC_FMA_EIGHTHS_WIDE
#define NBLDPC_FMA_EIGHTHS_WIDE 3
#endif
template <int Q> struct FmaEighths {
  static constexpr int v = Q >= 128 ? NBLDPC_FMA_EIGHTHS_WIDE : NBLDPC_FMA_EIGHTHS;
};
template <class g> struct FmaMax { static constexpr int v = (g::XN * g::AWN * FmaEighths<g::Q>::v) / 8; };

// Lane constants of the convolution, computed once per thread.
struct ConvLane {
  int a_off;      // word index of the lane's first packed A word
  uint32_t sel;   // byte_perm selector: identity, or swap of the 16-bit halves on odd lanes
  int c_off;      // 16-bit index of the lane's first output
};

template <class g> __device__ __forceinline__ ConvLane conv_lane(int s, int l) {
  ConvLane c;
  c.a_off = (((s << g::TB) * g::DN) + (l & ~1)) >> 1;
  c.sel = (l & 1) ? 0x1032u : 0x3210u;
  c.c_off = (s << g::TB) * g::DN + l;
  return c;
}

// ---------------------------------------------------------------- convolution
// C = A (*) B: C(x) = min_y max(A(y), B(x ^ y)); vectors are q 16-bit values
// in natural order (element v at 16-bit index v).  A group of G lanes; lane
// (s, l) owns x = xh * DN + l for the XN values of xh and the y values with
// register part yr in [s * 2^TB, (s + 1) * 2^TB).  A packed A word pairs the
// lane positions (l, l ^ 1), so offset d = 2*ds reaches lane positions l ^ d
// and l ^ d ^ 1 in one shuffle, and the matching B values B(j*DN + d),
// B(j*DN + d + 1) form one natural 32-bit word whatever the parity of x, read
// by all lanes from the same shared-memory address.  Accumulator slot r holds
// xh = r ^ (s << TB), which makes the B register index r ^ t independent of
// the lane and lets the final reduce-scatter keep and send fixed slots.
// Inputs and output must not alias; the caller syncs the group afterwards.
//
// When the shuffle steps span several chunks of B registers (q >= 128), the
// chunk loop is kept rolled (NBLDPC_CONV_ROLL): the fully unrolled q = 256
// convolution, inlined at each call site, no longer fits the instruction
// cache.  The rolled form starts the accumulators at the maximum and shuffles
// at offset 0 in the first step, so every step has the same code.
#ifndef NBLDPC_CONV_ROLL
#define NBLDPC_CONV_ROLL 1
#endif
template <class g> __device__ __forceinline__ void load_b_chunk(const uint32_t* __restrict__ B, int c0,
                                                                uint32_t (&bl)[g::DC][g::XN]) {
#pragma unroll
  for (int j = 0; j < g::XN; ++j) {
    const uint32_t* row = B + j * g::DS + c0;
    if constexpr (g::DC % 4 == 0) {
#pragma unroll
      for (int dd = 0; dd < g::DC; dd += 4) {
        const uint4 v = *reinterpret_cast<const uint4*>(row + dd);
        bl[dd][j] = v.x; bl[dd + 1][j] = v.y; bl[dd + 2][j] = v.z; bl[dd + 3][j] = v.w;
      }
    } else if constexpr (g::DC % 2 == 0) {
#pragma unroll
      for (int dd = 0; dd < g::DC; dd += 2) {
        const uint2 v = *reinterpret_cast<const uint2*>(row + dd);
        bl[dd][j] = v.x; bl[dd + 1][j] = v.y;
      }
    } else {
#pragma unroll
      for (int dd = 0; dd < g::DC; ++dd) bl[dd][j] = row[dd];
    }
  }
}

template <class g, bool FMA_MAX>
__device__ __forceinline__ void mm_conv(const uint32_t* __restrict__ A, const uint32_t* __restrict__ B,
                                        uint16_t* __restrict__ C, const ConvLane& ln, unsigned gmask) {
  uint32_t aown[g::AWN];
#pragma unroll
  for (int t = 0; t < g::AWN; ++t) aown[t] = __byte_perm(A[ln.a_off + t * g::DS], 0, ln.sel);
  uint32_t acc[g::XN];

  if constexpr (NBLDPC_CONV_ROLL && g::DS / g::DC > 1) {
#pragma unroll
    for (int r = 0; r < g::XN; ++r) acc[r] = 0xFFFFFFFFu;
#pragma unroll 1
    for (int c0 = 0; c0 < g::DS; c0 += g::DC) {
      uint32_t bl[g::DC][g::XN];
      load_b_chunk<g>(B, c0, bl);
#pragma unroll
      for (int dd = 0; dd < g::DC; ++dd) {
        const int d = 2 * (c0 + dd);
        uint32_t a[g::AWN];
#pragma unroll
        for (int t = 0; t < g::AWN; ++t) a[t] = __shfl_xor_sync(gmask, aown[t], d);
#pragma unroll
        for (int r = 0; r < g::XN; ++r)
#pragma unroll
          for (int t = 0; t < g::AWN; ++t) {
            const uint32_t m = (FMA_MAX && r * g::AWN + t < FmaMax<g>::v) ? vmax2_fma(a[t], bl[dd][r ^ t])
                                                                : vmax2(a[t], bl[dd][r ^ t]);
            acc[r] = vmin2(acc[r], m);
          }
      }
    }
  } else {
#pragma unroll
  for (int c0 = 0; c0 < g::DS; c0 += g::DC) {
    uint32_t bl[g::DC][g::XN];
    load_b_chunk<g>(B, c0, bl);
#pragma unroll
    for (int dd = 0; dd < g::DC; ++dd) {
      const int d = 2 * (c0 + dd);
      uint32_t a[g::AWN];
#pragma unroll
      for (int t = 0; t < g::AWN; ++t) a[t] = (d == 0) ? aown[t] : __shfl_xor_sync(gmask, aown[t], d);
#pragma unroll
      for (int r = 0; r < g::XN; ++r)
#pragma unroll
        for (int t = 0; t < g::AWN; ++t) {
          const uint32_t m = (FMA_MAX && r * g::AWN + t < FmaMax<g>::v) ? vmax2_fma(a[t], bl[dd][r ^ t])
                                                              : vmax2(a[t], bl[dd][r ^ t]);
          acc[r] = (d == 0 && t == 0) ? m : vmin2(acc[r], m);
        }
    }
  }
  }
  // reduce-scatter over the SB lane bits: keep slot r, receive the partner's r | 2^c
#pragma unroll
  for (int b = g::SB - 1; b >= 0; --b) {
    const int c = g::TB + b;
#pragma unroll
    for (int r = 0; r < (1 << c); ++r)
      acc[r] = vmin2(acc[r], __shfl_xor_sync(gmask, acc[r | (1 << c)], 1 << (g::LB + b)));
  }
#pragma unroll
  for (int r = 0; r < g::OPL; ++r) C[ln.c_off + r * g::DN] = (uint16_t)vmin2(acc[r], acc[r] >> 16);
}

// ---------------------------------------------------------------- pruned convolution
// The same C = A (*) B, visiting only the y that can decide a minimum.  For any
// bound T >= max_x C(x), a y with A(y) > T gives max(A(y), B(x ^ y)) > C(x) for
// every x, so C(x) = min over {y : A(y) <= T} of max(A(y), B(x ^ y)), and the
// same holds with the roles of A and B exchanged (C is symmetric in them).
// T is found in phases: the entries of the chosen side with value <= hi are
// folded in, M = max_x of the partial result is an upper bound of max_x C(x)
// (a partial minimum is never below the full one), and the phases stop as soon
// as M <= hi; otherwise hi moves towards M.  The result is C exactly, with no
// approximation; the work is the number of entries folded in, about
// 17 of 256 for the GF(256) decoder's vectors instead of 256.
//
// One group of 32 lanes (one warp, so every branch below is warp-uniform);
// lane L owns x = L * OPL + k (k < OPL), kept as OPL/2 packed pairs.  For
// y = L' * OPL + i, x ^ y = (L ^ L') * OPL + (k ^ i): one aligned vector load of
// block L ^ L' of the other side, and a permutation inside the block that
// depends only on i, which the unrolled loop over i makes static.
// tprev: prediction of max_x C(x) (the previous convolution's maximum); it
// picks the side with fewer entries below it and the first phase's bound.
// SW (q >= 128, else null): a scratch vector for the other side with the two
// halves of every word exchanged, so that the odd i read their block without
// permuting it.
// Returns max_x C(x); with folded non-null, adds the number of entries folded in
// (each entry is q pairs (x, y)).  Inputs and output must not alias.
#ifndef NBLDPC_PRUNE_BACK
#define NBLDPC_PRUNE_BACK 4          // first phase: hi = tprev - NBLDPC_PRUNE_BACK
#endif
#ifndef NBLDPC_PRUNE_UNROLL
#define NBLDPC_PRUNE_UNROLL 2        // entries folded in per loop step
#endif
#ifndef NBLDPC_PRUNE_FMA
#define NBLDPC_PRUNE_FMA 0           // eighths of the maxima on the FMA pipe
#endif
#ifndef NBLDPC_PRUNE_PHASES
#define NBLDPC_PRUNE_PHASES 6        // after this many phases hi jumps to M
#endif
template <int NW> __device__ __forceinline__ void load_words(const uint32_t* p, uint32_t (&w)[NW]) {
  if constexpr (NW == 4) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
  } else if constexpr (NW == 2) {
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    w[0] = v.x; w[1] = v.y;
  } else {
    w[0] = p[0];
  }
}

template <class g>
__device__ __forceinline__ int pr_conv(const uint32_t* __restrict__ A, const uint32_t* __restrict__ B,
                                       uint16_t* __restrict__ C, uint32_t* __restrict__ SW, int lane, int tprev,
                                       int* folded) {
  constexpr int OPL = g::Q / 32, NW = OPL / 2;
  static_assert(g::G == 32 && OPL >= 2 && NW <= 4, "one warp per convolution");
  uint32_t a[NW], b[NW];
  load_words<NW>(A + lane * NW, a);
  load_words<NW>(B + lane * NW, b);
  // side: fewer entries <= tprev.  Per 16-bit half, 0x8000 + t - v has bit 15
  // set exactly when v <= t (values and t below 2^15: no borrow between halves)
  const uint32_t kt = 0x80008000u + (uint32_t)tprev * 0x10001u;
  int ca = 0, cb = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    ca += __popc((kt - a[w]) & 0x80008000u);
    cb += __popc((kt - b[w]) & 0x80008000u);
  }
  ca = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)ca);
  cb = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)cb);
  const bool swap = cb < ca;
  const uint32_t* V = swap ? A : B;
  uint32_t u[NW];
  int left[OPL];                       // entry values still to fold in (0x10000 once folded)
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    u[w] = swap ? b[w] : a[w];
    left[2 * w] = (int)(u[w] & 0xFFFFu);
    left[2 * w + 1] = (int)(u[w] >> 16);
  }
  constexpr bool kSw = g::Q >= 128;
  if constexpr (kSw) {
    uint32_t t[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) t[w] = __byte_perm(swap ? a[w] : b[w], 0, 0x1032);
    if constexpr (NW == 4) *reinterpret_cast<uint4*>(SW + lane * NW) = make_uint4(t[0], t[1], t[2], t[3]);
    else *reinterpret_cast<uint2*>(SW + lane * NW) = make_uint2(t[0], t[1]);
    __syncwarp();
  }
  uint32_t acc[NW];
#pragma unroll
  for (int w = 0; w < NW; ++w) acc[w] = 0xFFFFFFFFu;
  int hi = max(tprev - NBLDPC_PRUNE_BACK, 0), M = 0;
  for (int phase = 1;; ++phase) {
    unsigned bal[OPL];
#pragma unroll
    for (int i = 0; i < OPL; ++i) {
      const bool p = left[i] <= hi;
      bal[i] = __ballot_sync(0xFFFFFFFFu, p);
      if (p) left[i] = 0x10000;
    }
#pragma unroll
    for (int i = 0; i < OPL; ++i) {
      unsigned m = bal[i];
      while (m) {
        // NBLDPC_PRUNE_UNROLL entries per step (a repeated entry changes no minimum)
        int lp[NBLDPC_PRUNE_UNROLL];
        lp[0] = __ffs(m) - 1;
        m &= m - 1;
#pragma unroll
        for (int k = 1; k < NBLDPC_PRUNE_UNROLL; ++k) {
          lp[k] = m ? __ffs(m) - 1 : lp[0];
          m &= m - 1;
        }
        uint32_t uy[NBLDPC_PRUNE_UNROLL], v[NBLDPC_PRUNE_UNROLL][NW];
#pragma unroll
        for (int k = 0; k < NBLDPC_PRUNE_UNROLL; ++k) {
          uy[k] = __byte_perm(__shfl_sync(0xFFFFFFFFu, u[i >> 1], lp[k]), 0, (i & 1) ? 0x3232 : 0x1010);
          load_words<NW>(((i & 1) && kSw ? SW : V) + (lane ^ lp[k]) * NW, v[k]);
        }
#pragma unroll
        for (int w = 0; w < NW; ++w)
#pragma unroll
          for (int k = 0; k < NBLDPC_PRUNE_UNROLL; ++k) {
            uint32_t t = v[k][w ^ (i >> 1)];
            if ((i & 1) && !kSw) t = __byte_perm(t, 0, 0x1032);
            acc[w] = vmin2(acc[w], (w * NBLDPC_PRUNE_UNROLL + k) * 8 < NBLDPC_PRUNE_FMA * NW * NBLDPC_PRUNE_UNROLL
                                       ? vmax2_fma(t, uy[k]) : vmax2(t, uy[k]));
          }
      }
    }
    uint32_t mx = acc[0];
#pragma unroll
    for (int w = 1; w < NW; ++w) mx = vmax2(mx, acc[w]);
    M = (int)__reduce_max_sync(0xFFFFFFFFu, max(mx & 0xFFFFu, mx >> 16));
    if (M <= hi || hi >= 0xFFFF) break;                     // (the second: every entry folded in)
    if (M == 0xFFFF) hi = 2 * hi + 8;                       // nothing folded in yet
    else if (phase >= NBLDPC_PRUNE_PHASES) hi = M;
    else hi = min(M, max(hi + 2, (hi + M + 1) >> 1));
  }
  if (folded) {               // folded entries carry 0x10000
    int f = 0;
#pragma unroll
    for (int i = 0; i < OPL; ++i) f += left[i] >> 16;
    *folded += (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)f);
  }
  uint32_t* c32 = reinterpret_cast<uint32_t*>(C) + lane * NW;
  if constexpr (NW == 4) *reinterpret_cast<uint4*>(c32) = make_uint4(acc[0], acc[1], acc[2], acc[3]);
  else if constexpr (NW == 2) *reinterpret_cast<uint2*>(c32) = make_uint2(acc[0], acc[1]);
  else c32[0] = acc[0];
  return M;
}

// ---------------------------------------------------------------- parameters
struct CodeBlob {           // offsets (bytes) into the code blob
  int exp2, log, row_ptr, edge_col, edge_lh, edge_lhi, vn_ptr, vn_edge, bytes;
  // FFT-SPA section, after `bytes` (the min-max kernels stage only [0, bytes)):
  // check of each edge, first check of each warp task, transposed-multiplication basis
  int edge_row, task_c0, at_log, fft_bytes;
};

// One code and the frames to decode with it.
struct JobDesc {
  const unsigned char* blob;  // code description (device)
  CodeBlob off;
  const uint8_t* gamma;       // [frames][n][q]
  uint8_t* out_sym;           // [frames][n]
  int32_t* out_iters;         // [frames]
  uint8_t* out_ok;            // [frames]
  int q, n, m, dmax, vmax;    // field order, columns, rows, largest row and column degree
  int variant;                // bit 0: layout; bit 2: pruned convolutions (q >= 128, mixed-code kernel)
  int key16;                  // (255 * (max column degree + 1) + 1) * q <= 65536: 16-bit argmin keys
  int group_bytes;            // per-group shared scratch for this code
  int frames, max_iters, early_stop;
  int item_begin;             // index of this job's first frame in the launch's work list
  unsigned long long* work;   // optional: adds the (x, y) pairs the convolutions visit (null: no count)
};

constexpr int kMaxJobs = 32;

// One launch: up to kMaxJobs jobs whose frames form one work list, served by
// persistent blocks of `fpb` frame slots each.
struct LaunchParams {
  JobDesc jobs[kMaxJobs];
  int njobs, total_items;
  unsigned int* counter;      // next work item
  uint8_t* msg;               // message slots, one per (block, frame slot)
  size_t slot_bytes;
  int fpb;                    // frame slots per block (blockDim / fpb threads each)
  int slot_smem;              // shared bytes per frame slot
  int blob_cap, n_cap;        // largest code blob and N among the jobs
  int xs_off;                 // resident launches: shared-memory offset of the slot's messages
  int static_items;           // 1: no more items than frame slots; slot s takes item s (no counter)
};

// Threads of a block whose frame keeps its messages in shared memory (two
// blocks per SM: the same 24 warps as three 256-thread blocks).
constexpr int kResidentThreads = 384;


// Check-node permutation by scatter from registers (8-bit messages, 16 <= q <=
// NBLDPC_SCATTER_MAXQ) instead of staging the incoming rows in shared memory
// and gathering them.
#ifndef NBLDPC_SCATTER_MAXQ
#define NBLDPC_SCATTER_MAXQ 256
#endif
template <int Q> __host__ __device__ constexpr bool scatter_perm(int mb) {
  return mb == 1 && Q >= 16 && Q <= NBLDPC_SCATTER_MAXQ;
}

// per-group shared scratch: the d incoming rows (q symbols of mb bytes each;
// not with the scatter permutation) and 2*dmax+1 16-bit vectors: P_0..P_{d-1},
// F_1..F_{d-2}, two B vectors and the middle beta R; q >= 128: one more, the
// pruned convolution's half-swapped copy of its second operand
template <int Q> __host__ __device__ constexpr int group_scratch_bytes(int dmax, int mb = 1) {
  return (scatter_perm<Q>(mb) ? 0 : ((dmax * Q * mb + 15) / 16) * 16) +
         (2 * dmax + 1 + (Q >= 128 ? 1 : 0)) * vec_bytes<Q>();
}

// named barrier over the threads of one frame slot (ids 1..fpb)
__device__ __forceinline__ void slot_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ int slot_sync_or(int id, int nthreads, int pred) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\t"
      "selp.s32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(pred), "r"(id), "r"(nthreads)
      : "memory");
  return r;
}

template <int N> __device__ __forceinline__ void store_bytes(uint8_t* p, const int (&v)[N]) {
  if constexpr (N == 1) {
    *p = (uint8_t)v[0];
  } else if constexpr (N == 2) {
    *reinterpret_cast<uint16_t*>(p) = (uint16_t)(v[0] | (v[1] << 8));
  } else if constexpr (N == 4) {
    *reinterpret_cast<uint32_t*>(p) = (uint32_t)(v[0] | (v[1] << 8) | (v[2] << 16) | (v[3] << 24));
  } else {
    uint2 w;
    w.x = (uint32_t)(v[0] | (v[1] << 8) | (v[2] << 16) | (v[3] << 24));
    w.y = (uint32_t)(v[4] | (v[5] << 8) | (v[6] << 16) | (v[7] << 24));
    *reinterpret_cast<uint2*>(p) = w;
  }
}

// NB bytes -> NB/2 words of two 16-bit values (byte 2i in the low half of word i)
template <int NB> __device__ __forceinline__ void load_pairs(const uint8_t* p, uint32_t (&w)[NB / 2]) {
  if constexpr (NB == 2) {
    w[0] = __byte_perm(*reinterpret_cast<const uint16_t*>(p), 0, 0x4140);
  } else if constexpr (NB == 4) {
    const uint32_t x = *reinterpret_cast<const uint32_t*>(p);
    w[0] = __byte_perm(x, 0, 0x4140); w[1] = __byte_perm(x, 0, 0x4342);
  } else if constexpr (NB == 8) {
    const uint2 x = *reinterpret_cast<const uint2*>(p);
    w[0] = __byte_perm(x.x, 0, 0x4140); w[1] = __byte_perm(x.x, 0, 0x4342);
    w[2] = __byte_perm(x.y, 0, 0x4140); w[3] = __byte_perm(x.y, 0, 0x4342);
  } else {
    const uint4 x = *reinterpret_cast<const uint4*>(p);
    w[0] = __byte_perm(x.x, 0, 0x4140); w[1] = __byte_perm(x.x, 0, 0x4342);
    w[2] = __byte_perm(x.y, 0, 0x4140); w[3] = __byte_perm(x.y, 0, 0x4342);
    w[4] = __byte_perm(x.z, 0, 0x4140); w[5] = __byte_perm(x.z, 0, 0x4342);
    w[6] = __byte_perm(x.w, 0, 0x4140); w[7] = __byte_perm(x.w, 0, 0x4342);
  }
}

// inverse of load_pairs (every 16-bit value must be <= 255)
template <int NB> __device__ __forceinline__ void store_pairs(uint8_t* p, const uint32_t (&w)[NB / 2]) {
  if constexpr (NB == 2) {
    *reinterpret_cast<uint16_t*>(p) = (uint16_t)__byte_perm(w[0], 0, 0x4420);
  } else if constexpr (NB == 4) {
    *reinterpret_cast<uint32_t*>(p) = __byte_perm(w[0], w[1], 0x6420);
  } else if constexpr (NB == 8) {
    uint2 x;
    x.x = __byte_perm(w[0], w[1], 0x6420);
    x.y = __byte_perm(w[2], w[3], 0x6420);
    *reinterpret_cast<uint2*>(p) = x;
  } else {
    uint4 x;
    x.x = __byte_perm(w[0], w[1], 0x6420);
    x.y = __byte_perm(w[2], w[3], 0x6420);
    x.z = __byte_perm(w[4], w[5], 0x6420);
    x.w = __byte_perm(w[6], w[7], 0x6420);
    *reinterpret_cast<uint4*>(p) = x;
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

template <int G> __device__ __forceinline__ unsigned group_mask(int lane) {
  return (G == 32) ? 0xFFFFFFFFu : (((1u << G) - 1u) << (lane & ~(G - 1)));
}

// ---------------------------------------------------------------- q = 4 in registers
// C(x) = min_y max(A(y), B(x ^ y)) on 4-symbol vectors held as two words of
// 16-bit values, (v0, v1) and (v2, v3): B ^ 1 swaps the halves of each word,
// B ^ 2 swaps the words.
__device__ __forceinline__ uint2 conv4(uint2 a, uint2 b) {
  const uint32_t a0 = __byte_perm(a.x, 0, 0x1010), a1 = __byte_perm(a.x, 0, 0x3232);
  const uint32_t a2 = __byte_perm(a.y, 0, 0x1010), a3 = __byte_perm(a.y, 0, 0x3232);
  const uint32_t s0 = __byte_perm(b.x, 0, 0x1032), s1 = __byte_perm(b.y, 0, 0x1032);
  return make_uint2(vmin2(vmin2(vmax2(a0, b.x), vmax2(a1, s0)), vmin2(vmax2(a2, b.y), vmax2(a3, s1))),
                    vmin2(vmin2(vmax2(a0, b.y), vmax2(a1, s1)), vmin2(vmax2(a2, b.x), vmax2(a3, s0))));
}


// ---------------------------------------------------------------- q = 4, one warp per frame
// A frame of a small GF(4) code (at most 32 checks of degree <= kW4Deg, columns
// of degree <= 2) decoded by one warp with no block barrier: lane r owns check r
// and keeps its edges' alpha and beta rows (4 bytes each) in registers; the
// permutation and de-permutation byte selectors and the GF(4) products of its
// edges are set up once per frame; beta goes to the slot's message area (one
// word per edge) only for the variable-node step of the other edge's owner.
// Each edge's owner computes its variable node's sum, decision and next alpha,
// so every variable node is handled by the lanes of its (one or two) edges.
// The arithmetic is that of the other forms (Alg. 2): the same convolutions,
// the same min-normalization, saturation at 255 and lowest-symbol argmin.
// Returns false, having done nothing, when the code is outside these limits.
// DW = 4: every check has degree 4 (the per-iteration loops need no degree tests).
constexpr int kW4Deg = 4;
template <int DW>
__device__ __forceinline__ bool decode_frame_warp4(const JobDesc& job, int frame, uint8_t* X,
                                                   const unsigned char* sblob, int lane) {
  if (job.m > 32 || job.dmax > kW4Deg || job.vmax > 2) return false;
  const uint8_t* exp2 = sblob + job.off.exp2;
  const uint8_t* glog = sblob + job.off.log;
  const uint16_t* row_ptr = reinterpret_cast<const uint16_t*>(sblob + job.off.row_ptr);
  const uint16_t* edge_col = reinterpret_cast<const uint16_t*>(sblob + job.off.edge_col);
  const uint8_t* edge_lh = sblob + job.off.edge_lh;
  const uint8_t* edge_lhi = sblob + job.off.edge_lhi;
  const uint16_t* vn_ptr = reinterpret_cast<const uint16_t*>(sblob + job.off.vn_ptr);
  const uint16_t* vn_edge = reinterpret_cast<const uint16_t*>(sblob + job.off.vn_edge);
  const uint8_t* gam = job.gamma + (size_t)frame * job.n * 4;
  const bool mine = lane < job.m;
  const int e0 = mine ? row_ptr[lane] : 0, d = mine ? row_ptr[lane + 1] - e0 : 0;
  // degree of the per-iteration loops: the lanes without a check compute on zeros and store nothing
  const int dd = DW > 0 ? DW : d;
  // per edge j < d: gamma row of its column, selectors, products, the other edge (-1: none)
  uint32_t gr[kW4Deg], psel[kW4Deg], bsel[kW4Deg], mt[kW4Deg], al[kW4Deg], be[kW4Deg];
  int oe[kW4Deg], col[kW4Deg];
  bool first_owner[kW4Deg];
#pragma unroll
  for (int j = 0; j < kW4Deg; ++j) {
    gr[j] = psel[j] = bsel[j] = mt[j] = al[j] = be[j] = 0u;
    oe[j] = -1;
    col[j] = 0;
    first_owner[j] = false;
    if (j < d) {
      const int e = e0 + j, c = edge_col[e];
      col[j] = c;
      gr[j] = *reinterpret_cast<const uint32_t*>(gam + (size_t)c * 4);
      // P_j(y) = alpha_j(h^-1 y) as the 16-bit pairs (P(0), P(1)), (P(2), P(3))
      const int lhinv = edge_lhi[e];
      const uint32_t s1 = exp2[lhinv], s2 = exp2[lhinv + 1], s3 = s1 ^ s2;
      psel[j] = (0x4040u | (s1 << 8)) | ((0x4040u | s2 | (s3 << 8)) << 16);
      // beta_j(a) = R(h a): byte a from the 16-bit value R(h a) of the pairs R
      const int lh = edge_lh[e];
      const int i1 = exp2[lh], i2 = exp2[lh + 1], i3 = i1 ^ i2;
      bsel[j] = (uint32_t)((((i1 >> 1) << 2) | ((i1 & 1) << 1)) << 4) |
                (uint32_t)((((i2 >> 1) << 2) | ((i2 & 1) << 1)) << 8) |
                (uint32_t)((((i3 >> 1) << 2) | ((i3 & 1) << 1)) << 12);
      // h c for c = 0..3, two bits each (syndrome)
      mt[j] = (uint32_t)exp2[lh] << 2 | (uint32_t)exp2[glog[2] + lh] << 4 | (uint32_t)exp2[glog[3] + lh] << 6;
      const int k0 = vn_ptr[c], k1 = vn_ptr[c + 1];
      first_owner[j] = vn_edge[k0] == e;
      for (int k = k0; k < k1; ++k)
        if (vn_edge[k] != e) oe[j] = vn_edge[k];
      al[j] = gr[j];                             // alpha^(0) = gamma
    }
  }
  const bool counting = job.work != nullptr;
  unsigned long long work = 0;
  // decisions from the sums S = gamma + the incoming betas (lowest symbol on ties), and the syndrome
  uint32_t cw = 0;                               // decisions of the lane's edges, two bits each
  auto decide = [&](int j, uint32_t s0, uint32_t s1) {
    const uint32_t kw = vmin2(s0 * 4u + 0x10000u, s1 * 4u + 0x30002u);
    const uint32_t key = min(kw & 0xFFFFu, kw >> 16);
    cw |= (key & 3u) << (2 * j);
  };
  auto syndrome_ok = [&]() -> bool {
    uint32_t sy = 0;
#pragma unroll
    for (int j = 0; j < kW4Deg; ++j)
      if (j < d) sy ^= (mt[j] >> (2 * ((cw >> (2 * j)) & 3u))) & 3u;   // (mt is 0 past d)
    return __all_sync(0xFFFFFFFFu, sy == 0);
  };
  auto unpack = [](uint32_t r, uint32_t& lo, uint32_t& hi) {
    lo = __byte_perm(r, 0, 0x4140);
    hi = __byte_perm(r, 0, 0x4342);
  };
  // c^(0) = argmin gamma
#pragma unroll
  for (int j = 0; j < kW4Deg; ++j)
    if (j < d) {
      uint32_t g0, g1;
      unpack(gr[j], g0, g1);
      decide(j, g0, g1);
    }
  const bool es = job.early_stop != 0;
  bool ok = (es || job.max_iters == 0) ? syndrome_ok() : false;
  int iters = 0;
  if (!(es && ok)) {
    for (int k = 1; k <= job.max_iters; ++k) {
      // check-node pass (the register form of one check)
      if (counting && d > 2) work += 16ull * 3 * (d - 2);
      uint2 P[kW4Deg], F[kW4Deg], Plast = make_uint2(0u, 0u);
#pragma unroll
      for (int j = 0; j < kW4Deg; ++j) {
        P[j] = make_uint2(0u, 0u);
        F[j] = make_uint2(0u, 0u);
        if (j < dd) {
          P[j].x = __byte_perm(al[j], 0, psel[j] & 0xFFFFu);
          P[j].y = __byte_perm(al[j], 0, psel[j] >> 16);
          Plast = P[j];
        }
      }
      F[0] = P[0];
      uint2 Flast = F[0];
#pragma unroll
      for (int j = 1; j < kW4Deg - 1; ++j)
        if (j <= dd - 2) {
          F[j] = conv4(F[j - 1], P[j]);
          Flast = F[j];
        }
      uint2 Bc = Plast;
      uint2 R[kW4Deg];
#pragma unroll
      for (int j = 0; j < kW4Deg; ++j) R[j] = make_uint2(0u, 0u);
#pragma unroll
      for (int j = kW4Deg - 2; j >= 1; --j) {
        if (j <= dd - 2) {
          R[j] = conv4(F[j - 1], Bc);
          Bc = conv4(Bc, P[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < kW4Deg; ++j) {
        if (j < dd) {
          // beta_0 = B_1, beta_{d-1} = F_{d-2}, else the middle R_j
          const uint2 r = j == 0 ? Bc : (j == dd - 1 ? Flast : R[j]);
          be[j] = __byte_perm(r.x, r.y, bsel[j]);
          if (mine) reinterpret_cast<uint32_t*>(X)[e0 + j] = be[j];
        }
      }
      __syncwarp();
      // variable-node step of each of the lane's edges: S = gamma + beta_e + beta_other;
      // alpha_e = min(255, (S - beta_e) - min (S - beta_e))
      const bool decide_now = es || k == job.max_iters;
      if (decide_now) cw = 0;
#pragma unroll
      for (int j = 0; j < kW4Deg; ++j) {
        if (j < dd) {
          uint32_t t0, t1, b0, b1;
          unpack(gr[j], t0, t1);
          if (oe[j] >= 0) {
            unpack(reinterpret_cast<const uint32_t*>(X)[oe[j]], b0, b1);
            t0 += b0;
            t1 += b1;
          }
          if (decide_now) {
            unpack(be[j], b0, b1);
            decide(j, t0 + b0, t1 + b1);
          }
          const uint32_t mw = vmin2(t0, t1);
          const uint32_t mm = min(mw & 0xFFFFu, mw >> 16) * 0x10001u;
          al[j] = __byte_perm(vmin2(t0 - mm, 0x00FF00FFu), vmin2(t1 - mm, 0x00FF00FFu), 0x6420);
        }
      }
      __syncwarp();
      iters = k;
      if (decide_now) ok = syndrome_ok();
      if (es && ok) break;
    }
  }
#pragma unroll
  for (int j = 0; j < kW4Deg; ++j)
    if (j < d && first_owner[j]) job.out_sym[(size_t)frame * job.n + col[j]] = (uint8_t)((cw >> (2 * j)) & 3u);
  if (lane == 0) {
    job.out_iters[frame] = iters;
    job.out_ok[frame] = ok ? 1 : 0;
  }
  if (counting && work) atomicAdd(job.work, work);
  return true;
}

// ---------------------------------------------------------------- one frame
// Decodes frame `frame` of `job` with the nthr threads of one frame slot
// (slot thread index stid, named barrier bar_id).  sblob holds the job's code
// description, chat[n] the decisions, scratch the per-group buffers; X is the
// slot's message area ([nnz][q] bytes).
// REG4: q = 4 codes take the register form of the check-node pass (single-field
// kernels; the all-field kernel keeps the group form).  PR: the check-node
// convolutions are pruned (pr_conv; 32-lane groups, 8-bit messages, minimal
// schedule).  W4: a GF(4) frame slot of one warp may take the one-warp form
// (decode_frame_warp4; resident-message kernels, which have the registers for it).
// D > 0: every check of the code has degree D (a compile-time loop bound and
// vector layout; 0: the degrees are read per check).
template <class g, int MB, bool T1, bool REG4 = true, bool PR = false, bool W4 = false, int D = 0>
__device__ __forceinline__ void decode_frame(const JobDesc& job, int frame, uint8_t* X, const unsigned char* sblob,
                                             uint8_t* chat, unsigned char* scratch, int stid, int nthr, int bar_id) {
  constexpr int Q = g::Q;
  constexpr int PW = g::PW;
  constexpr int RS = Q * MB;                 // bytes of one message row
  constexpr bool kScatter = scatter_perm<Q>(MB);
  static_assert(MB == 1 || MB == 2, "message bytes");
  static_assert(!PR || (g::G == 32 && MB == 1 && !T1), "pruned convolutions: 32-lane groups, 8-bit, minimal");
  if constexpr (Q == 4 && MB == 1 && !T1 && REG4 && W4) {
    // one warp per frame: a slot of 32 threads
    if (nthr == 32 && decode_frame_warp4<D == 4 ? 4 : 0>(job, frame, X, sblob, stid)) return;
  }
  // pairs (x, y) the convolutions visit in this frame (counted when job.work is set)
  const bool counting = job.work != nullptr;
  unsigned long long work = 0;
  const uint8_t* exp2 = sblob + job.off.exp2;        // x^(i mod (q-1)), i < 2(q-1)
  const uint8_t* glog = sblob + job.off.log;         // log_x(v), v >= 1
  const uint16_t* row_ptr = reinterpret_cast<const uint16_t*>(sblob + job.off.row_ptr);
  const uint16_t* edge_col = reinterpret_cast<const uint16_t*>(sblob + job.off.edge_col);
  const uint8_t* edge_lh = sblob + job.off.edge_lh;    // log_x(h) of each edge
  const uint8_t* edge_lhi = sblob + job.off.edge_lhi;  // log_x(h^-1) of each edge
  const uint16_t* vn_ptr = reinterpret_cast<const uint16_t*>(sblob + job.off.vn_ptr);
  const uint16_t* vn_edge = reinterpret_cast<const uint16_t*>(sblob + job.off.vn_edge);

  const int lane = threadIdx.x & 31;
  // check-node groups (G lanes per check)
  const int grp = stid / g::G, ngroups = nthr / g::G;
  const int gl = stid % g::G;
  const unsigned gmask = group_mask<g::G>(lane);
  const ConvLane cl = conv_lane<g>(gl >> g::LB, gl & (g::DN - 1));
  // variable-node groups (VG lanes per variable node)
  // (16-bit messages keep at most 8 symbols per lane: their rows are read symbol by symbol)
  constexpr int VBPL = (MB == 2 && g::VBPL > 8) ? 8 : g::VBPL, VG = Q / VBPL, VW = VBPL / 2;
  const int vgrp = stid / VG, nvgroups = nthr / VG;
  const int vgl = stid % VG;
  const unsigned vmask = group_mask<VG>(lane);
  constexpr bool kGammaRegs = Q <= 16 && MB == 1;
  uint32_t gcache[kGammaRegs ? VW : 1];

  // lane constants for the gather permutation (staged rows): logarithms of the
  // symbols this lane gathers, packed 8 bits per symbol; the zero symbol, which
  // every multiplication fixes, is flagged separately.
  uint32_t py_log0 = 0, py_log1 = 0, py_nz0 = 0;   // word i: bits [8i, 8i+8)
  if constexpr (!kScatter) {
#pragma unroll
    for (int i = 0; i < PW; ++i) {
      const int w = gl + i * g::G;
      if (w < g::W) {
        if (w) { py_log0 |= (uint32_t)glog[2 * w] << (8 * i); py_nz0 |= 1u << i; }
        py_log1 |= (uint32_t)glog[2 * w + 1] << (8 * i);
      }
    }
  }
  // de-permutation: log of the first symbol this lane writes (-1 for symbol 0)
  const int da_log0 = gl ? (int)glog[gl * g::BPL] : -1;

  unsigned char* gs = scratch + (size_t)grp * job.group_bytes;
  uint8_t* stage = gs;                                                   // [dmax][q * MB] bytes (staged rows)
  const int dm = D > 0 ? D : job.dmax;
  unsigned char* vecs = gs + (kScatter ? 0 : ((dm * RS + 15) / 16) * 16);
  auto vec = [&](int i) { return reinterpret_cast<uint32_t*>(vecs + (size_t)i * g::VB); };
  auto vec16 = [&](int i) { return reinterpret_cast<uint16_t*>(vecs + (size_t)i * g::VB); };
  // vectors: P_j = vec(j) (j < dmax), F_j = vec(dmax + j - 1) (1 <= j <= d-2),
  // B ping-pong = vec(2 dmax - 2), vec(2 dmax - 1), R = vec(2 dmax)
  const int vF = dm - 1, vB = 2 * dm - 2, vR = 2 * dm;
  const uint8_t* gam = job.gamma + (size_t)frame * job.n * Q;

    // ---- variable-node pass (Alg. 2, VNP and hard decision):
    //   S(a) = gamma(a) + sum over edges of beta(a);  c = argmin S (lowest a)
    //   alpha_e(a) = min(255, (S - beta_e)(a) - min_b (S - beta_e)(b))
    // Values are 16-bit halves of 32-bit words: every sum stays below 2^16
    // (at most 255 * (column degree + 1)), so plain 32-bit adds and
    // subtractions never carry or borrow across the halves.
    // 16-bit messages: the same pass on 32-bit sums, one symbol per register
    auto vnp_wide = [&](bool first, bool want_alpha) {
      constexpr int NB = VBPL;
      for (int vn = vgrp; vn < job.n; vn += nvgroups) {
        int S[NB];
        const uint8_t* gr = gam + (size_t)vn * Q + vgl * NB;
#pragma unroll
        for (int i = 0; i < NB; ++i) S[i] = gr[i];
        const int k0 = vn_ptr[vn], k1 = vn_ptr[vn + 1];
        if (!first) {
          for (int k = k0; k < k1; ++k) {
            const uint16_t* br = reinterpret_cast<const uint16_t*>(X + (size_t)vn_edge[k] * RS) + vgl * NB;
#pragma unroll
            for (int i = 0; i < NB; ++i) S[i] += br[i];
          }
        }
        int key = 0x7FFFFFFF;
#pragma unroll
        for (int i = 0; i < NB; ++i) key = min(key, (S[i] << 8) | (vgl * NB + i));
        key = group_min<VG>(key, vmask);
        if (vgl == 0) chat[vn] = (uint8_t)(key & 0xFF);
        if (!first && want_alpha) {
          for (int k = k0; k < k1; ++k) {
            uint16_t* row = reinterpret_cast<uint16_t*>(X + (size_t)vn_edge[k] * RS) + vgl * NB;
            int t[NB];
            int mn = 0x7FFFFFFF;
#pragma unroll
            for (int i = 0; i < NB; ++i) { t[i] = S[i] - row[i]; mn = min(mn, t[i]); }
            mn = group_min<VG>(mn, vmask);
#pragma unroll
            for (int i = 0; i < NB; ++i) row[i] = (uint16_t)min(65535, t[i] - mn);
          }
        }
      }
    };

    // 16-bit messages start from alpha^(0) = gamma widened into every edge row
    auto init_wide = [&]() {
      const int nnz = row_ptr[job.m];
      for (int i = stid; i < nnz * Q; i += nthr) {
        const int e = i / Q, a = i % Q;
        reinterpret_cast<uint16_t*>(X)[i] = gam[(size_t)edge_col[e] * Q + a];
      }
    };

    // q <= 16 with every variable node in one pass of the slot's lanes: each lane
    // keeps its node's gamma words in registers from the first pass on (the later
    // passes then start without a global-memory load)
    const bool gamma_regs = kGammaRegs && job.n <= nvgroups;
    auto vnp = [&](bool first, bool want_alpha) {
      // symbol values of this lane's packed words: (a, a + 1), a = vgl * VBPL + 2 i
      const uint32_t vsym0 = (uint32_t)(vgl * VBPL) * 0x10001u + 0x10000u;
      for (int vn = vgrp; vn < job.n; vn += nvgroups) {
        uint32_t S[VW];
        if (gamma_regs && !first) {
#pragma unroll
          for (int i = 0; i < VW; ++i) S[i] = gcache[i];
        } else {
          load_pairs<VBPL>(gam + (size_t)vn * Q + vgl * VBPL, S);
          if (gamma_regs) {
#pragma unroll
            for (int i = 0; i < VW; ++i) gcache[i] = S[i];
          }
        }
        const int k0 = vn_ptr[vn], k1 = vn_ptr[vn + 1];
        if (!first) {
          for (int k = k0; k < k1; ++k) {
            uint32_t b[VW];
            load_pairs<VBPL>(X + (size_t)vn_edge[k] * Q + vgl * VBPL, b);
#pragma unroll
            for (int i = 0; i < VW; ++i) S[i] += b[i];
          }
        }
        int key;
        if (job.key16) {        // key = S * q + a fits 16 bits: minimum value, lowest symbol
          uint32_t kw = S[0] * (uint32_t)Q + vsym0;
#pragma unroll
          for (int i = 1; i < VW; ++i) kw = vmin2(kw, S[i] * (uint32_t)Q + (vsym0 + 0x20002u * i));
          key = (int)min(kw & 0xFFFFu, kw >> 16);
          key = group_min<VG>(key, vmask);
          if (vgl == 0) chat[vn] = (uint8_t)(key & (Q - 1));
        } else {
          key = 0x7FFFFFFF;
#pragma unroll
          for (int i = 0; i < VW; ++i) {
            const uint32_t sy = vsym0 + 0x20002u * i;
            key = min(key, (int)(((S[i] & 0xFFFFu) << 8) | (sy & 0xFFFFu)));
            key = min(key, (int)(((S[i] >> 16) << 8) | (sy >> 16)));
          }
          key = group_min<VG>(key, vmask);
          if (vgl == 0) chat[vn] = (uint8_t)(key & 0xFF);
        }
        if (!first && want_alpha) {
          for (int k = k0; k < k1; ++k) {
            uint8_t* row = X + (size_t)vn_edge[k] * Q + vgl * VBPL;
            uint32_t t[VW];
            load_pairs<VBPL>(row, t);
#pragma unroll
            for (int i = 0; i < VW; ++i) t[i] = S[i] - t[i];
            uint32_t mw = t[0];
#pragma unroll
            for (int i = 1; i < VW; ++i) mw = vmin2(mw, t[i]);
            int mn = (int)min(mw & 0xFFFFu, mw >> 16);
            mn = group_min<VG>(mn, vmask);
            const uint32_t mm = (uint32_t)mn * 0x10001u;
#pragma unroll
            for (int i = 0; i < VW; ++i) t[i] = vmin2(t[i] - mm, 0x00FF00FFu);
            store_pairs<VBPL>(row, t);
          }
        }
      }
    };

    // ---- syndrome of chat over all checks (slot-wide)
    auto syndrome_ok = [&]() -> bool {
      int bad = 0;
      for (int r = stid; r < job.m; r += nthr) {
        int sy = 0;
        for (int e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
          const int c = chat[edge_col[e]];
          if (c) sy ^= exp2[glog[c] + edge_lh[e]];
        }
        bad |= sy;
      }
      return slot_sync_or(bar_id, nthr, bad) == 0;
    };

    // ---- check-node pass (Alg. 2, F & B matrices and beta), one group per check
    constexpr int CH = Q / 16 > 0 ? Q / 16 : 1;          // 16-byte pieces of one 8-bit row
    // scatter permutation: piece c of the check (edges e0 ..) holds symbols
    // a = 16 part + k (k < 16) of edge j = c / CH, part = c % CH, and
    // P_j(h_j a) = alpha_j(a) with h (16 part + k) = h (16 part) ^ h k, both
    // XOR sums of the h x^b = exp2[log h + b]
    auto scatter_piece = [&](bool first, int e0, int c) {
      const int j = c / CH, part = c - j * CH;
      // gamma on the first pass, else the edge's message row (through one pointer: a separate
      // read-only load of gamma measured 2 % slower at GF(64))
      const uint8_t* src = first ? gam + (size_t)edge_col[e0 + j] * Q : X + (size_t)(e0 + j) * Q;
      const uint4 v = reinterpret_cast<const uint4*>(src)[part];
      const int lh = edge_lh[e0 + j];
      const int h1 = exp2[lh], h2 = exp2[lh + 1], h4 = exp2[lh + 2], h8 = exp2[lh + 3];
      int yb = 0;
#pragma unroll
      for (int b = 4; b < g::P; ++b)
        if ((part >> (b - 4)) & 1) yb ^= exp2[lh + b];
      uint16_t* Pv = vec16(j);
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int y = yb ^ ((k & 1) ? h1 : 0) ^ ((k & 2) ? h2 : 0) ^ ((k & 4) ? h4 : 0) ^ ((k & 8) ? h8 : 0);
        Pv[y] = (uint16_t)__byte_perm(w[k >> 2], 0, 0x4440 | (k & 3));
      }
    };
    // predictions of max_x C(x), one per kind of convolution (F, B, beta): each
    // kind's maxima follow their own distribution
    int tpred[3] = {24, 24, 24};
    auto conv = [&](const uint32_t* A, const uint32_t* B, uint16_t* C, int kind) {
      if constexpr (PR) {
        int folded = 0;
        tpred[kind] = pr_conv<g>(A, B, C, Q >= 128 ? vec(2 * dm + 1) : nullptr, gl, tpred[kind],
                                 counting ? &folded : nullptr);
        if (counting && gl == 0) work += (unsigned long long)folded * Q;
      } else {
        mm_conv<g, MB == 1>(A, B, C, cl, gmask);
        if (counting && gl == 0) work += (unsigned long long)Q * Q;
      }
    };
    auto cnp = [&](bool first) {
      for (int r = grp; r < job.m; r += ngroups) {
        const int e0 = row_ptr[r], d = D > 0 ? D : row_ptr[r + 1] - e0;
        if constexpr (kScatter) {
          for (int c = gl; c < d * CH; c += g::G) scatter_piece(first, e0, c);
        } else {
          // stage incoming alpha rows (alpha^(0) = gamma on the first pass)
          if constexpr (MB == 2) {
            constexpr int CH2 = RS / 16 > 0 ? RS / 16 : 1, CB = RS / CH2;   // chunks of CB bytes
            for (int i = gl; i < d * CH2; i += g::G) {
              const int j = i / CH2, c = i % CH2;
              const uint8_t* src = X + (size_t)(e0 + j) * RS + c * CB;
              uint8_t* dst = stage + j * RS + c * CB;
              if constexpr (CB == 16) *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(src);
              else if constexpr (CB == 8) *reinterpret_cast<uint2*>(dst) = *reinterpret_cast<const uint2*>(src);
              else *reinterpret_cast<uint32_t*>(dst) = *reinterpret_cast<const uint32_t*>(src);
            }
          } else if constexpr (Q >= 16) {
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
          // permutation: P_j(y) = alpha_j(h_j^-1 y), 16-bit natural order
          for (int j = 0; j < d; ++j) {
            const int lhinv = edge_lhi[e0 + j];
            const uint8_t* a = stage + j * RS;
            const uint16_t* a16 = reinterpret_cast<const uint16_t*>(a);
            uint32_t* P = vec(j);
#pragma unroll
            for (int i = 0; i < PW; ++i) {
              const int w = gl + i * g::G;
              if (PW * g::G == g::W || w < g::W) {
                const int s0 = (py_nz0 >> i) & 1 ? exp2[((py_log0 >> (8 * i)) & 0xFF) + lhinv] : 0;
                const int s1 = exp2[((py_log1 >> (8 * i)) & 0xFF) + lhinv];
                if constexpr (MB == 2) P[w] = (uint32_t)a16[s0] | ((uint32_t)a16[s1] << 16);
                else P[w] = (uint32_t)a[s0] | ((uint32_t)a[s1] << 16);
              }
            }
          }
        }
        group_sync<g::G>(gmask);
        // beta_j(a) = R_j(h_j a), written over the edge's message row; the lane's
        // symbols are a0 + i (a0 = gl * BPL, i < BPL) and h (a0 + i) = h a0 ^ h i
        auto depermute = [=](const uint16_t* R16, int e) {
          const int lh = edge_lh[e];
          const int base = da_log0 >= 0 ? (int)exp2[da_log0 + lh] : 0;
          int hb[3] = {0, 0, 0};
#pragma unroll
          for (int b = 0; b < 3; ++b)
            if ((1 << b) < g::BPL) hb[b] = exp2[lh + b];
          int out[g::BPL];
#pragma unroll
          for (int i = 0; i < g::BPL; ++i)
            out[i] = R16[base ^ ((i & 1) ? hb[0] : 0) ^ ((i & 2) ? hb[1] : 0) ^ ((i & 4) ? hb[2] : 0)];
          if constexpr (MB == 2) {
            uint16_t* row = reinterpret_cast<uint16_t*>(X + (size_t)e * RS) + gl * g::BPL;
#pragma unroll
            for (int i = 0; i < g::BPL; ++i) row[i] = (uint16_t)out[i];
          } else {
            store_bytes<g::BPL>(X + (size_t)e * Q + gl * g::BPL, out);
          }
        };
        // forward: F_0 = P_0, F_j = F_{j-1} (*) P_j
        int fprev = 0;                                     // vector index of F_{j-1}
        for (int j = 1; j <= d - 2; ++j) {
          conv(vec(fprev), vec(j), vec16(vF + j), 0);
          group_sync<g::G>(gmask);
          fprev = vF + j;
        }
        depermute(vec16(fprev), e0 + d - 1);               // beta_{d-1} from F_{d-2}
        if constexpr (T1) {          // Table 1 schedule: F_{d-1} into the scratch vector, unused
          mm_conv<g, MB == 1>(vec(fprev), vec(d - 1), vec16(vR), cl, gmask);
          if (counting && gl == 0) work += (unsigned long long)Q * Q;
          group_sync<g::G>(gmask);
        }
        // backward: B_{d-1} = P_{d-1}; beta_j from F_{j-1} (*) B_{j+1}; B_j = B_{j+1} (*) P_j
        int bcur = d - 1;
        int pp = 0;
        for (int j = d - 2; j >= 1; --j) {
          const int fj = (j == 1) ? 0 : vF + j - 1;
          conv(vec(fj), vec(bcur), vec16(vR), 2);
          group_sync<g::G>(gmask);
          depermute(vec16(vR), e0 + j);
          const int bn = vB + pp;
          conv(vec(bcur), vec(j), vec16(bn), 1);
          group_sync<g::G>(gmask);
          bcur = bn;
          pp ^= 1;
        }
        depermute(vec16(bcur), e0);                        // beta_0 from B_1
        if constexpr (T1)            // Table 1 schedule: B_0 into the scratch vector, unused
        {
          mm_conv<g, MB == 1>(vec(bcur), vec(0), vec16(vR), cl, gmask);
          if (counting && gl == 0) work += (unsigned long long)Q * Q;
        }
        group_sync<g::G>(gmask);
      }
    };

    // ---- check-node pass for q = 4 in registers: one lane per check (checks of
    // degree <= kRegDeg).  A 4-symbol vector is two words of 16-bit values,
    // (v0, v1), (v2, v3); the coefficient permutations are byte permutes of the
    // 4-byte rows and the 16-pair convolutions use no shared memory, so the
    // pass has no memory round trip between its steps (at q = 4 the group form
    // is a chain of short shared-memory dependencies).
    constexpr int kRegDeg = 8;
    auto cnp_regs4 = [&](bool first) {
      // beta_e(a) = R(h a): byte a of the row from the 16-bit value R(i), i = h a, of the words R
      auto store_beta = [&](int e, uint2 R) {
        const int lh = edge_lh[e];
        const int i1 = exp2[lh], i2 = exp2[lh + 1], i3 = i1 ^ i2;
        const uint32_t sel = (uint32_t)((((i1 >> 1) << 2) | ((i1 & 1) << 1)) << 4) |
                             (uint32_t)((((i2 >> 1) << 2) | ((i2 & 1) << 1)) << 8) |
                             (uint32_t)((((i3 >> 1) << 2) | ((i3 & 1) << 1)) << 12);
        *reinterpret_cast<uint32_t*>(X + (size_t)e * 4) = __byte_perm(R.x, R.y, sel);
      };
      for (int r = stid; r < job.m; r += nthr) {
        const int e0 = row_ptr[r], d = row_ptr[r + 1] - e0;
        if (counting && d > 2) work += 16ull * 3 * (d - 2);
        // The last P and F are tracked as the loops run (Plast = P_{d-1}, Flast =
        // F_{d-2}): picking them out afterwards by "j == d - 1" turns into an indexed
        // access, which sends the arrays to local memory.
        uint2 P[kRegDeg], F[kRegDeg], Plast = make_uint2(0u, 0u);
#pragma unroll
        for (int j = 0; j < kRegDeg; ++j) {
          P[j] = make_uint2(0u, 0u);
          F[j] = make_uint2(0u, 0u);
          if (j < d) {
            // P_j(y) = alpha_j(h^-1 y): (alpha(0), alpha(h^-1)), (alpha(h^-1 2), alpha(h^-1 3))
            const int e = e0 + j;
            const uint32_t row = first ? *reinterpret_cast<const uint32_t*>(gam + (size_t)edge_col[e] * 4)
                                       : *reinterpret_cast<const uint32_t*>(X + (size_t)e * 4);
            const int lhinv = edge_lhi[e];
            const uint32_t s1 = exp2[lhinv], s2 = exp2[lhinv + 1], s3 = s1 ^ s2;
            P[j].x = __byte_perm(row, 0, 0x4040u | (s1 << 8));
            P[j].y = __byte_perm(row, 0, 0x4040u | s2 | (s3 << 8));
            Plast = P[j];
          }
        }
        // forward: F_0 = P_0, F_j = F_{j-1} (*) P_j; beta_{d-1} = F_{d-2}
        F[0] = P[0];
        uint2 Flast = F[0];
#pragma unroll
        for (int j = 1; j < kRegDeg - 1; ++j)
          if (j <= d - 2) {
            F[j] = conv4(F[j - 1], P[j]);
            Flast = F[j];
          }
        store_beta(e0 + d - 1, Flast);
        // backward: B_{d-1} = P_{d-1}; beta_j = F_{j-1} (*) B_{j+1}; B_j = B_{j+1} (*) P_j; beta_0 = B_1
        uint2 Bc = Plast;
#pragma unroll
        for (int j = kRegDeg - 2; j >= 1; --j) {
          if (j <= d - 2) {
            store_beta(e0 + j, conv4(F[j - 1], Bc));
            Bc = conv4(Bc, P[j]);
          }
        }
        store_beta(e0, Bc);
      }
    };

    // ---- decode one frame.  Without early stop only the final decision is
    // tested, so the stop test runs once, after the last iteration.
    const bool es = job.early_stop != 0;
    if constexpr (MB == 2) vnp_wide(true, false); else vnp(true, false);   // c^(0) = argmin gamma
    slot_sync(bar_id, nthr);
    bool ok = (es || job.max_iters == 0) ? syndrome_ok() : false;
    int iters = 0;
    if (!(es && ok)) {
      if constexpr (MB == 2) {
        init_wide();
        slot_sync(bar_id, nthr);
      }
      for (int k = 1; k <= job.max_iters; ++k) {
        if constexpr (Q == 4 && MB == 1 && !T1 && REG4) {
          if (job.dmax <= kRegDeg) cnp_regs4(k == 1); else cnp(k == 1);
        } else {
          cnp(MB == 1 && k == 1);
        }
        slot_sync(bar_id, nthr);
        if constexpr (MB == 2) vnp_wide(false, k < job.max_iters); else vnp(false, k < job.max_iters);
        slot_sync(bar_id, nthr);
        iters = k;
        if (es || k == job.max_iters) ok = syndrome_ok();
        if (es && ok) break;
      }
    }
    for (int i = stid; i < job.n; i += nthr) job.out_sym[(size_t)frame * job.n + i] = chat[i];
    if (counting && work) atomicAdd(job.work, work);
    if (stid == 0) {
      job.out_iters[frame] = iters;
      job.out_ok[frame] = ok ? 1 : 0;
    }
}

// ---------------------------------------------------------------- the kernel
// Persistent blocks of fpb frame slots; every slot takes work items (a frame
// of one job) from a global counter until the list is exhausted.  QSEL = q,
// VSEL = variant compiles the path of one field order and layout (single-code
// launches); QSEL = 0, VSEL = -1 compiles every path (mixed-code launches).
// Resident 256-thread blocks per SM the register allocation must allow: the
// q >= 128 paths need more than 85 registers per thread without spilling.
#ifndef NBLDPC_MINB_64
#define NBLDPC_MINB_64 4
#endif
#ifndef NBLDPC_MINB_WIDE
#define NBLDPC_MINB_WIDE 2
#endif
// The pruned kernels fit 80 registers without spilling: three 256-thread blocks
// per SM hide more of their shuffle and shared-memory latency (GF(256) (2,6)
// N=384: 119.8 ms at two blocks, 103.8 at three, 106.5 at four).
#ifndef NBLDPC_MINB_PRUNE
#define NBLDPC_MINB_PRUNE 3
#endif
template <int QSEL, int VSEL> struct MinBlocks {
  static constexpr int v = QSEL == 0 ? 2 : QSEL >= 128 ? NBLDPC_MINB_WIDE
                         : (QSEL == 64 ? (VSEL == 1 ? 3 : NBLDPC_MINB_64) : 4);
};

// VSEL = 0 or 1 compiles one layout variant; VSEL = -1 both (chosen per job,
// and for q >= 128 with or without pruned convolutions, bit 2 of the job's variant).
template <int Q, int VSEL, int MB, bool T1 = false, bool PR = false, bool W4 = false, int D = 0>
__device__ __forceinline__ void decode_variant(const JobDesc& job, int frame, uint8_t* X, const unsigned char* sblob,
                                               uint8_t* chat, unsigned char* scratch, int stid, int nthr,
                                               int bar_id) {
  if constexpr (VSEL >= 0) {
    decode_frame<Geo<Q, VSEL>, MB, T1, true, PR, W4, D>(job, frame, X, sblob, chat, scratch, stid, nthr, bar_id);
  } else if (Q >= 128 && (job.variant & 4)) {
    if constexpr (Q >= 128) {
      if (job.variant & 1) decode_frame<Geo<Q, 1>, MB, T1, false, true>(job, frame, X, sblob, chat, scratch, stid, nthr, bar_id);
      else decode_frame<Geo<Q, 0>, MB, T1, false, true>(job, frame, X, sblob, chat, scratch, stid, nthr, bar_id);
    }
  } else if ((job.variant & 1) == 0) {
    decode_frame<Geo<Q, 0>, MB, T1, false>(job, frame, X, sblob, chat, scratch, stid, nthr, bar_id);
  } else {
    decode_frame<Geo<Q, 1>, MB, T1, false>(job, frame, X, sblob, chat, scratch, stid, nthr, bar_id);
  }
}

// MB: message bytes per symbol (1: 8-bit messages; 2: 16-bit, single-field kernels only).
// T1: the Table 1 check-node schedule (3 d_c - 4 convolutions; single-field kernels only).
// XS: the frames' messages stay in shared memory (8-bit messages, single-field
// kernels; kResidentThreads threads, 1, 2 or 4 frame slots per block).
// PR: pruned check-node convolutions (single-field kernels whose layout has
// 32-lane groups; 8-bit messages, minimal schedule).  D > 0: every check has
// degree D (single-field kernels; see decode_frame).
template <int QSEL, int VSEL, int MB, bool T1 = false, bool XS = false, bool PR = false, int D = 0>
__global__ void __launch_bounds__(XS ? kResidentThreads : 256, XS ? 2 : PR ? NBLDPC_MINB_PRUNE : MinBlocks<QSEL, VSEL>::v)
    mma_decode_kernel(const __grid_constant__ LaunchParams p) {
  static_assert(!XS || (QSEL >= 2 && MB == 1 && !T1), "resident messages: 8-bit, minimal schedule, one field");
  static_assert(!PR || (QSEL >= 2 && MB == 1 && !T1), "pruned convolutions: 8-bit, minimal schedule, one field");
  extern __shared__ __align__(16) unsigned char smem[];
  const int nthr = blockDim.x / p.fpb;
  const int slot = threadIdx.x / nthr, stid = threadIdx.x % nthr;
  const int bar_id = 1 + slot;
  unsigned char* base = smem + (size_t)slot * p.slot_smem;
  unsigned char* sblob = base;
  uint8_t* chat = base + p.blob_cap;
  volatile int* ctl = reinterpret_cast<volatile int*>(base + p.blob_cap + p.n_cap);
  unsigned char* scratch = base + p.blob_cap + p.n_cap + 16;
  uint8_t* X = XS ? base + p.xs_off : p.msg + ((size_t)blockIdx.x * p.fpb + slot) * p.slot_bytes;
  int staged = -1;

  // a launch with no more items than frame slots assigns them statically (the
  // host then skips the counter reset)
  int static_item = p.static_items ? (int)blockIdx.x * p.fpb + slot : -1;
  for (;;) {
    if (stid == 0) ctl[0] = static_item >= 0 ? static_item : (int)atomicAdd(p.counter, 1u);
    if (static_item >= 0) static_item = p.total_items;
    slot_sync(bar_id, nthr);
    const int item = ctl[0];
    if (item >= p.total_items) break;
    int j = 0;
    if constexpr (QSEL == 0)
      while (j + 1 < p.njobs && item >= p.jobs[j + 1].item_begin) ++j;
    // single-field launches carry one job: static parameter offsets
    const JobDesc& job = (QSEL == 0) ? p.jobs[j] : p.jobs[0];
    const int frame = item - job.item_begin;
    if (j != staged) {      // stage the code description (GF tables, H, variable-node view)
      for (int i = stid; i < job.off.bytes / 16; i += nthr)
        reinterpret_cast<uint4*>(sblob)[i] = reinterpret_cast<const uint4*>(job.blob)[i];
      staged = j;
      slot_sync(bar_id, nthr);
    }
    if constexpr (QSEL != 0) {
      decode_variant<QSEL, VSEL, MB, T1, PR, XS, D>(job, frame, X, sblob, chat, scratch, stid, nthr, bar_id);
    } else {
      switch (job.q) {
        case 2: decode_variant<2, -1, 1>(job, frame, X, sblob, chat, scratch, stid, nthr, bar_id); break;
        case 4: decode_variant<4, -1, 1>(job, frame, X, sblob, chat, scratch, stid, nthr, bar_id); break;
        case 8: decode_variant<8, -1, 1>(job, frame, X, sblob, chat, scratch, stid, nthr, bar_id); break;
        case 16: decode_variant<16, -1, 1>(job, frame, X, sblob, chat, scratch, stid, nthr, bar_id); break;
        case 32: decode_variant<32, -1, 1>(job, frame, X, sblob, chat, scratch, stid, nthr, bar_id); break;
        case 64: decode_variant<64, -1, 1>(job, frame, X, sblob, chat, scratch, stid, nthr, bar_id); break;
        case 128: decode_variant<128, -1, 1>(job, frame, X, sblob, chat, scratch, stid, nthr, bar_id); break;
        default: decode_variant<256, -1, 1>(job, frame, X, sblob, chat, scratch, stid, nthr, bar_id); break;
      }
    }
    slot_sync(bar_id, nthr);
  }
}

}  // namespace nbldpc
