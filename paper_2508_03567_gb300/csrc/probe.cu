// Throughput probes of the instruction forms the min-max convolution is built
// from (nbldpc_probe_minmax in include/nbldpc.h).  They measure the integer
// min/max rate that the roofline of the decode kernels is taken against:
// a min-max pair is one 16-bit maximum and one 16-bit minimum, as in
// C(x) = min_y max(A(y), B(x ^ y)) (Alg. 2, F/B/beta equations).
//
// Register forms: every thread repeats the shuffle step of the convolution's
// inner loop on registers -- 8 accumulators, 4 packed A words, 8 packed B
// words per step (32 in all), 32 maxima and 32 minima per step, 4 steps per
// round -- with a chosen
// share of the maxima computed on the FMA pipe (vmax2_fma) and, optionally,
// the A words of steps 1..3 fetched by shfl.xor as in mm_conv.  Each round
// feeds its accumulators back as the next round's A words, so nothing can be
// hoisted out of the loop.  Convolution forms: the decode kernels' own
// mm_conv on shared-memory vectors, chained (the output of one convolution is
// an input of the next).
#include "nbldpc.h"

#include <cuda_runtime.h>

#include "host_internal.h"
#include "mma_kernels.cuh"

namespace {

using nbldpc::vmax2;
using nbldpc::vmax2_fma;
using nbldpc::vmin2;

constexpr int kProbeThreads = 256;

// FMA32: how many of the 32 maxima of a step use the FMA pipe; SHFL: A words
// of steps 1..3 come from lane offsets 2, 4, 6 (the convolution's exchange).
// Every step has its own 8 B words (32 registers, as the convolution holds
// them), so the 128 maxima of a round are 128 distinct pairs.
template <int FMA32, bool SHFL>
__global__ void __launch_bounds__(kProbeThreads) probe_mix_kernel(int rounds, unsigned int* sink) {
  uint32_t a[4], b[4][8], acc[8];
  const uint32_t t0 = threadIdx.x * 0x00010001u;
#pragma unroll
  for (int i = 0; i < 4; ++i) a[i] = (t0 + 0x00050003u * (i + 1)) & 0x00FF00FFu;
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int i = 0; i < 8; ++i) b[s][i] = (t0 * 7u + 0x000B0011u * (8 * s + i + 3)) & 0x00FF00FFu;
#pragma unroll
  for (int i = 0; i < 8; ++i) acc[i] = 0x00FF00FFu;
  for (int k = 0; k < rounds; ++k) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      uint32_t av[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) av[t] = (SHFL && s) ? __shfl_xor_sync(0xFFFFFFFFu, a[t], 2 * s) : a[t];
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const uint32_t m = (r * 4 + t < FMA32) ? vmax2_fma(av[t], b[s][r ^ t]) : vmax2(av[t], b[s][r ^ t]);
          acc[r] = vmin2(acc[r], m);
        }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) a[t] = acc[t + 4];
  }
  uint32_t f = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) f ^= acc[i];
  if (f == 0x9E3779B9u) atomicXor(sink, f);   // keeps the results live; never true for values <= 255
}

// The decode kernels' convolution: each group of G lanes chains convolutions
// over three shared-memory vectors (C = A (*) B, then A <- C).
template <class g>
__global__ void __launch_bounds__(kProbeThreads) probe_conv_kernel(int rounds, unsigned int* sink) {
  __shared__ __align__(16) unsigned char vecs[(kProbeThreads / g::G) * 3 * g::VB];
  const int grp = threadIdx.x / g::G, gl = threadIdx.x % g::G;
  const unsigned gmask = nbldpc::group_mask<g::G>(threadIdx.x & 31);
  unsigned char* base = vecs + (size_t)grp * 3 * g::VB;
  for (int i = gl; i < 3 * g::VB / 2; i += g::G)
    reinterpret_cast<uint16_t*>(base)[i] = (uint16_t)((i * 37 + grp * 11 + blockIdx.x) & 0xFF);
  nbldpc::group_sync<g::G>(gmask);
  const nbldpc::ConvLane cl = nbldpc::conv_lane<g>(gl >> g::LB, gl & (g::DN - 1));
  int ia = 0, ib = 1, ic = 2;
  for (int k = 0; k < rounds; ++k) {
    nbldpc::mm_conv<g, true>(reinterpret_cast<const uint32_t*>(base + ia * g::VB),
                             reinterpret_cast<const uint32_t*>(base + ib * g::VB),
                             reinterpret_cast<uint16_t*>(base + ic * g::VB), cl, gmask);
    nbldpc::group_sync<g::G>(gmask);
    const int t = ia; ia = ic; ic = t;
  }
  const uint16_t v = reinterpret_cast<const uint16_t*>(base + ia * g::VB)[gl];
  if (v == 0x9E37u) atomicXor(sink, v);     // keeps the results live; never true for values <= 255
}

struct ProbeForm {
  const void* kernel;
  double pairs_per_thread_round;   // min-max pairs per thread and round
};

template <class g> constexpr double conv_pairs_per_thread() { return (double)g::Q * g::Q / g::G; }

bool form_of(int form, ProbeForm* f) {
  using nbldpc::Geo;
  switch (form) {
    case NBLDPC_PROBE_ALU: *f = {(const void*)&probe_mix_kernel<0, false>, 256.0}; return true;
    case NBLDPC_PROBE_FMA_1_8: *f = {(const void*)&probe_mix_kernel<4, false>, 256.0}; return true;
    case NBLDPC_PROBE_FMA_3_8: *f = {(const void*)&probe_mix_kernel<12, false>, 256.0}; return true;
    case NBLDPC_PROBE_FMA_4_8: *f = {(const void*)&probe_mix_kernel<16, false>, 256.0}; return true;
    case NBLDPC_PROBE_FMA_3_8_SHFL: *f = {(const void*)&probe_mix_kernel<12, true>, 256.0}; return true;
    case NBLDPC_PROBE_CONV_64:
      *f = {(const void*)&probe_conv_kernel<Geo<64, 1>>, conv_pairs_per_thread<Geo<64, 1>>()};
      return true;
    case NBLDPC_PROBE_CONV_256:
      *f = {(const void*)&probe_conv_kernel<Geo<256, 0>>, conv_pairs_per_thread<Geo<256, 0>>()};
      return true;
  }
  return false;
}

}  // namespace

extern "C" int nbldpc_probe_minmax(int form, int rounds, unsigned int* sink_dev, double* pairs, int* blocks,
                                   void* cuda_stream) {
  ProbeForm f{};
  if (!form_of(form, &f) || rounds < 1 || !sink_dev) return NBLDPC_ERR_ARG;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f.kernel, kProbeThreads, 0) != cudaSuccess)
    return NBLDPC_ERR_CUDA;
  if (per_sm < 1) return NBLDPC_ERR_UNSUPPORTED;
  const int grid = per_sm * sms;
  void* args[] = {&rounds, &sink_dev};
  if (cudaLaunchKernel(f.kernel, dim3(grid), dim3(kProbeThreads), args, 0,
                       reinterpret_cast<cudaStream_t>(cuda_stream)) != cudaSuccess)
    return NBLDPC_ERR_CUDA;
  if (pairs) *pairs = f.pairs_per_thread_round * rounds * (double)grid * kProbeThreads;
  if (blocks) *blocks = grid;
  return NBLDPC_OK;
}
