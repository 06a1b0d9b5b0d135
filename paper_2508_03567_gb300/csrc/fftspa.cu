// FFT-SPA kernels of one field order per translation unit (built with
// -DNBLDPC_FQ=q), so the field orders compile in parallel.
#include "fftspa_kernels.cuh"

#ifndef NBLDPC_FQ
#error "NBLDPC_FQ must name the field order"
#endif

#define NBLDPC_CAT2(a, b) a##b
#define NBLDPC_CAT(a, b) NBLDPC_CAT2(a, b)

namespace nbldpc {

// Address of the FFT-SPA kernel of this unit's field order for column degrees
// <= dv (2, 4 or 8) and check degrees <= dc (4 or 8: distributed check-node
// pass), or dc = 0 (lane-per-edge check-node pass, q <= 64, check degree
// <= 32), and its block size; null when there is none.
template <int DC, int DV> const void* fft_entry(int* threads) {
  if (threads) *threads = FftThreads<NBLDPC_FQ, DC, DV>::v;
  return reinterpret_cast<const void*>(&fftspa_decode_kernel<NBLDPC_FQ, DC, DV>);
}

template <int DC> const void* fft_entry_dv(int dv, int* threads) {
  if (dv == 2) return fft_entry<DC, 2>(threads);
  if (dv == 4) return fft_entry<DC, 4>(threads);
  if (dv == 8) return fft_entry<DC, 8>(threads);
  return nullptr;
}

const void* NBLDPC_CAT(fft_kernel_q, NBLDPC_FQ)(int dc, int dv, int* threads) {
#if NBLDPC_FQ <= 64
  if (dc == 0) return fft_entry_dv<0>(dv, threads);
#endif
  if (dc == 4) return fft_entry_dv<4>(dv, threads);
  if (dc == 8) return fft_entry_dv<8>(dv, threads);
  return nullptr;
}

}  // namespace nbldpc
