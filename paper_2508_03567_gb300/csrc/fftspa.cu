// FFT-SPA kernels of one field order per translation unit (built with
// -DNBLDPC_FQ=q), so the field orders compile in parallel.
#include "fftspa_kernels.cuh"

#ifndef NBLDPC_FQ
#error "NBLDPC_FQ must name the field order"
#endif

#define NBLDPC_CAT2(a, b) a##b
#define NBLDPC_CAT(a, b) NBLDPC_CAT2(a, b)

namespace nbldpc {

// Address of the FFT-SPA kernel for check degrees <= dc (4 or 8) and column
// degrees <= dv (2, 4 or 8) of this unit's field order, and its block size;
// null otherwise.
const void* NBLDPC_CAT(fft_kernel_q, NBLDPC_FQ)(int dc, int dv, int* threads) {
  constexpr int q = NBLDPC_FQ;
  if (threads) {
    *threads = dc == 4 ? (dv == 2 ? FftThreads<q, 4, 2>::v : dv == 4 ? FftThreads<q, 4, 4>::v : FftThreads<q, 4, 8>::v)
                       : (dv == 2 ? FftThreads<q, 8, 2>::v : dv == 4 ? FftThreads<q, 8, 4>::v : FftThreads<q, 8, 8>::v);
  }
  if (dc == 4) {
    if (dv == 2) return reinterpret_cast<const void*>(&fftspa_decode_kernel<q, 4, 2>);
    if (dv == 4) return reinterpret_cast<const void*>(&fftspa_decode_kernel<q, 4, 4>);
    if (dv == 8) return reinterpret_cast<const void*>(&fftspa_decode_kernel<q, 4, 8>);
  } else if (dc == 8) {
    if (dv == 2) return reinterpret_cast<const void*>(&fftspa_decode_kernel<q, 8, 2>);
    if (dv == 4) return reinterpret_cast<const void*>(&fftspa_decode_kernel<q, 8, 4>);
    if (dv == 8) return reinterpret_cast<const void*>(&fftspa_decode_kernel<q, 8, 8>);
  }
  return nullptr;
}

}  // namespace nbldpc
