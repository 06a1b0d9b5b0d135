// Prints the compile-time butterfly schedule of the select-free FFT-SPA
// transforms (make_fft_signs in fftspa_kernels.cuh) for q = 8..64 with 4
// elements per lane: per forward and inverse stage the lane mask of -1
// coefficients, and per register the lane mask of negated inverse outputs.
// Host code only; built with nvcc and read by tests/test_fft_sign_schedule.py.
#include <cstdio>

#include "fftspa_kernels.cuh"

template <int Q> void dump() {
  constexpr nbldpc::FftSigns T = nbldpc::make_fft_signs<Q, 4>();
  int lq = 0;
  while ((1 << lq) < Q) ++lq;
  std::printf("q %d ok %d fwd", Q, (int)T.ok);
  for (int s = 0; s < lq; ++s) std::printf(" %x", T.fwd[s]);
  std::printf(" inv");
  for (int s = 0; s < lq; ++s) std::printf(" %x", T.inv[s]);
  std::printf(" out");
  for (int i = 0; i < 4; ++i) std::printf(" %x", T.out[i]);
  std::printf("\n");
}

int main() {
  dump<8>();
  dump<16>();
  dump<32>();
  dump<64>();
  return 0;
}
