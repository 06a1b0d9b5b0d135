// Prints the compile-time butterfly schedule of the select-free FFT-SPA
// transforms (make_fft_signs in fftspa_kernels.cuh) for the kernels' field
// orders and elements per lane (4 for q <= 128, 8 for q = 256): per forward
// and inverse stage the lane mask of -1
// coefficients, and per register the lane mask of negated inverse outputs.
// Host code only; built with nvcc and read by tests/test_fft_sign_schedule.py.
#include <cstdio>

#include "fftspa_kernels.cuh"

template <int Q, int R> void dump() {
  constexpr nbldpc::FftSigns T = nbldpc::make_fft_signs<Q, R>();
  int lq = 0;
  while ((1 << lq) < Q) ++lq;
  std::printf("q %d r %d ok %d fwd", Q, R, (int)T.ok);
  for (int s = 0; s < lq; ++s) std::printf(" %x", T.fwd[s]);
  std::printf(" inv");
  for (int s = 0; s < lq; ++s) std::printf(" %x", T.inv[s]);
  std::printf(" out");
  for (int i = 0; i < R; ++i) std::printf(" %x", T.out[i]);
  std::printf("\n");
}

int main() {
  dump<8, 4>();
  dump<16, 4>();
  dump<32, 4>();
  dump<64, 4>();
  dump<128, 4>();
  dump<256, 8>();
  return 0;
}
