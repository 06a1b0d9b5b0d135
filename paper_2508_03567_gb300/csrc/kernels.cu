// One translation unit per kernel family, so the field orders compile in
// parallel: built with -DNBLDPC_KQ=q for the two layout variants of field
// order q (single-code launches), or -DNBLDPC_KQ=0 for the kernel that
// serves every field order (mixed-code launches).
#include "mma_kernels.cuh"

#ifndef NBLDPC_KQ
#error "NBLDPC_KQ must name the field order (or 0)"
#endif

#define NBLDPC_CAT2(a, b) a##b
#define NBLDPC_CAT(a, b) NBLDPC_CAT2(a, b)

namespace nbldpc {

// Address of the decode kernel for variant v (bit 0: layout; bit 1: messages
// resident in shared memory), mb-byte messages and the check-node schedule t1
// (1: Table 1's 3 d_c - 4 convolutions, 8-bit messages only) of this unit's
// field order; null when there is none.
const void* NBLDPC_CAT(kernel_q, NBLDPC_KQ)(int v, int mb, int t1) {
#if NBLDPC_KQ == 0
  (void)v;
  return (mb == 1 && !t1) ? reinterpret_cast<const void*>(&mma_decode_kernel<0, -1, 1>) : nullptr;
#else
  if (v >= 2) {
    if (mb != 1 || t1) return nullptr;
    return (v & 1) ? reinterpret_cast<const void*>(&mma_decode_kernel<NBLDPC_KQ, 1, 1, false, true>)
                   : reinterpret_cast<const void*>(&mma_decode_kernel<NBLDPC_KQ, 0, 1, false, true>);
  }
  if (t1) {
    if (mb != 1) return nullptr;
    return v ? reinterpret_cast<const void*>(&mma_decode_kernel<NBLDPC_KQ, 1, 1, true>)
             : reinterpret_cast<const void*>(&mma_decode_kernel<NBLDPC_KQ, 0, 1, true>);
  }
  if (mb == 2)
    return v ? reinterpret_cast<const void*>(&mma_decode_kernel<NBLDPC_KQ, 1, 2>)
             : reinterpret_cast<const void*>(&mma_decode_kernel<NBLDPC_KQ, 0, 2>);
  return v ? reinterpret_cast<const void*>(&mma_decode_kernel<NBLDPC_KQ, 1, 1>)
           : reinterpret_cast<const void*>(&mma_decode_kernel<NBLDPC_KQ, 0, 1>);
#endif
}

}  // namespace nbldpc
