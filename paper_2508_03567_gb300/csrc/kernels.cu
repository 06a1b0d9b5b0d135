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

// pruned-convolution kernel of one layout, if that layout has 32-lane groups
// (a template, so that the layouts without them are never instantiated)
template <int Q> const void* pruned_kernel(int layout) {
  if constexpr (Geo<Q, 0>::G == 32)
    if (layout == 0) return reinterpret_cast<const void*>(&mma_decode_kernel<Q, 0, 1, false, false, true>);
  if constexpr (Geo<Q, 1>::G == 32)
    if (layout == 1) return reinterpret_cast<const void*>(&mma_decode_kernel<Q, 1, 1, false, false, true>);
  return nullptr;
}

// Address of the decode kernel for variant v (bit 0: layout; bit 1: messages
// resident in shared memory; bit 2: pruned convolutions, layouts of 32-lane
// groups only, not with bit 1), mb-byte messages and the check-node schedule t1
// (1: Table 1's 3 d_c - 4 convolutions, 8-bit messages only) of this unit's
// field order; dreg: the code's check degree when all are equal (GF(4) and
// GF(64) have resident-message kernels for degree 4), else 0; null when there is none.
const void* NBLDPC_CAT(kernel_q, NBLDPC_KQ)(int v, int mb, int t1, int dreg) {
  (void)dreg;
#if NBLDPC_KQ == 0
  (void)v;
  return (mb == 1 && !t1) ? reinterpret_cast<const void*>(&mma_decode_kernel<0, -1, 1>) : nullptr;
#else
  if (v & 4) {
    if (mb != 1 || t1 || (v & 2)) return nullptr;
    return pruned_kernel<NBLDPC_KQ>(v & 1);
  }
  if (v >= 2) {
    if (mb != 1 || t1) return nullptr;
#if NBLDPC_KQ == 64 || NBLDPC_KQ == 4
    // every check of degree 4 (the regular (2,4) codes): a compile-time check degree
    if (dreg == 4)
      return (v & 1) ? reinterpret_cast<const void*>(&mma_decode_kernel<NBLDPC_KQ, 1, 1, false, true, false, 4>)
                     : reinterpret_cast<const void*>(&mma_decode_kernel<NBLDPC_KQ, 0, 1, false, true, false, 4>);
#endif
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
