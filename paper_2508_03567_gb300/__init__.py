"""GB300 (sm_103a) min-max decoder for non-binary LDPC codes over GF(2^p).

Implements Alg. 2 of "In-Memory Non-Binary LDPC Decoding" (arXiv 2508.03567)
as hand-written CUDA kernels behind the C ABI in include/nbldpc.h.

    from paper_2508_03567_gb300 import binding   # C-ABI functions, Decoder
    from paper_2508_03567_gb300 import inputs    # seeded synthetic workloads

The binding loads libnbldpc.so on first use and raises if it is missing.
"""
__all__ = ["binding", "inputs", "build"]
