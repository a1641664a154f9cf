"""GB300 (sm_103a) finite-difference micromagnetics hot path.

Demagnetising field H_d = -N * M by zero-padded FFT convolution with the Newell
tensor, and the fused LLG RK stage update that consumes it, after "Boris
Computational Spintronics" (arXiv 2008.02478), Section 7 and Eq. 1.

The compute path is the CUDA library built from ``csrc/`` (``libboris.so``),
called through its C ABI (``include/boris.h``).  ``binding`` holds the thin
Python layer; importing this package does not load the library.
"""

__all__ = ["binding", "inputs", "build"]
