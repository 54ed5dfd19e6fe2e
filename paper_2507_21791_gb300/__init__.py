"""GB300-native reorthogonalized block classical Gram-Schmidt QR (BCGSI+,
BCGSI+P-1S, BCGSI+P-2S).  The compute path is the CUDA library built from
csrc/; `bcgs` is its ctypes binding and loads it on first use."""
