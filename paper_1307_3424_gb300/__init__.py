"""GB300-native sparse w-projection (Wolz et al. 2013, arXiv:1307.3424).

The compute path is the CUDA library `libwproj.so` (C-ABI, include/wproj.h);
`wproj` is its thin Python binding.  `synth` draws seeded synthetic inputs.
"""
