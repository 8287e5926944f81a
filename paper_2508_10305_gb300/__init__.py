"""GB300 (sm_103a) implementation of GPZ, the error-bounded lossy compressor
for particle data (Li et al., arXiv 2508.10305).

The compute path is libgpz.so (C ABI in include/gpz.h, CUDA kernels under
csrc/); `gpz` is its Python binding.  `synth` holds the seeded synthetic
input generators.  `batch` and `serve` hold the batched and served forms.
"""
