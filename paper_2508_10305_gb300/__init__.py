"""GB300 (sm_103a) implementation of GPZ, the error-bounded lossy compressor
for particle data (Li et al., arXiv 2508.10305).

The compute path is libgpz.so (C ABI in include/gpz.h, include/gpz_batch.h,
include/gpz_serve.h; CUDA kernels under csrc/), built by `build`.  `gpz` is
its Python binding: the single-array calls (Compressor, Decompressor), the
batched plans (BatchCompressor, BatchDecompressor) and the serving engine
(Server) all live there.  `synth` holds the seeded synthetic input
generators.
"""
