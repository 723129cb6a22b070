"""GB300-native splitting conic solver: ADMM on the homogeneous self-dual
embedding with an indirect (CG) subspace projection, as CUDA kernels behind a
C ABI (``include/scs_gpu.h``).

Submodules are imported lazily so that the input generator (``synth``) can be
used without loading the CUDA library.
"""
