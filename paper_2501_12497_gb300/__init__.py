"""GB300-native MMGKS-OF operators and solver (arXiv 2501.12497).

The compute path is the CUDA library built from csrc/ (libmof.so, C ABI in
include/mof.h); `api` is its thin ctypes binding. `synth` makes seeded inputs.
"""
