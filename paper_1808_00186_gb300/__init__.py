"""GB300-native hot path of the secondary-field CSEM forward solver (PETGEM method).

The compute path is the CUDA library libpetgem.so (built from csrc/, C ABI in
include/petgem.h); `api` is its thin ctypes binding.  `synth` builds seeded synthetic
models.  Importing this package loads nothing; `api.load()` loads the library and fails
loudly when it is missing.
"""
