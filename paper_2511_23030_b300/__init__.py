"""B300-native (sm_103a) hot path of a chunk-based 3D Gaussian splatting mapper.

The product is the C-ABI library libdcg.so (include/dcg.h, sources in csrc/);
`dcg` is its thin ctypes binding, `synth` the seeded synthetic inputs.
Importing this package loads nothing; the binding loads the library on first
use and raises if it is missing.
"""
__all__ = ["dcg", "synth", "build"]
