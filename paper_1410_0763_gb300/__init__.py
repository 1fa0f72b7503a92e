"""GB300-native implementation of the diffuse-radiation ray-tracing scheme of
Tanaka, Yoshikawa, Okamoto & Hasegawa (2014): a C-ABI CUDA library (libart,
include/art.h) for sm_103a with a thin ctypes binding.

``paper_1410_0763_gb300.art``       -- binding of the C ABI (ArtSweep, art_* names)
``paper_1410_0763_gb300.workloads`` -- seeded synthetic inputs
``paper_1410_0763_gb300.build``     -- in-tree nvcc build of libart.so
"""

__all__ = ["art", "workloads", "build"]
