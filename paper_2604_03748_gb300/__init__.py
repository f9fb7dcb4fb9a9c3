"""GB300-native neural six-way lightmaps (arXiv 2604.03748): guide march,
lightmap network and six-way shading as sm_103a CUDA kernels behind a C ABI
(include/nsl.h).  ``nsl`` is the ctypes binding, ``build`` compiles the
library, ``inputs`` draws seeded synthetic inputs."""
