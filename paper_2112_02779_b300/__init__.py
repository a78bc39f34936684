"""B300-native multi-scale range-image point-to-plane registration.

The compute path is the CUDA library librimg.so behind the C ABI in
include/rimg.h; ``paper_2112_02779_b300.rimg`` is its Python binding (it
raises ImportError when the library has not been built) and
``paper_2112_02779_b300.build`` compiles it for sm_103a.
"""
