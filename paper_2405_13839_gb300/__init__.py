"""GB300-native Diffusing Winding Gradients (arXiv 2405.13839).

The compute path is libdwg.so (CUDA, sm_103a) behind the C ABI in
include/dwg.h; ``paper_2405_13839_gb300.dwg`` is its ctypes binding and
``paper_2405_13839_gb300.build`` compiles it.
"""
