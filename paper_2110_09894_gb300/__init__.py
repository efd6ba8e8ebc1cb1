"""GB300-native sliced contraction of quantum-circuit tensor networks.

The compute path is libqx.so (CUDA kernels for sm_103a behind the C ABI of
include/qx.h), built by ``paper_2110_09894_gb300.build.build()``;
``paper_2110_09894_gb300.qx`` is its Python binding.
"""
