"""AdaGScale 3D Gaussian Splatting hot path for one NVIDIA GB300 (sm_103a).

The CUDA kernels live in ``csrc/`` and are exported through the C ABI in
``include/ags.h`` (``libags.so``); ``binding`` is the thin ctypes layer with the
same names, and ``render`` strings the stages together for PyTorch tensors.
"""
