"""GB300-native masked keypoint detection for video (arXiv 1503.06959).

The hot path lives in the CUDA library ``libfkd.so`` (``csrc/``) behind the
C ABI declared in ``include/fkd.h``; ``fkd`` is its ctypes binding. Nothing is
loaded at import time: ``synth`` (input frames only) imports without a GPU.
"""
