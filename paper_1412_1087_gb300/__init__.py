"""GB300-native (sm_103a) MHD-PIC cosmic-ray particle update.

The compute path is a CUDA shared library with a C ABI (``include/mhdpic.h``);
:mod:`paper_1412_1087_gb300.mhdpic` is its thin ctypes binding and
:mod:`paper_1412_1087_gb300.workloads` holds the seeded synthetic inputs.
Nothing is imported eagerly so that the input generators can be used without
a GPU.
"""
__all__ = ["mhdpic", "workloads"]
