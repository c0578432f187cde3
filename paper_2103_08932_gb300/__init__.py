"""GB300 (sm_103a) library for the splitting random-choice dynamic relaxation
of Total-Lagrangian SPH (Zhu, Zhang & Hu, arXiv 2103.08932).

``srdr`` is the ctypes binding of the C ABI in ``include/srdr.h``; ``synth``
holds the seeded synthetic bodies; ``build`` compiles the CUDA library.
"""
__all__ = ["srdr", "synth", "build"]
