"""GB300-native UGKWP particle phase for frequency-dependent radiation transport.

The compute path is a C-ABI CUDA library (``csrc/``, declared in
``include/ugkwp.h``); ``binding`` marshals arguments to it.  ``inputs`` holds
problem descriptions and seeded synthetic workloads.  Submodules are imported
lazily so that describing a problem never loads the CUDA library.
"""
__all__ = ["inputs", "binding"]
