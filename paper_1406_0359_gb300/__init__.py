"""GB300-native SARA-SDMM radio-interferometric imaging (hot path).

The compute path is the CUDA library ``libpurify_gb300.so`` built from
``csrc/`` for sm_103a; ``binding`` marshals arguments to its C-ABI (declared
in ``include/purify.h``).  ``synth`` holds the seeded input generators.
Importing this package does not load the CUDA library; the first call into
``binding`` does, and raises if it is missing.
"""
__all__ = ["binding", "synth"]
