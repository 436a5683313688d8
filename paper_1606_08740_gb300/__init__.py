"""GB300 (sm_103a) implementation of the Alternating Anderson-Richardson (AAR) solver hot path.

``paper_1606_08740_gb300.aar`` is the Python binding of ``libaar.so`` (C ABI in
``include/aar.h``); ``paper_1606_08740_gb300.build`` compiles it with nvcc.
"""
__all__ = ["aar", "build"]
