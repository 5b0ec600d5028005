"""GB300 solver for the per-time-step saddle-point systems of the ternary Cahn-Hilliard model.

The compute lives in ``libch.so`` (CUDA, sm_103a) behind the C ABI of ``include/ch.h``;
``paper_2204_03575_gb300.ch`` is its Python binding and ``inputs`` the seeded input generator.
Nothing is loaded at import time.
"""
__all__ = ["ch", "inputs", "build"]
