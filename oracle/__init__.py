"""FP64 CPU oracle of the RTGS rasterizer -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is independent of the CUDA library:
no shared code, headers or constants.
"""
