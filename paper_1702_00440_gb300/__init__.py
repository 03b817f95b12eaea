"""GB300-native Hermite-4 block-step N-body hot path (GraviDy, arXiv 1702.00440).

The compute path is the CUDA library ``libgravidy_gb300.so`` (sources in
``csrc/``, C ABI declared in ``include/gravidy.h``); ``gravidy`` is its thin
ctypes binding.  ``inputs`` holds the seeded synthetic input generators.
"""
