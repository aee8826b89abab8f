"""GB300-native lid-driven-cavity pressure-projection path (arXiv 2504.03697).

The compute path lives in the CUDA shared library built from ``csrc/`` and is
reached through ``paper_2504_03697_gb300.cfd`` (a thin ctypes binding of the
C-ABI declared in ``include/cfd.h``).  Importing this package loads nothing;
``paper_2504_03697_gb300.synthetic`` holds the seeded input generators.
"""
