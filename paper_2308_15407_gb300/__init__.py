"""GB300-native FDLB solver for the simplified Enskog equation (arXiv 2308.15407).

The compute path is the CUDA library ``libfdlb.so`` (C ABI declared in
``include/fdlb.h``); this package only marshals arguments to it.  There is no CPU
fallback: importing :mod:`paper_2308_15407_gb300.fdlb` without the built library
raises.  Build it with ``python -m paper_2308_15407_gb300.build``.
"""
