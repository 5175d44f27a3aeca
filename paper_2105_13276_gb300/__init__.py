"""GB300-native dynamic mesh refinement (DMR) EM-plasma time step.

The compute path is the C-ABI library ``libdmr.so`` (hand-written CUDA for
sm_103a) in ``csrc/``; ``dmr.py`` is a thin ctypes binding over it.  Importing
this package does not load the library; the binding loads it on first use and
raises if it is missing.
"""
