"""Numerical entanglement for fail-stop mitigation on GB300 (sm_103a).

The compute path is the CUDA library ``libne.so`` (C ABI declared in
``include/ne.h``); :mod:`paper_1509_03838_gb300.ne` is its thin ctypes
binding.  :mod:`paper_1509_03838_gb300.synth` draws the seeded inputs.
"""
