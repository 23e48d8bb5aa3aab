"""GB300 (sm_103a) DBaS-Log-MPPI step (arXiv 2504.06437).

``binding``   ctypes binding of the C ABI in ``include/dbasmppi.h``
``workloads`` seeded synthetic worlds and parameter presets
"""
