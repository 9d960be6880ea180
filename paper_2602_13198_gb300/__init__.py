"""GB300-native Monte Carlo radiative transfer hot path (GPUmonty, arXiv 2602.13198).

The compute path is the CUDA library ``libmcgb.so`` (sm_103a) behind the C ABI in
``include/mc.h``; :mod:`paper_2602_13198_gb300.mc` is its thin ctypes binding and
:mod:`paper_2602_13198_gb300.synth` builds seeded synthetic inputs.
"""
