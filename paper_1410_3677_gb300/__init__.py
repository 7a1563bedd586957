"""All-sky F-statistic search hot path on GB300 (sm_103a).

Submodules:
  fstat  -- ctypes binding of the C-ABI library libfstat.so (CUDA kernels)
  synth  -- seeded synthetic inputs shaped like the search's narrow-band segments

Importing the package loads nothing; `paper_1410_3677_gb300.fstat` loads the
CUDA library and fails loudly when it is missing.
"""
