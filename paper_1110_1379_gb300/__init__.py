"""GB300-native FAS multigrid solver for the Hu-Sawicki f(R) scalaron equation.

The compute path is the CUDA library ``libfrmg.so`` (sm_103a) behind the C ABI
declared in ``include/frmg.h``; ``paper_1110_1379_gb300.frmg`` is its thin
Python binding.  ``paper_1110_1379_gb300.synth`` holds seeded input generators.
Submodules are imported lazily so that the generators load without a GPU.
"""
