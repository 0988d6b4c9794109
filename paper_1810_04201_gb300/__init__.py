"""Wilson-Dirac Dslash and device-resident CG solvers for GB300 (sm_103a).

The compute path is a C-ABI CUDA library (``csrc/``, declared in
``include/wd.h``); ``wd.py`` is its thin ctypes binding.  ``gen.py`` draws the
seeded synthetic inputs.
"""
