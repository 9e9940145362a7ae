"""GB300-native FFT bispectrum-multipole estimator (arXiv:1708.05303).

The compute path is the C-ABI library ``libbsp.so`` (hand-written sm_103a CUDA
kernels); ``paper_1708_05303_gb300.bsp`` is its thin ctypes binding and
``paper_1708_05303_gb300.synth`` draws seeded synthetic inputs.  Submodules are
imported explicitly so that importing the package loads nothing.
"""
