"""FP64 CPU oracle for the FFT bispectrum-multipole estimator (arXiv:1708.05303).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_1708_05303_gb300``) and imports nothing from it.
"""
from .oracle import *  # noqa: F401,F403
