"""GB300 (sm_103a) NLINV: iteratively regularised Gauss-Newton MRI reconstruction with hand-written CUDA kernels.

Importing the package is cheap; the CUDA library is loaded on first use by :mod:`paper_1301_1215_gb300.nlinv`.
"""
__version__ = "0.1.0"
