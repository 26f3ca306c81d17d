"""GB300 (sm_103a) library for the online tensor method of Huang, Niranjan,
Hakeem and Anandkumar, "Online Tensor Methods for Learning Latent Variable
Models".

The compute path is the C-ABI shared library ``_build/libotm.so`` (CUDA
kernels, see ``include/otm.h``); :mod:`paper_1309_0787_gb300.otm` is its thin
Python binding over PyTorch device tensors.  Build the library with
``python -m paper_1309_0787_gb300.build``.
"""
__all__ = ["otm", "build"]
