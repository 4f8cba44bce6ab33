"""GB300-native LB-IMB-DEM hot path (Xiong et al., arXiv:1011.2613).

The compute path is the C-ABI library ``liblbm_imb.so`` built from ``csrc/``
(hand-written sm_103a CUDA kernels).  ``lbm`` is a thin ctypes binding over it;
``inputs`` draws seeded synthetic suspensions.  Importing the package does not
load the CUDA library; the first call into ``lbm`` does, and fails loudly when
it is missing.
"""
__all__ = ["inputs", "lbm"]
