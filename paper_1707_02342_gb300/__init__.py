"""GB300-native information-theoretic MPC (IT-MPC / MPPI) control iteration.

The hot path of Williams et al., "Information Theoretic Model Predictive
Control: Theory and Applications to Autonomous Driving" (arXiv 1707.02342):
K perturbed control sequences are sampled around the nominal sequence (Alg. 1),
rolled out through a network-plus-kinematics vehicle model (Sec. V-B), costed
on a track costmap with speed and stabilizing terms (Sec. V-C), and the nominal
sequence is replaced by the exp(-S/lambda)-weighted mean (Alg. 2, Sec. III-D).

All arithmetic runs in hand-written sm_103a CUDA kernels inside ``libitmpc.so``
(C ABI declared in ``include/itmpc.h``); ``itmpc`` is a thin ctypes binding.
Importing this package does not load the library; creating a controller does,
and fails loudly if the library is missing.
"""
__all__ = ["inputs"]
