"""GB300-native local ensemble transform Kalman filter (LETKF) analysis for
adaptive optics (Gray et al., arXiv:1408.7069).

The compute path is the CUDA library ``libletkf.so`` (sm_103a) behind the C ABI
declared in ``include/letkf.h``; ``paper_1408_7069_gb300.letkf`` is its thin
Python binding.
"""
__all__ = ["synth", "workloads", "opcount"]
