"""GB300 (sm_103a) exponential time propagator for elastodynamics (arXiv 2405.05213).

The compute path is ``libetp.so`` (CUDA kernels behind the C ABI of
``include/etp.h``); ``paper_2405_05213_gb300.etp`` is its ctypes binding.
"""
from .etp import (Context, EtpError, Mesh, Trajectory, ETP_PREC_FP64, ETP_PREC_MIXED,  # noqa: F401
                  ETP_MAT_LINEAR, ETP_MAT_NEOHOOKE, ETP_MAT_MOONEY_RIVLIN, ETP_MAT_SVK, ETP_MAT_YEOH)
