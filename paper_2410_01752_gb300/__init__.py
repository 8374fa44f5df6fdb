"""GB300-native SISSO hot path (arXiv 2410.01752): SIS screening and exhaustive l0 on sm_103a.

The computation lives in ``libsisso_gb300.so`` (CUDA C++ behind the C ABI of
``include/sisso.h``); ``sisso`` is its ctypes binding and ``inputs`` the seeded synthetic
workloads.  Build the library with ``paper_2410_01752_gb300.build.build()``.
"""
from .sisso import (GRAMMAR_EQ2, GRAMMAR_NEW_X_PREV, PREC_FP32, PREC_FP64, PREC_MIXED_BF16,  # noqa: F401
                    PREC_MIXED_FP16, MLP, Batch, Descriptor, Sisso, fit_batch,
                    SissoError, load)
