"""FP64 CPU oracle for SAFR (arXiv 2510.19542).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use this package; the library product never
imports it.  It shares no code with the CUDA path.

The arithmetic lives in ``oracle.c`` (plain C99, FP64, built with gcc into
``oracle/_build/liboracle.so``); this module only builds it and marshals numpy
arrays through ctypes.
"""
from .safr_oracle import (  # noqa: F401
    build,
    dft2,
    idft2,
    svd,
    group_B,
    group_B_learned,
    mlp_phi,
    philox4x32_10,
    filter_frames_loss,
    filter_frame,
    polc,
    integrate,
    MLP_PARAMS,
    cone,
    remove_tt,
    resample,
    pupil_mask,
    OraclePlan,
    threads,
)
