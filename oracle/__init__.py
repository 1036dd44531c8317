"""CPU FP64 oracle of the ghost-point IBM / ADE impedance / 2D LEE method.

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product path.  The
C source (``lee_oracle.c``) is written from the paper and shares no code with
the CUDA path.  ``build()`` compiles it with gcc (``-ffp-contract=off``,
OpenMP).
"""
from .oracle import (Oracle, build, deriv_1d, ade_drive, ade_regime, ade_stability, stage_forcing, lib_path,  # noqa: F401
                     rational_drive)
