"""CPU oracle for phaseless AFQMC (Motta & Zhang 2017).

TEST INFRASTRUCTURE.  A plain float64 numpy implementation of the hot path,
written from the paper and checked against closed forms, brute-force Fock
space results and library routines in ``tests/``.  It shares no code with the
GPU library.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` may import it.
"""
from . import afqmc, mcd, multidet, philox, scf  # noqa: F401
