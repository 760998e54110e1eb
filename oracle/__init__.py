"""Reference oracle for the multiphase curved-boundary lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY: a plain, slow, FP64 C++ implementation of the method of Yao, Liu,
Zhong & Wen (arXiv 2203.04508) that the CUDA implementation is checked against.  It shares no
code with the CUDA path.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it.

Functions whose parity with the paper is not pinned by an independent check are listed in
``PARITY_UNPINNED`` (currently none).
"""
from .oracle import (Oracle, OracleConfig, build, eos_eval, lattice, mrt_matrices, feq, meq,
                     collide, link_value, q_cylinder, BC_PRESENT, BC_IBC, BC_MIBC, BC_HBB,
                     EOS_NONE, EOS_CS, EOS_PR, COLL_BGK, COLL_MRT, FORCE_CHEMPOT, FORCE_PSEUDO,
                     set_threads, get_threads)

PARITY_UNPINNED = ()
