"""GB300 (sm_103a) implementation of the D2Q9 chemical-potential multiphase lattice Boltzmann
step with the multiphase curved boundary condition of Yao, Liu, Zhong & Wen (arXiv 2203.04508).

Every step of the method runs in the CUDA library liblbm_gb300.so behind the C ABI of
include/lbm.h; this package only marshals arguments and takes device memory and streams from
PyTorch.  There is no CPU fallback: without the built library every call raises.
"""
from . import _abi  # noqa: F401
from ._abi import (LBM_FP32, LBM_FP64, LBM_FORCE_CHEMPOT, LBM_FORCE_PSEUDO, LBM_LAYOUT_AA, LBM_LAYOUT_AB,  # noqa: F401
                   LbmError, declared_symbols, load)
from .lattice import Batch, Lattice, make_config, workspace_size  # noqa: F401
from .autograd import params_vector, rollout, with_params  # noqa: F401

EOS_NONE, EOS_CS, EOS_PR = 0, 1, 2
COLL_BGK, COLL_MRT = 0, 1
BC_PRESENT, BC_IBC, BC_MIBC, BC_HBB = 0, 1, 2, 3
