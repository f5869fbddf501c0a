"""GB300 (sm_103a) implementation of the time step of the CTU lattice
Boltzmann model for bubble cavitation (arXiv:1802.01272).

The compute path is the CUDA library ``lib/libctulbm.so`` behind the C ABI of
``include/ctulbm.h``; ``binding`` marshals arguments to it.
"""
from .binding import (LBM_BC_PERIODIC, LBM_BC_SHEAR_WALLS, LBM_FP16_SHIFTED, LBM_FP32_SHIFTED,
                      LBM_FP64,
                      LBM_LIM_MC, LBM_LIM_ONE, LBM_LIM_ZERO, LBMError, Lattice, Params,
                      lbm_create, lbm_default_params, lbm_destroy, lib, lib_path)

__all__ = ["Lattice", "Params", "LBMError", "lbm_create", "lbm_destroy", "lbm_default_params",
           "lib", "lib_path", "LBM_BC_PERIODIC", "LBM_BC_SHEAR_WALLS", "LBM_FP64",
           "LBM_FP32_SHIFTED", "LBM_FP16_SHIFTED", "LBM_LIM_MC", "LBM_LIM_ZERO", "LBM_LIM_ONE"]
