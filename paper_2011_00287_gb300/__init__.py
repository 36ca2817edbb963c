"""GB300-native hybrid lattice-Boltzmann step for 3D active cholesteric droplets
(Carenza, Gonnella & Negro, arXiv:2011.00287): CUDA kernels for sm_103a behind the
C ABI of include/lbcad.h, with a thin ctypes binding."""
from .lbcad import (D3Q15, D3Q19, EULER, FIELD_G, FIELD_PSI, FIELD_Q, FIELD_RHO, FIELD_U, FP32, FP64, HEUN, LAGGED, SYNC,
                    LB_BODY_FORCE, LB_STRESS_EQ, STENCIL_ISO, STENCIL_R2, LbcadError, Simulation,
                    default_params, lattice, lbcad_create, lbcad_create_batch, lbcad_destroy, lbcad_get_fields,
                    lbcad_observables, lbcad_set_fields, lbcad_step, library)

__all__ = ["D3Q15", "D3Q19", "EULER", "FIELD_G", "FIELD_PSI", "FIELD_Q", "FIELD_RHO", "FIELD_U", "FP32", "FP64", "HEUN", "LAGGED",
           "SYNC", "LB_BODY_FORCE", "LB_STRESS_EQ", "STENCIL_ISO", "STENCIL_R2", "LbcadError", "Simulation",
           "default_params", "lattice", "lbcad_create", "lbcad_create_batch", "lbcad_destroy", "lbcad_get_fields",
           "lbcad_observables", "lbcad_set_fields", "lbcad_step", "library"]
