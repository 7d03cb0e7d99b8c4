"""GB300-native equivariant interaction layer (energy, forces, stress).

The compute path is the CUDA library libmlip.so (C ABI in include/mlip.h);
this package only builds it and marshals arguments to it.
"""
from .binding import (MLIP_PREC_BF16, MLIP_PREC_F16, MLIP_PREC_FP32, MlipError, Model, lib, mlip_energy_forces,  # noqa: F401
                      mlip_model_create, mlip_model_free, mlip_model_load, mlip_model_num_weights,
                      mlip_neighbors)
