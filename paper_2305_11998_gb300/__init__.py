"""GB300-native MOLC (method of long characteristics) high-order sweep: C-ABI library libmolc (include/molc.h)
with hand-written sm_103a CUDA kernels, and this thin Python binding."""
from .molc import (AREA_RENORM, AUTOTUNE, BALANCE, EXPORTED, TILED, HOST_ONLY, Batch, FP32, FP64, MOMENTS, RAYS_PAPER, RAYS_UNIFORM, MolcError, Plan,  # noqa: F401
                   PlanInfo, fp64_fma_rate, load, quadrature_product, tune_cache)
