"""B300-native batched SALT synthetic photometry (JAX-bandflux's hot path).

The computation lives in libsalt_b300.so (hand-written sm_103a CUDA behind the
C ABI of include/salt.h). This package is its Python binding: ctypes
marshalling (_abi) and a torch front end (torch_api) that keeps batches
resident on the device and exposes chi^2 with a hand-written adjoint as a
torch.autograd.Function.
"""
from ._abi import (SALT_KERNEL_AUTO, SALT_KERNEL_BANDWARP, SALT_KERNEL_DIRECT, SALT_KERNEL_FACTORISED, SALT_OK,
                   SALT_OPT_GRAPHS, SALT_OPT_KERNEL, SALT_OPT_SERVE_CHUNK, SALT_OPT_TILE_SAMPLES,
                   Context, Plan, SaltError, bandflux_offsets)

__all__ = ["Context", "Plan", "SaltError", "bandflux_offsets", "SALT_OK", "SALT_OPT_KERNEL",
           "SALT_OPT_TILE_SAMPLES", "SALT_OPT_GRAPHS", "SALT_OPT_SERVE_CHUNK", "SALT_KERNEL_AUTO",
           "SALT_KERNEL_DIRECT", "SALT_KERNEL_FACTORISED", "SALT_KERNEL_BANDWARP"]
