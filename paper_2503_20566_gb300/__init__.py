"""GB300-native VMC for gauge-canonical-form gauge-invariant PEPS (Z_N LGT, 2+1D).

The compute path is the CUDA library ``libgcfvmc.so`` (C ABI in
``include/gcfvmc.h``); this package only builds it and marshals arguments.
"""

from .binding import (BF16, COMPLEX, FP32, FP64, REAL, SR, TDVP_STAGE1, TDVP_STAGE2, TF32, Context,
                      GcfError, exported_symbols, load_library, sample_multi)

__all__ = ["Context", "GcfError", "load_library", "exported_symbols", "sample_multi", "REAL", "COMPLEX", "FP64", "FP32",
           "TF32", "BF16", "SR", "TDVP_STAGE1", "TDVP_STAGE2"]
