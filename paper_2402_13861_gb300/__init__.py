"""GB300 (sm_103a) hierarchical iso-surface extraction on ReLU-MLP implicit neural representations.

The computation lives in the CUDA library ``libisx.so`` (C interface: include/isx.h); this package
only builds it and marshals arguments to it (``_lib``).
"""
from ._lib import (BF16, CLT, FP32, RAUA, SOUND, Batch, Inr, IsxError, Proposer, load, mc_table,  # noqa: F401
                   profile_enable, profile_read, profile_reset, tune_read, tune_reset)
