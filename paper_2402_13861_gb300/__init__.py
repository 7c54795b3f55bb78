"""GB300 (sm_103a) hierarchical iso-surface extraction on MLP implicit neural representations
(ReLU, ELU and sine activations).

The computation lives in the CUDA library ``libisx.so`` (C interface: include/isx.h); this package
only builds it and marshals arguments to it (``_lib``).
"""
from ._lib import (ACTS, BF16, CLT, FP32, MODES, RAFIXED, RAUA, SOUND, Batch, Inr, IsxError, Proposer,  # noqa: F401
                   load, mc_table, profile_enable, profile_read, profile_reset, tune_read, tune_reset)
