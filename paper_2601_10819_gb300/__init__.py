"""GB300-native Multi-Scale Deformable Aggregation (MSDA).

The operator (Sec. 3.1, 3.2 and 5.3 of arXiv 2601.10819): every anchor's
keypoints are projected into every camera; each projected location is
bilinearly sampled from that camera's multi-scale feature maps (zero padding
outside a map), multiplied by per-group attention weights and summed into one
C-channel feature per anchor.

The computation runs in hand-written CUDA kernels for sm_103a behind a C-ABI
shared library (``include/msda.h``); ``paper_2601_10819_gb300.msda`` is the
thin ctypes binding (argument marshalling only) plus a
``torch.autograd.Function``.  Importing this package does not load the
library; the first call does, and fails loudly if it is missing.
"""

__all__ = ["inputs"]
