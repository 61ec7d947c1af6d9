"""GB300-native rank-profile-revealing PLUQ / echelon forms over GF(p).

Tile-recursive elimination (Dumas, Gautier, Pernet, Sultan, "Parallel
computation of echelon forms", arXiv:1402.3501, Sec. 4.1) with hand-written
CUDA kernels for sm_103a behind a C ABI (include/pluqmodp.h).  This package
holds the CUDA sources (csrc/), the in-tree build (build.py) and the Python
binding (binding.py).
"""
from .binding import (BatchPlan, FORM_AUTO, FORM_FP64, FORM_LIMB_F16, Context, PluqError, PLUQResult,
                      column_echelon_modp, default_context, echelon_modp, echelon_modp_batched,
                      fgemm_modp,
                      fgemm_modp_noalloc, load, pluq_modp, pluq_modp_batched, rank_profile_modp,
                      rank_profile_modp_batched, sync_status)

__all__ = [
    "BatchPlan",
    "FORM_AUTO", "FORM_FP64", "FORM_LIMB_F16", "Context", "PluqError", "PLUQResult",
    "column_echelon_modp", "default_context", "echelon_modp", "echelon_modp_batched", "fgemm_modp",
    "fgemm_modp_noalloc",
    "load", "pluq_modp", "pluq_modp_batched", "rank_profile_modp", "rank_profile_modp_batched",
    "sync_status",
]
