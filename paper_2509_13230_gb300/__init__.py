"""GB300-native Miller-Hagberg sampling of maximum-entropy network models.

Li, Wang, Kojaku, "Fast unbiased sampling of networks with given expected
degrees and strengths" (arXiv 2509.13230): UBCM (Sec. 2.4) and UECM
(Sec. 2.5, Algorithm 1) samplers and the expected degree/strength sums of
parameter inference, as hand-written sm_103a CUDA kernels behind a C ABI
(include/maxent_mh.h).  PyTorch provides device memory and streams only.
"""
from ._native import (MH_BOUND_PAPER, MH_CSR_SYMMETRIC, MH_DIRECTED, MH_FP64_ONLY, MH_INIT_PREV, MH_OUT_COO,
                      MH_OUT_CSR, MH_UBCM, MH_UECM, MhError)
from .expected import ExpectedDegrees, FitResult, expected_degrees, fit
from .ensemble import Ensemble
from .sampler import (BipartiteSampler, SampleResult, Sampler, expected_bwd, expected_fwd, expected_jacobian_diag,
                      row_shard, sample_bipartite, sample_ubcm, sample_weighted, segment_table)

__all__ = [
    "MH_UBCM", "MH_UECM", "MH_OUT_COO", "MH_OUT_CSR", "MH_BOUND_PAPER", "MH_INIT_PREV", "MH_DIRECTED",
    "MH_CSR_SYMMETRIC", "MH_FP64_ONLY",
    "MhError", "Sampler", "BipartiteSampler", "SampleResult", "sample_ubcm", "sample_weighted", "sample_bipartite",
    "segment_table", "expected_fwd", "expected_bwd", "expected_jacobian_diag", "row_shard", "Ensemble",
    "ExpectedDegrees", "expected_degrees", "fit", "FitResult",
]
