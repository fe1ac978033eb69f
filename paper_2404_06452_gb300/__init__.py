"""GB300-native batched WCRT analysis of PAAM (arxiv 2404.06452, Sec. IV-F).

The compute path is ``libpaam_rta.so`` (hand-written sm_103a CUDA behind the
C ABI of ``include/paam_rta.h``); this package is its thin Python binding
plus convenience wrappers that allocate outputs with PyTorch.
"""
from ._binding import (PAAM_MAX_CHAINS, PAAM_ST_DEP, PAAM_ST_ITERCAP, PAAM_ST_OVERRUN, PAAM_ST_SCHED,
                       AnalysisOpts, Batch, Context, PaamError, SystemsView, analysis_opts, launch_count, lib,
                       paam_rta_analyze_batch, paam_rta_autotune, paam_rta_get_launch_config,
                       paam_rta_load_systems, paam_rta_num_launch_configs, paam_rta_set_launch_config,
                       PAAM_NOALLOC_MAX_SYS, paam_rta_analyze_noalloc, paam_rta_search_priorities, paam_tc_gemm_bf16, paam_rta_search_ordered, paam_diag_gelu, paam_diag_divisor, paam_rta_end_to_end, paam_measure_preemption, PREEMPTION_KERNELS,
                       paam_rta_audsley_order, paam_rta_analyze_host, paam_rta_autotune_search, strerror)
from ._binding import (Model, TrainOpts, paam_surrogate_features, paam_surrogate_grad, paam_surrogate_infer,
                       paam_surrogate_search,
                       paam_surrogate_predict, paam_surrogate_train, train_opts)
from .api import analyze, audsley_order, search, to_device

__all__ = [
    "Context", "Batch", "PaamError", "SystemsView", "AnalysisOpts", "analysis_opts", "lib", "strerror",
    "paam_rta_load_systems", "paam_rta_analyze_batch", "analyze", "to_device", "launch_count",
    "paam_rta_autotune", "paam_rta_num_launch_configs", "paam_rta_set_launch_config",
    "paam_rta_get_launch_config", "paam_rta_analyze_noalloc", "PAAM_NOALLOC_MAX_SYS",
    "paam_rta_search_priorities", "search", "paam_rta_audsley_order", "audsley_order", "paam_rta_analyze_host", "paam_rta_autotune_search", "paam_tc_gemm_bf16", "paam_rta_search_ordered", "paam_diag_gelu", "paam_diag_divisor", "paam_rta_end_to_end", "paam_measure_preemption", "PREEMPTION_KERNELS",
    "Model", "TrainOpts", "train_opts", "paam_surrogate_train", "paam_surrogate_infer", "paam_surrogate_predict", "paam_surrogate_search",
    "paam_surrogate_grad", "paam_surrogate_features",
    "PAAM_ST_SCHED", "PAAM_ST_OVERRUN", "PAAM_ST_DEP", "PAAM_ST_ITERCAP", "PAAM_MAX_CHAINS",
]
