"""GB300-native multilevel hypergraph partitioning for mapping spiking
neural networks onto neuromorphic cores (Ronzani & Silvano, Sec. 4.1).

The work runs in libsnnmap (hand-written CUDA kernels for sm_103a behind the
C ABI of include/snnmap.h); this package is its Python binding plus a small
convenience layer that keeps inputs in torch device tensors.
"""
from ._native import (  # noqa: F401
    Params, Stats, SnnmapError, lib,
    snnmap_default_params, snnmap_build_hgraph, snnmap_coarsen_level, snnmap_contract,
    snnmap_num_levels, snnmap_level_dims, snnmap_project, snnmap_refine, snnmap_partition, snnmap_connectivity,
    snnmap_partition_host, snnmap_level_copy, snnmap_last_matching, snnmap_level_cid,
    snnmap_round_logs, snnmap_level_logs, snnmap_device_bytes, snnmap_free, snnmap_last_error,
    snnmap_profile, snnmap_stage_times, snnmap_launch_count, snnmap_set_level_budget, snnmap_set_row_budget, snnmap_connectivity_noalloc,
    snnmap_set_coarsen_mode, snnmap_set_histogram_tiers, snnmap_hist_ceiling,
    snnmap_set_tier_table,
    snnmap_partition_graph, snnmap_partition_graph_copy, PlaceLog, snnmap_place_refine,
    snnmap_place_trd, snnmap_place_best, snnmap_place_initial, snnmap_hilbert_order,
    Job, ServeOpts, snnmap_peak_bytes, snnmap_job_footprint, snnmap_serve_create, snnmap_serve_submit,
    snnmap_serve_wait, snnmap_serve_hgraph, snnmap_serve_release, snnmap_serve_info,
    snnmap_serve_destroy, snnmap_batch_partition,
)
from .api import HGraph, lattice_for, params_for, partition, place  # noqa: F401
from .serve import JobBuffers, Server, batch_partition  # noqa: F401
