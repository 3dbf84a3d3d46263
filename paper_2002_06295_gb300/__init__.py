"""GB300 (sm_103a) combinatorial Kalman-filter track building and Kalman fit.

The compute path is libmkf.so (hand-written CUDA behind the C ABI in
include/mkf.h); this package only marshals torch tensors to it."""
from .api import (MkfError, Context, mkf_create, mkf_destroy, mkf_sync, mkf_load_geometry, mkf_bin_hits,
                  mkf_bin_hits_masked, mkf_used_hits,
                  mkf_get_binning, mkf_build_tracks, mkf_set_debug, mkf_set_build_config, mkf_set_build_dedup,
                  mkf_set_adjoint_config,
                  mkf_get_stats, mkf_set_timing, mkf_get_timings, mkf_set_strip_config, mkf_cluster_strips,
                  mkf_seed_tracks, mkf_set_seed_config, mkf_get_seed_stats, mkf_find_overlaps, mkf_get_overlap_stats,
                  mkf_set_overlap_config,
                  mkf_dedup_tracks, mkf_dedup_tracks_noalloc,
                  mkf_fit_tracks, mkf_fit_backward, mkf_fit_tracks_adjoint, alloc_build_outputs, TRK_SHORT, TRK_KEPT,
                  TRK_DUP)

__all__ = ["MkfError", "Context", "mkf_create", "mkf_destroy", "mkf_sync", "mkf_load_geometry", "mkf_bin_hits",
           "mkf_bin_hits_masked", "mkf_used_hits",
           "mkf_get_binning", "mkf_build_tracks", "mkf_set_debug", "mkf_set_build_config", "mkf_set_build_dedup",
           "mkf_set_adjoint_config",
           "mkf_get_stats", "mkf_set_timing", "mkf_get_timings", "mkf_set_strip_config", "mkf_cluster_strips",
           "mkf_seed_tracks", "mkf_set_seed_config", "mkf_get_seed_stats", "mkf_find_overlaps", "mkf_get_overlap_stats",
           "mkf_set_overlap_config",
           "mkf_dedup_tracks", "mkf_dedup_tracks_noalloc",
           "mkf_fit_tracks", "mkf_fit_backward", "mkf_fit_tracks_adjoint", "alloc_build_outputs", "TRK_SHORT",
           "TRK_KEPT", "TRK_DUP"]
