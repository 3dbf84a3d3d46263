"""Seeded synthetic inputs shared by the tests, the oracle runs and the benchmark.

This package only *generates inputs*: detector descriptions, simulated charged
particles crossing them, the resulting smeared hits, noise hits and smeared
seeds.  It contains no reconstruction arithmetic (no covariance transport, no
Jacobian, no chi2, no Kalman update, no candidate ranking): those live on one
side in the CPU oracle and on the other in the CUDA library, and neither side
imports the other.
"""
from .geometry import Geometry, geometry_barrel10, geometry_barrel14, geometry_cmslike
from .events import (Event, EventBatch, simulate_event, make_config_event, make_batch,
                     WORKLOAD_SPECS, config_seed)

__all__ = ["Geometry", "geometry_barrel10", "geometry_barrel14", "geometry_cmslike",
           "Event", "EventBatch", "simulate_event", "make_config_event", "make_batch",
           "WORKLOAD_SPECS", "config_seed"]
