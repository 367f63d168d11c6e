"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module holds no arithmetic of the WASABI method: it draws random numbers
(SplitMix64, a public-domain counter-based generator by G. Steele, D. Lea and
C. Flood, 2014) and shapes them into point clouds and workload parameter sets.
Depth quantisation, radii, coefficient budgets and everything else the method
computes live on each side separately (the oracle and the CUDA library).
"""
from .splitmix import splitmix64, uniform01
from .clouds import uniform_cloud, heightfield_cloud, aligned
from .configs import CONFIGS, Workload, Job, serving_stream

__all__ = ["splitmix64", "uniform01", "uniform_cloud", "heightfield_cloud",
           "aligned", "CONFIGS", "Workload", "Job", "serving_stream"]
