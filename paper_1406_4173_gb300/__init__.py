"""Exact betweenness centrality on GB300: plain Brandes and Brandes++ (Erdos et al.).

The computation runs in ``libbcpp.so`` (CUDA, sm_103a; C ABI in include/bcpp.h).  This
package is its thin Python binding (``api``) plus the seeded input generators (``gen``).
Importing the package does not load the library; the first call does, and raises if the
library has not been built (there is no CPU fallback).
"""
from .api import (  # noqa: F401
    Arena, BcppError, Context, Graph, HostCSR, SigmaOverflow, brandes, brandes_batched, brandes_batched_host, brandes_host, brandes_pp,
    brandes_pp_host, brandes_noalloc, brandes_pp_st, brandes_pp_all, build_arena, Plan, autotune, autotune_batched, partition_lp, plan_brandes, plan_brandes_pp, csr_build, csr_validate, default_context, graph_from_edgelist, load_library,
    shard_bounds, skeleton, sssp,
)
from . import sharded  # noqa: F401

__all__ = [
    "Arena", "BcppError", "Context", "Graph", "HostCSR", "SigmaOverflow", "brandes", "brandes_batched",
    "brandes_batched_host",
    "brandes_host", "brandes_noalloc", "brandes_pp", "brandes_pp_st", "brandes_pp_all", "brandes_pp_host", "build_arena", "csr_build", "csr_validate", "default_context",
    "graph_from_edgelist", "load_library", "Plan", "autotune", "autotune_batched", "partition_lp", "plan_brandes", "plan_brandes_pp", "shard_bounds", "sharded", "skeleton", "sssp",
]
