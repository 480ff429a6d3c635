"""Seeded synthetic workloads (scene synthesis only; none of the method's arithmetic)."""
from .gen import Workload, tiny, tracking, global_graph, batched, differentiation  # noqa: F401
