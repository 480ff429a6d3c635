"""Seeded synthetic workloads (scene synthesis only; none of the method's arithmetic)."""
from .gen import Workload, batched, batched_graph, batched_storage, differentiation, global_graph, merge, tiny, tracking  # noqa: F401
