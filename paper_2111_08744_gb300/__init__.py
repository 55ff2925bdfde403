"""GB300-native null-geodesic ray tracing through AMR potentials (arXiv 2111.08744 method).

The compute path lives in the CUDA library built from `csrc/` and is reached
through `paper_2111_08744_gb300.binding`; importing this package does not load it.
"""
__all__ = ["inputs", "binding"]
