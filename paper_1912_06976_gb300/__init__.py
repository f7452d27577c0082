"""GB300-native fast BTTB forward / transpose products for 3-D gravity and magnetic prisms.

The CUDA library behind the C ABI (include/gravmag.h) is loaded lazily by
``paper_1912_06976_gb300.gravmag`` so that the seeded workload generators can
be imported on machines without a GPU.
"""
__all__ = ["workloads"]
