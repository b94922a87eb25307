"""GB300-native HOPU convection hot path (arXiv 2408.06698), behind the libhopu C ABI.

``build.build()`` compiles libhopu.so for sm_103a; ``hopu.Hopu`` binds a context.
"""
from .hopu import ConvectionApply, Hopu, HopuBatch, HopuHex, Rollout, measure_alu_peak, selftest  # noqa: F401
