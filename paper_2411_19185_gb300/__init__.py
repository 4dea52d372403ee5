"""GB300 (sm_103a) implementation of the per-Runge-Kutta-stage tendency of HOPE's
cubed-sphere shallow-water core (arXiv 2411.19185) behind a C ABI (include/hope.h).
"""
from ._lib import (HOPE_TPP, HOPE_WENO2D, HOPE_WENO1D, HOPE_FP64, HOPE_FP32, HOPE_SSPRK3, HOPE_WSRK3,  # noqa: F401
                   HopeError, load)
from .hope import Sphere, measure_fma_peak, measure_fma_peak_clock, IC_GEOSTROPHIC, IC_ROSSBY, IC_DAMBREAK, IC_BUMPS  # noqa: F401
from .hope import IC_MOUNTAIN_SURFACE, IC_MOUNTAIN_FLOW, IC_JET, MOUNTAIN, JET  # noqa: F401
