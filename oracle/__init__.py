"""TEST INFRASTRUCTURE ONLY: the plain FP64 CPU oracle of the HOPE shallow-water core.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It shares no code with the CUDA library.
"""
from .oracle import Oracle, build_oracle, gauss, weights_1d, tpp_weights_2d, \
    tpp_weights_2d_literal, weno_gamma, weno_beta, metric, jacobian, xyz, locate  # noqa: F401
