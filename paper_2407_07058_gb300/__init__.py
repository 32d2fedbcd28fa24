"""GB300-native all-pairs minimax-path (APPD) library (arxiv 2407.07058).

The public API is the C ABI in include/appd.h; ``paper_2407_07058_gb300.appd``
is its Python binding.
"""
from . import appd  # noqa: F401
from .appd import (AppdError, Server, check_symmetric, last_device_status, leaf_order, mst,  # noqa: F401
                   solve, solve_alg4, solve_batched, solve_host)
