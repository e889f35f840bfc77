"""GB300-native preconditioned FR/CPR implicit hot path (Wang & Yu, arXiv 1903.06304).

Importing the package is cheap and loads no compiled code.  The CUDA path lives in
``paper_1903_06304_gb300.fr`` (C-ABI binding); seeded synthetic workloads live in
``paper_1903_06304_gb300.inputs``.
"""

__all__ = ["inputs", "fr"]
