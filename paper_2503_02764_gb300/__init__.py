"""GB300-native FLD radiation substep (limiter, backward-Euler multigrid diffusion,
gas-radiation exchange) behind a C-ABI CUDA library.

The CUDA binding lives in ``paper_2503_02764_gb300.fld`` and is loaded on first
use; ``paper_2503_02764_gb300.inputs`` holds the seeded input recipes.
"""
