"""GB300-native Moment Tensor Potential hot path (MLIP-3 method, arXiv 2304.13144).

Importing the package is cheap; the CUDA library is loaded on first use by
`paper_2304_13144_gb300.api` and fails loudly if it has not been built.
"""
__all__ = ["basis", "synth", "api"]
