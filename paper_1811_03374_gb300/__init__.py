"""GB300-native ray/fiber intersection (Binder & Keller, arXiv 1811.03374).

The CUDA library is loaded on first use (``paper_1811_03374_gb300.fiberx``);
importing the package itself touches no GPU.
"""
__all__ = ["inputs"]
