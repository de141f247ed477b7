"""GB300-native (sm_103a) loss, gradient and Hessian-vector product of the
sampled Hilbert-Schmidt cost of a brickwall circuit, by recursive
tangent-state propagation (arXiv 2604.20384).

Importing the package loads nothing native; the CUDA library is loaded on
first use by :mod:`paper_2604_20384_gb300.native` and raises if it is absent.
"""
__all__ = ["inputs"]
