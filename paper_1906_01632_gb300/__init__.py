"""GB300-native implicit time step of the stochastic 3D Elder problem.

Importing the package loads nothing native; ``paper_1906_01632_gb300.elder``
loads the CUDA library and raises if it is missing.
"""
__all__ = ["elder", "inputs"]
