"""GB300-native separable tensor-operator solver (computational tensor algebra).

Importing the package loads nothing native; ``paper_1001_5460_gb300.tca``
loads the CUDA library and fails loudly when it is missing.
"""
__all__ = ["synth"]
