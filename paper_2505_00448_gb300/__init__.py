"""GB300-native all-pairs statistical tests with pairwise deletion (NApy, arXiv 2505.00448).

Importing the package loads nothing; `paper_2505_00448_gb300.napg` binds the
CUDA library (and fails loudly when it is missing), `synth` draws inputs.
"""
__all__ = ["napg", "synth"]
