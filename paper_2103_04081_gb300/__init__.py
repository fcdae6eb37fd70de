"""GB300-native block-randomized weighted SGD for CP decomposition.

Importing the package loads nothing; ``paper_2103_04081_gb300.cpd`` loads the
CUDA library and fails loudly if it has not been built.
"""
