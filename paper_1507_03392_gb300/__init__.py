"""GB300-native ECRIS ion time step (arXiv:1507.03392): CUDA kernels behind a C ABI.

Importing the package loads nothing compiled; `paper_1507_03392_gb300.ecris`
loads the CUDA library and fails loudly if it is missing.
"""
