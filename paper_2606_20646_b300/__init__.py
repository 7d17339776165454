"""B300-native total-Lagrangian vectorial LBM (arXiv 2606.20646): the collide-stream
sweep with level-set cut-link closure and compatibility projection, as hand-written
sm_103a CUDA kernels behind a C ABI (``include/lbm.h``).

Importing the package loads nothing; ``paper_2606_20646_b300.lbm`` loads the CUDA
library and fails loudly when it is missing.
"""
