"""GB300-native fused collide-stream step of the coupled D1Q3Q3 entropy lattice Boltzmann scheme
(Dubois, Graille, Lallemand, sections 6 and 8), with the paper's finite-difference comparison solver
(section 9) and single-distribution D1Q3 schemes (sections 2 and 4).

Importing the package loads nothing compiled; ``paper_1802_02369_gb300.lbm`` loads the CUDA
library ``liblbm.so`` on first use and raises if it is missing.
"""
__all__ = ["lbm", "workloads"]
