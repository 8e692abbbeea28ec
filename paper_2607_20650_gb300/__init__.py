"""GB300-native D2Q9I lattice-BGK stream-and-collide (PortLBM, arXiv 2607.20650).

``paper_2607_20650_gb300.lbm`` binds the C ABI of ``liblbm.so`` (CUDA kernels
for sm_103a); ``paper_2607_20650_gb300.geometry`` builds seeded inputs.
Importing the package loads nothing: the binding loads the library on first
use and raises if it is missing.
"""
