"""GB300-native monopole + quadrupole tree-force hot path (arXiv:1812.07313).

``qgrav``     -- binding of the ``qg_*`` C-ABI (CUDA, sm_103a)
``tree``      -- host oct-tree / group walk producing the interaction lists
``workloads`` -- seeded synthetic particle sets
"""
