"""GB300-native (sm_103a) Valencia GRMHD meshblock RHS and update (arXiv:2409.10384).

The compute path is the C-ABI library ``libgrmhd`` (hand-written CUDA, see
``csrc/``); ``grmhd`` is its thin ctypes binding and ``synth`` the seeded
synthetic-input generators.
"""
