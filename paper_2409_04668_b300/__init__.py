"""B300-native Monte Carlo neutron transport (time-dependent, multigroup,
fixed-source, non-multiplying) behind a C-ABI CUDA library.

Importing the package loads nothing; ``paper_2409_04668_b300.mcdc`` binds the
C-ABI library and fails loudly if it is missing.
"""
