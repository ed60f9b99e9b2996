"""GB300-native SLPIC-MCC (speed-limited particle-in-cell with Monte-Carlo
collisions) for a 1D3V argon-filled parallel-plate gap.

The compute path is the CUDA library ``libslpic.so`` behind the C-ABI declared
in ``include/slpic.h``; :mod:`paper_2103_12194_gb300.slpic` is its thin Python
binding.  :mod:`paper_2103_12194_gb300.inputs` generates seeded synthetic
inputs.
"""
