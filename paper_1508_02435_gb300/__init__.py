"""GB300-native particle-in-tree / particle-in-dual-tree particle step.

The compute path is the C-ABI library ``libpic.so`` built from ``csrc/``
(hand-written CUDA for sm_103a); :mod:`paper_1508_02435_gb300.pic` is its thin
Python binding.  :mod:`paper_1508_02435_gb300.workloads` holds the seeded input
generators.
"""
