"""GB300-native parallel orbital-updating Kohn-Sham minimisation (arXiv 1510.07230).

The compute path lives in the C-ABI library ``libpou.so`` (hand-written CUDA
for sm_103a); :mod:`paper_1510_07230_gb300.pou` is its thin ctypes binding.
"""
