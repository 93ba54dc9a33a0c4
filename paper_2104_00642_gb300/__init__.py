"""GB300-native relativistic electromagnetic PIC hot path (Song, Wang & Li,
arXiv:2104.00642): hand-written sm_103a CUDA behind a C ABI (``libpic.so``).

The binding is in :mod:`paper_2104_00642_gb300.pic`; the seeded synthetic
inputs are in :mod:`paper_2104_00642_gb300.workloads`.
"""
