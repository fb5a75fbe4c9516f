"""GB300-native (sm_103a) TPC track reconstruction: CA seeding, Kalman following, sector merging,
Kalman refit and its calibration adjoint (arxiv 1712.09434, section 3).

The compute path is ``libtpc.so`` (C ABI in ``include/tpc.h``); ``capi`` is its Python binding.
``synth`` generates seeded synthetic events.
"""
