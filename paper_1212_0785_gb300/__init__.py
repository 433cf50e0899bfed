"""GB300-native device-resident Hybrid Monte Carlo for SU(3) lattice gauge theory
with two flavours of Wilson fermions.

The compute path is the C-ABI library ``liblqcd.so`` (hand-written CUDA kernels
for sm_103a, declared in ``include/lqcd.h``); ``lqcd`` is its thin ctypes binding.
"""
__all__ = ["inputs", "lqcd"]
