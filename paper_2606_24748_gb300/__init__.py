"""Blocked smoothed-aggregation AMG reuse phase on one GB300 (sm_103a).

The compute lives in ``libbamg.so`` (CUDA kernels behind the C ABI of
``include/bamg.h``); :mod:`paper_2606_24748_gb300.bamg` is the thin binding
and :mod:`paper_2606_24748_gb300.bytes_model` the algorithmic byte and flop
counts used for roofline reporting.
"""
