"""Microbenchmarks of per-SM instruction rates (``python -m paper_0901_1413_gb300.microbench``).

Builds ``rates.cu`` and ``tcgen05_rate.cu`` for sm_103a with nvcc and runs them
on cuda:0; prints one JSON line per probe (operations per clock per SM, and for
``rates.cu`` the implied clock and whole-GPU rate).
"""
