"""Microbenchmarks of per-SM instruction rates (``python -m paper_0901_1413_gb300.microbench``).

Builds ``rates.cu`` for sm_103a with nvcc and runs it on cuda:0; prints one JSON
line per probe (operations per clock per SM, implied clock, whole-GPU rate).
"""
