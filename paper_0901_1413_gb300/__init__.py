"""Exact dense matrix products over F_3, F_5, F_7 and GF(4) on GB300 (sm_103a).

Boothby & Bradshaw, "Bitslicing and the Method of Four Russians Over Larger
Finite Fields": bitsliced bit-plane matrices and the Method of Four Russians
with an additive basis, as hand-written CUDA behind a small C ABI
(``include/fq.h``).  ``paper_0901_1413_gb300.fq`` is the Python binding;
``paper_0901_1413_gb300.inputs`` draws seeded synthetic inputs.
"""
