"""GB300-native spectral semi-Lagrangian Gauss-Newton-Krylov registration.

The compute path is a C-ABI CUDA library (``libreg.so``, built from ``csrc/``
for sm_103a); ``paper_1608_03630_gb300.reg`` is its thin Python binding
(argument marshalling only), ``learned_init`` drives the U-Net initial
velocity (training pairs from the solver, training, evaluation) and
``synth`` makes seeded synthetic inputs.
Importing this package loads nothing; the library is loaded on first use of
``reg`` and a missing or unbuildable library raises instead of falling back.
"""
