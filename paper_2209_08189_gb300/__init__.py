"""GB300-native semi-Lagrangian Gauss-Newton-Krylov registration hot path
(arXiv 2209.08189).  The compute path is the C-ABI library ``libclaire.so``
built from ``csrc/``; ``claire`` is its thin ctypes binding and ``synth``
draws seeded synthetic inputs."""
