"""FP64 CPU oracle for the occ-RI-K exchange build -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package. The product
path (the CUDA library and its Python binding) never imports, calls or links
anything here, and this package imports nothing from the product path.

Every function is a plain, slow restatement of a definition or algorithm of
Lee, Rettig, Feng, Epifanovsky and Head-Gordon (arXiv:2207.09028), citing the
section or equation it follows. Pins against closed forms, invariants and
brute force live in ``tests/test_oracle_pins.py``. No function here is
"parity unpinned".
"""
from .occri_oracle import *  # noqa: F401,F403
