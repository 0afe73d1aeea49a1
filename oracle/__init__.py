"""CPU oracle of the dense-block recursive-skeletonization inverse (arXiv:1303.5466).

Test infrastructure only: tests, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline may use it; the product library never does.
"""
from .oracle import *  # noqa: F401,F403
