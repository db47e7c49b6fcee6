"""FP64 CPU oracle of the hexagonal porous Saint-Venant step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  It shares no code with the CUDA library.
"""
from .oracle import (Problem, Ledger, friction, sigma, phi, build, from_scenario, max_threads, WALL, FREE, W, E, S, N)  # noqa: F401
