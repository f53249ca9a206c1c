"""FP64 CPU oracle for the Lennard-Jones MD hot path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or calls it, and shares no code,
tables or constants with it.

The oracle computes the plain definitions: all-pairs O(N^2) forces with the
Eq. 2 truncated potential, velocity-Verlet, energies, the brute-force pair set
within the search length, the cell labels and counting sort of the grid method
(Sec. 2.2), the sorted pair list (Sec. 2.4, KeyPointer/SortedList), and the
derivatives used by the differentiable form.
"""
from .oracle import *  # noqa: F401,F403
