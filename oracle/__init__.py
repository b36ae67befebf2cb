"""FP64 CPU oracle for the lattice-sum path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA library never does, and this
package never imports the library.
"""
from .lattice_oracle import *  # noqa: F401,F403
