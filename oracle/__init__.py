"""CPU oracle for the range-separated (RS) canonical/Tucker Newton-potential method.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow FP64 statement of what
the CUDA path computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` may import it; the library and its Python
binding never do, and the oracle never imports them.  The two share no code: the
only common dependency is the ``workloads`` package, which generates seeded inputs
and holds none of the method's arithmetic.

Parity status: every function in ``rs_oracle`` is pinned by ``tests/test_oracle_pins.py``
against closed forms, numerical integration, brute force on tiny grids, textbook
constants or invariants; no function is "parity unpinned".
"""
from . import rs_oracle  # noqa: F401
