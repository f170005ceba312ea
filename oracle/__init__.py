"""Plain CPU oracle for quasi-F-split heights -- test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import this package.
The product path (``paper_2502_12428_gb300``) never imports it and shares no code with it.
"""
from .oracle import *  # noqa: F401,F403
