"""CPU oracle for the Hypercube-Givens Transform (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product package never imports it,
and it imports nothing from the product package.
"""
from .oracle import *  # noqa: F401,F403
