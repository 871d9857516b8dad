"""FP64 CPU oracle of the two-level Schwarz method.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py``; never by the product
package.
"""
from .asm_oracle import *  # noqa: F401,F403
from . import asm_oracle  # noqa: F401
