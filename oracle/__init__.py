"""Plain, slow FP64 CPU oracle for Poisson MaZe.

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import this
package: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it. It shares no code with the CUDA path; both receive
their inputs from the seeded generator in ``paper_2505_20418_gb300.synth``.
"""
from .maze_oracle import *  # noqa: F401,F403
