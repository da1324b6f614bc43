"""Plain FP64 CPU oracle for low-precision Gaussian-process solves.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the tests, the ``smoke()`` self-check and the CPU
baseline leg of the benchmark use it.  It shares no code with the CUDA path;
both sides receive the same seeded arrays and nothing else.

Every function follows the paper ("Low-Precision Arithmetic for Fast Gaussian
Processes", Maddox, Potapczynski & Wilson, 2022) by section / equation /
algorithm, written for a reader checking it against the paper by eye: no
blocking beyond what memory forces, no fusion, no reordering.
"""

from .gp_oracle import *  # noqa: F401,F403
