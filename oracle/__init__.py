"""CPU FP64 oracle for the OkMC + FFT elastic-interaction hot path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it. The
product path (``paper_2403_09158_gb300``) never imports, links or runs anything
here, and this package never imports the product path: the two share no code.
"""
from .okmc_oracle import *  # noqa: F401,F403
