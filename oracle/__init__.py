"""Plain FP64 CPU oracle of the SPFOM iteration -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline /
reference leg may import this package. The solver library never does, and the
two share no code (both read instances from the ``instances`` generator).
"""
from .oracle import Oracle, OracleRun, Params, build, sample_hash

__all__ = ["Oracle", "OracleRun", "Params", "build", "sample_hash"]
