"""FP64 CPU oracle for the HICU hot path.

Test infrastructure, not product code: only tests/, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA library in ``paper_2004_08962_gb300``.
"""
from . import hicu_oracle  # noqa: F401
