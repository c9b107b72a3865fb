"""ORACLE — test infrastructure only.

Plain, slow, obviously-correct CPU restatement (FP64 / complex128) of the
method of arXiv 2411.18026.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with the CUDA path in ``paper_2411_18026_gb300``.
"""
