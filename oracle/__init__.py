"""FP64 CPU oracle of the temporally adaptive finite-volume solver.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may import this package.
It shares no code with the CUDA path.
"""
