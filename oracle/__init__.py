"""CPU oracle for the DGP scalar-field FAS solver: test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import anything from here.  The CUDA library never does.
"""
