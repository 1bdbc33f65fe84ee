"""CPU FP64 oracle of the spin-1 GPE split-step hot path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference leg of ``bench.py`` may import it.  The CUDA library and its binding never do.
"""
