"""GB300 Katz-query library: LRC-Katz and plain CG on M = I - beta W.

The compute lives in libkatz.so (CUDA, sm_103a); ``katz`` is its ctypes
binding and ``synth`` draws seeded synthetic graphs and query sets.
"""
