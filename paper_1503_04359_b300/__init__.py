"""Direction-optimized BFS on one B300: CUDA kernels for sm_103a behind a C ABI.

``paper_1503_04359_b300.dobfs`` is the Python binding of ``libdobfs.so``;
``paper_1503_04359_b300.build`` compiles it.
"""
