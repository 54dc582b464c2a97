"""GB300-native PRIEST projection library (arXiv 2309.08235).

The compute path is the C-ABI library ``libpriest.so`` (CUDA kernels for
sm_103a); ``paper_2309_08235_gb300.priest`` is its thin ctypes binding.
``paper_2309_08235_gb300.workloads`` holds seeded synthetic inputs only.
"""
