"""GB300-native DeepMatching hot path (descriptors, correlation pyramid,
backtracking, reciprocal verification) behind a C-ABI CUDA library.

``paper_1506_07656_gb300.dm`` is the binding to that library; ``synth`` makes
seeded synthetic inputs.  Importing the package loads nothing native.
"""
