"""GB300-native randomized proximal TT-ALS with TensorSketch (TT-TS).

The compute path lives in a C-ABI CUDA library (``libttsketch.so``, declared in
``include/tt_sketch.h``); ``paper_2309_08093_gb300.lib`` is a thin ctypes binding to it and
``paper_2309_08093_gb300.synth`` builds seeded synthetic inputs. Importing the package does not
load the CUDA library; ``lib.load()`` does, and fails loudly when it is missing.
"""
