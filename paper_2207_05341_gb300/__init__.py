"""GB300-native NN-QST maximum-likelihood hot path (arXiv:2207.05341).

The CUDA library (``libqst.so``) is loaded lazily by :mod:`.qst`, so that
importing :mod:`.synth` alone never touches a GPU or the shared library.
"""
