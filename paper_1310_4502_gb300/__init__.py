"""GB300-native hashed oct-tree gravity (Warren 2013, "2HOT") force path.

Importing the package is cheap: the CUDA library is loaded on first use by
``paper_1310_4502_gb300.hot`` and raises if it is missing.
"""
