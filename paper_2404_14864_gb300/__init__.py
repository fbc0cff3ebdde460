"""GB300-native KFBI operator application (arXiv 2404.14864).

The CUDA library (``_build/libkfbi.so``) is loaded lazily by
``paper_2404_14864_gb300.kfbi``; importing this package alone loads nothing.
"""
