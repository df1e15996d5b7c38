"""GB300-native forward dynamics of serial chains (ABIA, JSIIA, CFA with OEE).

The CUDA library is loaded lazily by :mod:`paper_1609_06779_gb300.fd` on first
use; importing the package does not need a GPU.
"""
__all__ = ["fd", "synth", "build"]
