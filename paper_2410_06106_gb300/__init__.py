"""GB300-native decentralized ADMM tomography with quantized messages.

The compute path is the C-ABI library ``libtomo.so`` (hand-written CUDA for
sm_103a, declared in ``include/tomo.h``); ``api`` is its thin Python binding.
Importing this package does not load the library: the first call into
``api`` does, and fails loudly if the library has not been built.
"""
__all__ = ["api", "synth"]
