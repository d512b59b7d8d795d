"""GB300-native UMI sliding-window asymmetric robust detrending.

The compute path is the C-ABI library ``libumi.so`` (hand-written CUDA for
sm_103a, see ``include/umi.h``); ``umi`` is its thin ctypes binding.
"""
