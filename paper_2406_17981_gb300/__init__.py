"""btmv: split-FFT block Toeplitz matrix-vector product for one GB300 GPU.

The compute path is the C-ABI shared library ``libbtmv.so`` built from
``csrc/`` (hand-written sm_103a CUDA); ``btmv`` is its thin ctypes binding.
"""
