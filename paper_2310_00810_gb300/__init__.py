"""GB300 (sm_103a) differentiable lattice Boltzmann hot path of arXiv 2310.00810.

The compute path lives in the C-ABI shared library built from ``csrc/``
(declared in ``include/lbm.h``); ``lbm`` is its thin ctypes binding and
``autograd`` wraps it in a ``torch.autograd.Function``.
"""
