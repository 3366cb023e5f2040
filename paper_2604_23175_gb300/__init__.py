"""GB300-native multi-area WLS state estimation (boundary-condensed
Gauss-Newton, arXiv 2604.23175).

The compute path is the C-ABI library ``libmase`` (CUDA, sm_103a) built from
``csrc/``; :mod:`paper_2604_23175_gb300.mase` is its thin ctypes binding.
Importing this package does not load the library; :func:`mase.load` does,
and raises if it is missing.  :mod:`paper_2604_23175_gb300.synth` draws the
seeded synthetic inputs.
"""
__all__ = ["synth", "mase"]
