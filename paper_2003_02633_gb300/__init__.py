"""Inline 3-vector compression (Trojak & Witherden, arXiv:2003.02633) on GB300.

The compute path lives in a C-ABI shared library built from ``csrc/`` for
sm_103a; ``ivc`` is its ctypes binding.  ``synth`` draws the seeded inputs.
"""
__all__ = ["ivc", "synth"]
