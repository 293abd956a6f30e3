"""GB300-native E-field direct imaging (MOFF / EPIC) behind a small C-ABI.

The imaging path is hand-written CUDA for sm_103a in ``libepic.so``; the
Python side (``epic``) only marshals arguments to it.  ``synth`` draws the
seeded synthetic inputs.
"""
__all__ = ["epic", "synth"]
