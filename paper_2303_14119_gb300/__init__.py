"""GB300-native solver for one explicit time step of the 1D2V continuum-kinetic
model of vacuum surface flashover (Sun et al., arXiv 2303.14119).

``fk`` is the Python binding of the C ABI (``include/fk.h``) implemented by
the CUDA library ``libflashkin.so``; ``synth`` generates the seeded
synthetic inputs; ``_build`` compiles the library for sm_103a.
"""
__all__ = ["fk", "synth"]
