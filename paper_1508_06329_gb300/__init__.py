"""GB300 (sm_103a) parallel chordality test: LexBFS by partition refinement
plus the perfect-elimination check, in hand-written CUDA behind the C ABI of
``include/chordal.h`` (libchordal.so).  ``binding`` is the thin ctypes layer;
torch supplies device memory and streams only.
"""
__version__ = "0.1.0"
