"""GB300-native simplex-in-cell (SIC) Vlasov-Poisson step (arXiv:1506.07207).

The hot path (deposit of sheet segments by exact overlap integration, the
periodic field solve, linear gather and leapfrog push) runs in hand-written
sm_103a CUDA behind the C ABI declared in ``include/sic.h``.  ``sic`` is the
thin ctypes binding with the same names; importing it loads the CUDA library
and fails loudly when it is missing.  ``inputs`` builds seeded synthetic
initial conditions and holds none of the method's arithmetic.
"""
__version__ = "0.1.0"
