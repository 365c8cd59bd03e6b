"""GB300 library for the hybrid lattice-Boltzmann / finite-difference step of
Gonnella, Lamura & Tiribocchi, "Thermal and hydrodynamic effects in the
ordering of lamellar fluids" (arXiv:1102.3094).

The method runs in ``liblf.so`` (CUDA, sm_103a) behind the C ABI of
``include/lf.h``; ``lf`` is the ctypes binding of that ABI.
"""
from . import lf  # noqa: F401
