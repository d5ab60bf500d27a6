"""GB300 (sm_103a) implementation of the field-dislocation-mechanics layer-case time step
of Morin, Brenner & Suquet (arXiv 1911.03225): FFT static solve, stress-driven celerity and
the Kurganov-Noelle-Petrova central-upwind transport, behind the C ABI of include/fdm.h."""
from .binding import Batch, FDM, FDMError, Params, StepInfo, load  # noqa: F401
