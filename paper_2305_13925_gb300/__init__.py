"""GB300 (sm_103a) Jac-PCG regularized zero-forcing precoder.

The compute path is the CUDA library libjacpcg.so behind the C ABI of
include/jacpcg.h; ``binding`` is its thin ctypes face and ``channels`` the
seeded synthetic-channel generator.  Importing the package does not load
the library; the first call into ``binding`` does, and raises if it is not
built.
"""
from . import binding, channels  # noqa: F401
from .binding import Precoder, instance  # noqa: F401

__all__ = ["binding", "channels", "Precoder", "instance"]
