"""GB300 (sm_103a) implicit neutrino--matter collision solve.

The compute path is the C-ABI library ``libnmc.so`` (``include/nmc.h``) built from
``csrc/``; ``nmc`` is its thin ctypes binding and ``synthetic`` produces seeded
input data.
"""

from . import synthetic  # noqa: F401
