"""GB300-native (sm_103a) HHS-FSI hot path: direct-summation acceleration, force-gradient
and symmetrised time-step passes, on-device slow/fast partition and kick/drift, behind the
C-ABI declared in include/frost.h.

Submodules:
  frost  -- ctypes binding of libfrost.so (same names as the C-ABI); imports lazily
  ics    -- seeded synthetic initial conditions (Plummer, Kroupa, binaries, cluster batches)
  build  -- nvcc build of libfrost.so for sm_103a
"""

__all__ = ["frost", "ics", "build"]
