"""GB300-native reverse time migration with quantified uncertainty.

The compute path is a CUDA shared library (``csrc/``, C ABI in
``include/rtm.h``) for sm_103a; ``rtm`` is its thin ctypes binding and
``inputs`` makes seeded synthetic inputs.  Importing the package loads
nothing; the library is loaded on first use and a missing or unbuildable
library raises instead of falling back to anything else.
"""

__all__ = ["rtm", "inputs"]
