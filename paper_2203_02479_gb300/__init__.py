"""GB300-native (sm_103a) LArTPC signal simulation hot path (arXiv 2203.02479).

``wiresim`` is the Python binding of the C ABI in ``include/wiresim.h``;
``inputs`` draws seeded synthetic depos and responses; ``build`` compiles the
CUDA library in-tree.  Importing the package does not load the library: the
first call into ``wiresim`` does, and fails loudly if it was not built.
"""
from . import inputs  # noqa: F401
from .wiresim import (DeviceDepos, Params, Plane, WiresimError,  # noqa: F401
                      load_library)
