"""B300-native batched simulator of the EMT6/Ro spheroid CA under radiotherapy
protocols (arxiv 2303.08123), behind the C ABI in include/sim.h.

  sim        ctypes binding of libsim (Simulator, make_config, csr)
  _build     nvcc build of the in-tree shared libraries (sm_103a)
"""
from .sim import Simulator, SimError, make_config, csr, load_library  # noqa: F401
