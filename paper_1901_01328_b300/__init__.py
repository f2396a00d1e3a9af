"""KPA grouping path of StreamBox-HBM on B300 (sm_103a).

The kernels and the C ABI live in libsbh.so (sources in csrc/, header in
include/sbh.h); ``sbh`` is the Python binding (argument marshalling only).
"""
from . import sbh  # noqa: F401  (raises ImportError when libsbh.so is missing)
from .sbh import *  # noqa: F401,F403
