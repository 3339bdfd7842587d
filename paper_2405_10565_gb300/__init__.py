"""GB300 (sm_103a) level-of-detail strand-hair ray tracer.

The product is the C ABI library ``libhairrt.so`` (include/hairrt.h); this
package holds its CUDA sources (``csrc/``), the in-tree build
(``build.py``) and a thin ctypes binding (``_lib.py``) whose functions carry
the C entry points' names.
"""
from ._lib import *  # noqa: F401,F403
from ._lib import HairRTError, load, ptr, render_desc, camera, header_functions  # noqa: F401
