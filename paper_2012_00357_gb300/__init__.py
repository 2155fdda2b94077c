"""GB300 (sm_103a) data-driven computational mechanics: the per-iteration
nearest-data projection P_D and constraint projection P_C of Eggersmann,
Stainier, Ortiz & Reese (arXiv:2012.00357), behind the C ABI of
include/dd.h (libdd.so).  This package is the thin Python binding."""
from .binding import *  # noqa: F401,F403
from .binding import lib, DDError, Result, EXPORTS  # noqa: F401
from ._build import build  # noqa: F401
