"""FP64 CPU oracle (test infrastructure only; never imported by the library)."""
from .oracle import *  # noqa: F401,F403
from .oracle import Operator, WILSON, BRILLOUIN, STAGGERED  # noqa: F401
