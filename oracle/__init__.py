"""FP64 CPU oracle for the PPRviz hot path. TEST INFRASTRUCTURE ONLY.

Only tests, the smoke check in __graft_entry__ and the CPU-baseline leg of
bench.py may import this package. The product path (the C-ABI library and its
Python binding) never imports, links or executes anything here.
"""
from .pprviz_oracle import *  # noqa: F401,F403
from .pprviz_oracle import __all__  # noqa: F401
from .hierarchy import *  # noqa: F401,F403,E402
from .hierarchy import __all__ as _hier_all  # noqa: E402

__all__ = list(__all__) + list(_hier_all)
