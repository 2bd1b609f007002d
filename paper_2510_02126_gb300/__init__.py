"""liblyap: mixed-precision iterative refinement for low-rank Lyapunov equations on GB300.

The compute path is the C-ABI shared library ``liblyap.so`` (CUDA, sm_103a);
``paper_2510_02126_gb300.lyap`` is its ctypes binding (import it explicitly).
There is no CPU fallback: loading fails loudly when the library is missing.
"""
from . import build_lib  # noqa: F401
