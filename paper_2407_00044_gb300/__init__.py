"""Stream-K GEMM for NVIDIA GB300 (sm_103a).

The compute path is the C-ABI library ``lib/libskgemm.so`` (hand-written
TMA + tcgen05/TMEM kernels and an FP32 SIMT kernel); this package only
marshals tensors into it.  Importing the package loads the library and
raises if it has not been built -- there is no fallback path.
"""
from . import binding
from .binding import SkError, load as _load

_load()

from .api import (Config, Workspace, default_workspace, gemm, gemm_backward,  # noqa: E402
                  grouped_gemm, layout_of, make_problem, plan, quantize_e4m3,
                  shape_problem, trace_gemm, transpose16, unit_items)
from .autograd import SkMatmul, sk_matmul  # noqa: E402
from . import autotune  # noqa: E402
from .pipeline import HostGemmPipeline  # noqa: E402

__all__ = ["binding", "SkError", "Config", "Workspace", "default_workspace", "gemm", "HostGemmPipeline",
           "gemm_backward", "grouped_gemm", "layout_of", "make_problem", "plan",
           "quantize_e4m3", "shape_problem", "trace_gemm", "transpose16", "unit_items", "SkMatmul", "sk_matmul", "autotune"]
