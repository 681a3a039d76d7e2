"""Torch-tensor front end of the C ABI: reads shapes, strides, dtypes and
device pointers off tensors, owns a per-device workspace, and calls the
library on the current CUDA stream.  No arithmetic happens here.
"""
from __future__ import annotations

import ctypes
import threading
from dataclasses import dataclass

import torch

from . import binding as B

_DTYPES = {torch.float32: B.SK_F32, torch.bfloat16: B.SK_BF16,
           torch.float8_e4m3fn: B.SK_E4M3, torch.uint8: B.SK_E4M3}
_OUT_TORCH = {B.SK_F32: torch.float32, B.SK_BF16: torch.bfloat16}


@dataclass
class Config:
    """Python mirror of ``sk_config`` (0 / 'auto' = library default)."""
    tile_m: int = 0
    tile_n: int = 0
    stages: int = 0
    mode: str = "auto"
    num_ctas: int = 0
    min_iters_per_unit: int = 0
    timeout_ns: int = 0
    debug_flags: int = 0
    trace: int = 0          # device pointer of a timeline buffer (see trace_gemm)
    raster_group: int = 0   # rasterisation group in tile rows (0 = default)
    fixup: str = "owner"    # "owner" (owner waits for peers), "last_arriver", "split" or "split_cluster"
    f32_kernel: str = "auto"   # FP32 problems: "auto", "ffma" or "tf32x3"
    coverage: int = 0       # device pointer of a coverage-count buffer (see coverage_counts)

    def to_c(self) -> B.sk_config:
        c = B.sk_config()
        c.tile_m = self.tile_m
        c.tile_n = self.tile_n
        c.stages = self.stages
        c.mode = B.MODE_NAMES[self.mode] if isinstance(self.mode, str) else int(self.mode)
        c.num_ctas = self.num_ctas
        c.min_iters_per_unit = self.min_iters_per_unit
        c.timeout_ns = self.timeout_ns
        c.debug_flags = self.debug_flags
        c.trace = self.trace or None
        c.raster_group = self.raster_group
        c.fixup = B.FIXUP_NAMES[self.fixup] if isinstance(self.fixup, str) else int(self.fixup)
        c.f32_kernel = (B.F32_KERNEL_NAMES[self.f32_kernel] if isinstance(self.f32_kernel, str)
                        else int(self.f32_kernel))
        c.coverage = self.coverage or None
        return c


def _cfg(config) -> B.sk_config:
    if config is None:
        return Config().to_c()
    if isinstance(config, B.sk_config):
        return config
    if isinstance(config, dict):
        return Config(**config).to_c()
    return config.to_c()


def layout_of(t: torch.Tensor, prefer=None):
    """(sk_layout, leading dimension) of a 2-D tensor, from its strides.

    A single row or column is contiguous in both layouts; ``prefer`` picks
    the one the caller wants then (A row-major and B column-major keep
    both operands K-major, which the TMA path needs for a vector operand)."""
    if t.dim() != 2:
        raise ValueError("expected a 2-D tensor")
    r, c = t.shape
    if t.numel() == 0:
        return B.SK_ROW_MAJOR, max(1, c)
    s0, s1 = t.stride()
    pad16 = lambda x: -(-max(1, x) // 16) * 16   # noqa: E731
    if prefer == B.SK_COL_MAJOR and c == 1 and (s0 == 1 or r == 1):
        return B.SK_COL_MAJOR, pad16(r)
    if prefer == B.SK_ROW_MAJOR and r == 1 and (s1 == 1 or c == 1):
        return B.SK_ROW_MAJOR, pad16(c)
    if s1 == 1 and (r <= 1 or s0 >= max(1, c)):
        ld = s0 if r > 1 else -(-max(1, c) // 16) * 16
        return B.SK_ROW_MAJOR, ld
    if s0 == 1 and (c <= 1 or s1 >= max(1, r)):
        ld = s1 if c > 1 else -(-max(1, r) // 16) * 16
        return B.SK_COL_MAJOR, ld
    raise ValueError(f"tensor with strides {t.stride()} is neither row- nor column-major")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def make_problem(A: torch.Tensor, Bm: torch.Tensor, C: torch.Tensor, *, C_in=None,
                 alpha: float = 1.0, beta: float = 0.0, scale_a=None, scale_b=None) -> B.sk_problem:
    M, K = A.shape
    K2, N = Bm.shape
    if K != K2 or tuple(C.shape) != (M, N):
        raise ValueError(f"shape mismatch A{tuple(A.shape)} B{tuple(Bm.shape)} C{tuple(C.shape)}")
    p = B.sk_problem()
    p.m, p.n, p.k = M, N, K
    p.a_type = _DTYPES[A.dtype]
    p.b_type = _DTYPES[Bm.dtype]
    p.c_type = _DTYPES[C.dtype]
    p.a_layout, p.lda = layout_of(A, B.SK_ROW_MAJOR)
    p.b_layout, p.ldb = layout_of(Bm, B.SK_COL_MAJOR)
    p.c_layout, p.ldc = layout_of(C, B.SK_ROW_MAJOR)
    p.A = A.data_ptr()
    p.B = Bm.data_ptr()
    p.C = C.data_ptr()
    p.C_in = C_in.data_ptr() if C_in is not None else None
    if C_in is not None and (C_in.dtype != C.dtype or C_in.stride() != C.stride()):
        raise ValueError("C_in must have C's dtype and strides")
    p.alpha = float(alpha)
    p.beta = float(beta)
    p.scale_a = scale_a.data_ptr() if scale_a is not None else None
    p.scale_b = scale_b.data_ptr() if scale_b is not None else None
    return p


def default_workspace_bytes(sms: int) -> int:
    """Workspace for any call on a GPU with ``sms`` SMs: status word (256 B),
    the fixed flag region (1024 words), and two 128 x 512 FP32 slots per CTA
    (a CTA's share of the widest tile, 256 x 512 on a CTA pair; the second
    slot is used by the last-arriver fixup only)."""
    return 256 + 4096 + 2 * sms * 128 * 512 * 4


class Workspace:
    """A zero-initialised device buffer large enough for any call on one
    device (sized for the largest tile, every SM and either fixup)."""

    def __init__(self, device=None, nbytes: int | None = None):
        self.device = torch.device(device if device is not None else torch.cuda.current_device())
        if nbytes is None:
            nbytes = default_workspace_bytes(torch.cuda.get_device_properties(self.device).multi_processor_count)
        self.nbytes = int(nbytes)
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)
        with torch.cuda.device(self.device):
            B.check(B.sk_workspace_init(ctypes.c_void_p(self.buf.data_ptr()), self.nbytes,
                                        _stream()), "sk_workspace_init")

    @property
    def ptr(self):
        return ctypes.c_void_p(self.buf.data_ptr())

    def status(self, clear: bool = True) -> int:
        out = ctypes.c_int(0)
        with torch.cuda.device(self.device):
            B.check(B.sk_get_status(self.ptr, self.nbytes, _stream(), int(clear), ctypes.byref(out)),
                    "sk_get_status")
        return out.value


_ws_lock = threading.Lock()
_ws_cache: dict = {}
_ws_retired: list = []


def default_workspace(device=None, min_bytes: int = 0) -> Workspace:
    """The workspace calls without an explicit one use: one per device and
    stream (the current stream of that device), so GEMMs running on
    different streams at the same time never share partial slots or flags.
    Calls on one stream are ordered by it and share its workspace.  A call
    that needs more (a group of more than 64 problems keeps its problem
    table there) replaces it with a larger one; make such a call once
    before capturing a CUDA graph, as the allocation cannot be captured."""
    dev = torch.device(device if device is not None else torch.cuda.current_device())
    if dev.index is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    key = (dev.index, torch.cuda.current_stream(dev).cuda_stream)
    with _ws_lock:
        ws = _ws_cache.get(key)
        if ws is None or ws.nbytes < min_bytes:
            if ws is not None:
                _ws_retired.append(ws)   # CUDA graphs captured earlier may still use it
            base = default_workspace_bytes(torch.cuda.get_device_properties(dev).multi_processor_count)
            ws = Workspace(dev, max(base, int(min_bytes)))
            _ws_cache[key] = ws
        return ws


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def gemm(A: torch.Tensor, Bm: torch.Tensor, out: torch.Tensor | None = None, *,
         alpha: float = 1.0, beta: float = 0.0, C_in: torch.Tensor | None = None,
         out_dtype=None, scale_a=None, scale_b=None, config=None,
         workspace: Workspace | None = None) -> torch.Tensor:
    """C = alpha * A @ B + beta * C_in on the current stream (Stream-K)."""
    if out is None:
        dt = out_dtype or (torch.float32 if A.dtype == torch.float32 else torch.bfloat16)
        out = torch.empty((A.shape[0], Bm.shape[1]), dtype=dt, device=A.device)
    ws = workspace or default_workspace(A.device)
    p = make_problem(A, Bm, out, C_in=C_in, alpha=alpha, beta=beta, scale_a=scale_a, scale_b=scale_b)
    cfg = _cfg(config)
    B.check(B.sk_gemm(ctypes.byref(p), ctypes.byref(cfg), ws.ptr, ws.nbytes, _stream()), "sk_gemm")
    return out


def grouped_gemm(As, Bs, outs=None, *, alpha: float = 1.0, beta: float = 0.0, C_ins=None,
                 out_dtype=None, config=None, workspace: Workspace | None = None):
    """One persistent launch over len(As) independent GEMMs."""
    n = len(As)
    if outs is None:
        outs = [torch.empty((a.shape[0], b.shape[1]),
                            dtype=out_dtype or (torch.float32 if a.dtype == torch.float32 else torch.bfloat16),
                            device=a.device) for a, b in zip(As, Bs)]
    arr = (B.sk_problem * n)()
    for i in range(n):
        arr[i] = make_problem(As[i], Bs[i], outs[i], C_in=None if C_ins is None else C_ins[i],
                              alpha=alpha, beta=beta)
    cfg = _cfg(config)
    if workspace is None:
        need = 0
        if n > 64:   # the problem table goes into the workspace
            nb = ctypes.c_size_t(0)
            with torch.cuda.device(As[0].device):
                B.check(B.sk_workspace_size(arr, n, ctypes.byref(cfg), ctypes.byref(nb)), "sk_workspace_size")
            need = nb.value
        ws = default_workspace(As[0].device, need)
    else:
        ws = workspace
    B.check(B.sk_gemm_grouped(arr, n, ctypes.byref(cfg), ws.ptr, ws.nbytes, _stream()), "sk_gemm_grouped")
    return outs


def gemm_backward(A: torch.Tensor, Bm: torch.Tensor, dC: torch.Tensor, *, need_dA: bool = True,
                  need_dB: bool = True, config=None, workspace: Workspace | None = None):
    """dA = dC @ B^T and dB = A^T @ dC, with dA/dB in A's/B's dtype and
    storage order, in one grouped Stream-K launch."""
    M, K = A.shape
    N = Bm.shape[1]
    dA = torch.empty_strided(A.shape, A.stride(), dtype=A.dtype, device=A.device) if need_dA else None
    dB = torch.empty_strided(Bm.shape, Bm.stride(), dtype=Bm.dtype, device=Bm.device) if need_dB else None
    c_layout, lddc = layout_of(dC, B.SK_ROW_MAJOR)
    if c_layout != B.SK_ROW_MAJOR:
        raise ValueError("dC must be row-major")
    fwd = B.sk_problem()
    fwd.m, fwd.n, fwd.k = M, N, K
    fwd.a_type, fwd.b_type, fwd.c_type = _DTYPES[A.dtype], _DTYPES[Bm.dtype], _DTYPES[dC.dtype]
    fwd.a_layout, fwd.lda = layout_of(A, B.SK_ROW_MAJOR)
    fwd.b_layout, fwd.ldb = layout_of(Bm, B.SK_COL_MAJOR)
    fwd.c_layout, fwd.ldc = B.SK_ROW_MAJOR, lddc
    fwd.A, fwd.B = A.data_ptr(), Bm.data_ptr()
    fwd.alpha, fwd.beta = 1.0, 0.0
    ldda = layout_of(dA, B.SK_ROW_MAJOR)[1] if dA is not None else 0
    lddb = layout_of(dB, B.SK_COL_MAJOR)[1] if dB is not None else 0
    cfg = _cfg(config)
    if workspace is None:
        # room for K-major copies of the operands the backward GEMMs would
        # read MN-major (the library transposes them there first)
        need = ctypes.c_size_t(0)
        B.check(B.sk_gemm_backward_workspace_size(ctypes.byref(fwd), int(need_dA), int(need_dB), ctypes.byref(cfg),
                                                  ctypes.byref(need)), "sk_gemm_backward_workspace_size")
        ws = default_workspace(A.device, need.value)
    else:
        ws = workspace
    B.check(B.sk_gemm_backward(ctypes.byref(fwd), _ptr(dC), lddc, _ptr(dA), ldda, _ptr(dB), lddb,
                               ctypes.byref(cfg), ws.ptr, ws.nbytes, _stream()), "sk_gemm_backward")
    return dA, dB


def transpose16(x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """x.T materialised row-major by the library's transpose kernel (16-bit
    element types; x row-major with unit column stride)."""
    if x.dim() != 2 or x.element_size() != 2 or x.stride(1) != 1:
        raise ValueError("expected a row-major 2-D tensor of a 16-bit type")
    rows, cols = x.shape
    if out is None:
        out = torch.empty((cols, rows), dtype=x.dtype, device=x.device)
    if out.shape != (cols, rows) or out.stride(1) != 1 or out.dtype != x.dtype:
        raise ValueError("out must be a row-major (cols x rows) tensor of x's type")
    B.check(B.sk_transpose16(_ptr(x), rows, cols, max(1, x.stride(0)), _ptr(out), max(1, out.stride(0)), _stream()),
            "sk_transpose16")
    return out


def quantize_e4m3(x: torch.Tensor):
    """Per-tensor FP8 quantisation on the GPU: returns (codes uint8, scale)."""
    x = x.contiguous()
    if x.dtype != torch.float32:
        raise ValueError("x must be float32")
    q = torch.empty(x.shape, dtype=torch.uint8, device=x.device)
    scale = torch.empty((), dtype=torch.float32, device=x.device)
    amax = torch.empty((), dtype=torch.float32, device=x.device)
    B.check(B.sk_quantize_e4m3(_ptr(x), x.numel(), _ptr(q), _ptr(scale), _ptr(amax), _stream()),
            "sk_quantize_e4m3")
    return q, scale


def plan(problems, config=None, num_sms: int = 0):
    """Resolve the plan of a call (no launch).  ``problems`` is an
    ``sk_problem`` or a list of them."""
    if isinstance(problems, B.sk_problem):
        problems = [problems]
    arr = (B.sk_problem * len(problems))(*problems)
    info = B.sk_plan_info()
    cfg = _cfg(config)
    B.check(B.sk_plan_query(arr, len(problems), ctypes.byref(cfg), num_sms, ctypes.byref(info)),
            "sk_plan_query")
    return info


def unit_items(problems, unit: int, config=None, num_sms: int = 0):
    if isinstance(problems, B.sk_problem):
        problems = [problems]
    arr = (B.sk_problem * len(problems))(*problems)
    cfg = _cfg(config)
    n = ctypes.c_int(0)
    B.check(B.sk_plan_unit_items(arr, len(problems), ctypes.byref(cfg), num_sms, unit, None, 0,
                                 ctypes.byref(n)), "sk_plan_unit_items")
    items = (B.sk_work_item * max(1, n.value))()
    B.check(B.sk_plan_unit_items(arr, len(problems), ctypes.byref(cfg), num_sms, unit, items,
                                 n.value, ctypes.byref(n)), "sk_plan_unit_items")
    return [items[i] for i in range(n.value)]


def shape_problem(M: int, N: int, K: int, dtype: str = "bf16", out: str | None = None,
                  a_layout: str = "row", b_layout: str = "col") -> B.sk_problem:
    """A pointer-free problem description for plan queries."""
    t = {"f32": B.SK_F32, "bf16": B.SK_BF16, "e4m3": B.SK_E4M3}[dtype]
    ct = {"f32": B.SK_F32, "bf16": B.SK_BF16}[out or ("f32" if dtype == "f32" else "bf16")]
    p = B.sk_problem()
    p.m, p.n, p.k = M, N, K
    p.a_type = p.b_type = t
    p.c_type = ct
    p.a_layout = B.SK_ROW_MAJOR if a_layout == "row" else B.SK_COL_MAJOR
    p.b_layout = B.SK_ROW_MAJOR if b_layout == "row" else B.SK_COL_MAJOR
    p.c_layout = B.SK_ROW_MAJOR
    # leading dimensions padded to 16 elements: legal TMA row pitches
    pad = lambda x: -(-max(1, x) // 16) * 16   # noqa: E731
    p.lda = pad(K if a_layout == "row" else M)
    p.ldb = pad(N if b_layout == "row" else K)
    p.ldc = max(1, N)
    p.A = p.B = p.C = 16   # non-null placeholders; plan queries never dereference
    p.alpha, p.beta = 1.0, 0.0
    return p


def trace_gemm(A: torch.Tensor, Bm: torch.Tensor, out: torch.Tensor | None = None, config=None, **kw):
    """Run one GEMM with per-CTA timeline tracing.  Returns (C, events)
    where events[cta] is a time-sorted list of (event name, item, t_ns)
    with t_ns relative to the earliest CTA start."""
    import dataclasses
    cfg = config or Config()
    sms = torch.cuda.get_device_properties(A.device).multi_processor_count
    buf = torch.zeros(sms * B.SK_TRACE_ENTRIES * 2, dtype=torch.int64, device=A.device)
    cfg = dataclasses.replace(cfg, trace=buf.data_ptr())
    C = gemm(A, Bm, out, config=cfg, **kw)
    torch.cuda.synchronize()
    raw = buf.view(sms, B.SK_TRACE_ENTRIES, 2).cpu()
    t0 = None
    per = []
    for c in range(sms):
        evs = []
        for e in range(B.SK_TRACE_ENTRIES):
            code, t = int(raw[c, e, 0]), int(raw[c, e, 1])
            if code == 0:
                continue
            evs.append((B.TRACE_EVENTS.get(code >> 32, "?"), code & 0xFFFFFFFF, t))
        evs.sort(key=lambda x: x[2])
        if evs:
            t0 = evs[0][2] if t0 is None else min(t0, evs[0][2])
        per.append(evs)
    per = [[(n, i, t - t0) for (n, i, t) in evs] for evs in per]
    return C, per


def coverage_counts(As, Bs, outs=None, config=None, **kw):
    """Run one GEMM (``As``, ``Bs`` tensors) or one grouped GEMM (lists) with
    the kernel's coverage counting on.  Returns (outputs, words, plan) with
    ``words`` the SK_COVERAGE words as a host int64 tensor: the first
    ``total_iters`` count the MAC-loop iterations, the rest the 32 x 32
    blocks of C each unit stored (layout in include/skgemm.h)."""
    import dataclasses
    cfg = config or Config()
    grouped = isinstance(As, (list, tuple))
    A_list, B_list = (list(As), list(Bs)) if grouped else ([As], [Bs])
    if outs is None:
        out_dtype = kw.pop("out_dtype", None)
        outs = [torch.empty((a.shape[0], b.shape[1]),
                            dtype=out_dtype or (torch.float32 if a.dtype == torch.float32 else torch.bfloat16),
                            device=a.device) for a, b in zip(A_list, B_list)]
    elif not grouped:
        outs = [outs]
    probs = [make_problem(a, b, c) for a, b, c in zip(A_list, B_list, outs)]
    info = plan(probs, cfg)
    buf = torch.zeros(max(1, info.coverage_words), dtype=torch.int32, device=A_list[0].device)
    cfg = dataclasses.replace(cfg, coverage=buf.data_ptr())
    if grouped:
        grouped_gemm(A_list, B_list, outs, config=cfg, **kw)
    else:
        gemm(A_list[0], B_list[0], outs[0], config=cfg, **kw)
    torch.cuda.synchronize()
    words = buf[:info.coverage_words].cpu().to(torch.int64) & 0xFFFFFFFF
    return (outs if grouped else outs[0]), words, info
