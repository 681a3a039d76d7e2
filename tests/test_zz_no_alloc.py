"""sk_gemm_static_ws: the GEMM entry point for callers that cannot allocate
device memory (their memory belongs to another allocator or pool, or they
have nowhere to keep a workspace).  It uses a fixed workspace array inside
the library instead of one passed by the caller.

Checked through the C ABI against the ordinary entry point (sk_gemm with a
caller workspace) on two calls in a row, within the normwise bound the other
GPU tests use.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_common import dev, sk, to_np

pytestmark = pytest.mark.gpu


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_static_ws_matches_sk_gemm_two_calls():
    m = sk()
    B = m.binding
    d = dev()
    ws = m.Workspace(d)
    cfg = B.sk_config()
    cfg.tile_n = 128
    cfg.mode = B.SK_MODE_SK          # every tile split: the workspace is exercised
    for call, (M, N, K) in enumerate([(1000, 1200, 3000), (384, 640, 8192)]):
        a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=300 + call)
        ad, bd = a.to(d), b.to(d)
        c_ref = torch.empty(M, N, dtype=torch.bfloat16, device=d)
        c_new = torch.full((M, N), float("nan"), dtype=torch.bfloat16, device=d)
        p_ref = m.make_problem(ad, bd, c_ref)
        p_new = m.make_problem(ad, bd, c_new)
        B.check(B.sk_gemm(ctypes.byref(p_ref), ctypes.byref(cfg), ws.ptr, ws.nbytes, _stream()), "sk_gemm")
        B.check(B.sk_gemm_static_ws(ctypes.byref(p_new), ctypes.byref(cfg), _stream()), "sk_gemm_static_ws")
        torch.cuda.synchronize()
        assert ws.status() == 0
        _, S = oracle.gemm(a, b)
        got, ref = to_np(c_new), to_np(c_ref)
        tol = oracle.bound(S, ref, "bf16")
        assert np.all(np.abs(got - ref) <= tol), f"call {call}"


@pytest.mark.parametrize("f32k", ["tf32x3", "ffma"])
def test_static_ws_fp32_bitwise(f32k):
    """FP32 (both kernels) through the fixed workspace: the same schedule
    and summation order as with a caller workspace, so the same bits."""
    m = sk()
    B = m.binding
    d = dev()
    ws = m.Workspace(d)
    cfg = m.Config(mode="sk", f32_kernel=f32k).to_c()
    a, b = workloads.gemm_inputs(384, 384, 2048, dtype="f32", seed=320)
    ad, bd = a.to(d), b.to(d)
    c_ref = torch.empty(384, 384, device=d)
    c_new = torch.full((384, 384), float("nan"), device=d)
    B.check(B.sk_gemm(ctypes.byref(m.make_problem(ad, bd, c_ref)), ctypes.byref(cfg), ws.ptr, ws.nbytes,
                      _stream()), "sk_gemm")
    B.check(B.sk_gemm_static_ws(ctypes.byref(m.make_problem(ad, bd, c_new)), ctypes.byref(cfg), _stream()),
            "sk_gemm_static_ws")
    torch.cuda.synchronize()
    assert ws.status() == 0
    assert torch.equal(c_new, c_ref)


def test_static_ws_rejects_oversized_plan():
    m = sk()
    B = m.binding
    d = dev()
    sms = torch.cuda.get_device_properties(d).multi_processor_count
    if sms <= 95:
        pytest.skip("128x256 tiles fit the fixed workspace on this GPU")
    a, b = workloads.gemm_inputs(256, 512, 1024, dtype="bf16", seed=310)
    c = torch.empty(256, 512, dtype=torch.bfloat16, device=d)
    p = m.make_problem(a.to(d), b.to(d), c)
    cfg = B.sk_config()
    cfg.tile_n = 256                  # 128 KB of partials per CTA on every SM: > 12 MiB
    assert B.sk_gemm_static_ws(ctypes.byref(p), ctypes.byref(cfg), _stream()) == B.SK_ERR_WORKSPACE_TOO_SMALL
