"""sk_gemm_static_ws: the GEMM entry point for callers that cannot allocate
device memory (their memory belongs to another allocator or pool, or they
have nowhere to keep a workspace).  It uses a fixed workspace array inside
the library instead of one passed by the caller.

Checked through the C ABI against the ordinary entry point (sk_gemm with a
caller workspace) on two calls in a row: both run the same plan and add the
partials in the same order, so the results must agree bit for bit; each is
also checked against the FP64 oracle within the normwise bound the other GPU
tests use, and the fixed array's status word is read back after every call.
This file is collected last on purpose.
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


def _static_status(B, clear=True) -> int:
    out = ctypes.c_int(-1)
    B.check(B.sk_static_ws_status(_stream(), int(clear), ctypes.byref(out)), "sk_static_ws_status")
    return out.value


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
        assert _static_status(B) == B.SK_OK, f"call {call}"
        # same plan, same summation order: the same bits
        assert torch.equal(c_new.view(torch.int16), c_ref.view(torch.int16)), f"call {call}"
        ref, S = oracle.gemm(a, b)
        got = to_np(c_new)
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
    assert _static_status(B) == B.SK_OK
    assert torch.equal(c_new, c_ref)


def test_static_ws_timeout_is_reported_then_cleared():
    """A bounded fixup wait that expires is recorded in the fixed array's
    status word and stays there across a later call until it is read and
    cleared; the next call then computes the right result.  (The wait is made
    to expire by the test-only flag that stops peers from raising their
    flags, with a 50 ms limit: no fault, no hang.)"""
    m = sk()
    B = m.binding
    d = dev()
    a, b = workloads.gemm_inputs(512, 512, 4096, dtype="bf16", seed=330)
    ad, bd = a.to(d), b.to(d)
    c = torch.empty(512, 512, dtype=torch.bfloat16, device=d)
    p = m.make_problem(ad, bd, c)
    assert _static_status(B) == B.SK_OK
    bad = m.Config(mode="sk", tile_m=128, tile_n=128, timeout_ns=50_000_000, debug_flags=1).to_c()
    B.check(B.sk_gemm_static_ws(ctypes.byref(p), ctypes.byref(bad), _stream()), "sk_gemm_static_ws")
    good = m.Config(mode="sk", tile_m=128, tile_n=128).to_c()
    # a later, healthy call does not wipe the record
    B.check(B.sk_gemm_static_ws(ctypes.byref(p), ctypes.byref(good), _stream()), "sk_gemm_static_ws")
    assert _static_status(B, clear=False) == B.SK_ERR_TIMEOUT
    assert _static_status(B, clear=True) == B.SK_ERR_TIMEOUT
    assert _static_status(B) == B.SK_OK
    B.check(B.sk_gemm_static_ws(ctypes.byref(p), ctypes.byref(good), _stream()), "sk_gemm_static_ws")
    assert _static_status(B) == B.SK_OK
    ref, S = oracle.gemm(a, b)
    assert np.all(np.abs(to_np(c) - ref) <= oracle.bound(S, ref, "bf16"))


def test_static_ws_size_limits():
    """Plans whose workspace exceeds the fixed 12 MiB are refused before any
    launch: 128x256 tiles on every SM, and the last-arriver fixup (two
    partial slots per CTA) on more than 95 CTAs of 128x128; 95 CTAs fit."""
    m = sk()
    B = m.binding
    d = dev()
    sms = torch.cuda.get_device_properties(d).multi_processor_count
    if sms <= 95:
        pytest.skip("every plan fits the fixed workspace on this GPU")
    a, b = workloads.gemm_inputs(256, 512, 1024, dtype="bf16", seed=310)
    ad, bd = a.to(d), b.to(d)
    c = torch.empty(256, 512, dtype=torch.bfloat16, device=d)
    p = m.make_problem(ad, bd, c)
    # 128x256 tiles, Stream-K on every SM with the owner fixup: 128 KB of
    # partials per CTA, > 12 MiB
    cfg = m.Config(mode="sk", tile_m=128, tile_n=256, num_ctas=sms).to_c()
    assert B.sk_gemm_static_ws(ctypes.byref(p), ctypes.byref(cfg), _stream()) == B.SK_ERR_WORKSPACE_TOO_SMALL
    la = m.Config(mode="sk", tile_m=128, tile_n=128, fixup="last_arriver").to_c()
    assert B.sk_gemm_static_ws(ctypes.byref(p), ctypes.byref(la), _stream()) == B.SK_ERR_WORKSPACE_TOO_SMALL
    la.num_ctas = 95
    c_ref = torch.empty_like(c)
    ws = m.Workspace(d)
    B.check(B.sk_gemm_static_ws(ctypes.byref(p), ctypes.byref(la), _stream()), "sk_gemm_static_ws")
    B.check(B.sk_gemm(ctypes.byref(m.make_problem(ad, bd, c_ref)), ctypes.byref(la), ws.ptr, ws.nbytes,
                      _stream()), "sk_gemm")
    torch.cuda.synchronize()
    assert _static_status(B) == B.SK_OK
    assert torch.equal(c.view(torch.int16), c_ref.view(torch.int16))
