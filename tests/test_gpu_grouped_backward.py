"""GPU parity of the grouped launch (Stream-K ranges crossing problem
boundaries) and of the backward pass (transposed-operand kernels), against
the FP64 oracle; autograd against the oracle gradient."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_common import assert_within_bound, dev, sk, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    return sk()


SHAPES = [(64, 1024, 1024), (300, 256, 2048), (1000, 512, 128), (17, 2048, 4096),
          (512, 1024, 1024), (128, 128, 8), (700, 300, 520), (256, 7168, 256), (1, 8, 64)]


@pytest.mark.parametrize("mode", ["sk", "hybrid2", "dp"])
def test_grouped_int_exact(m, mode):
    d = dev()
    As, Bs, refs = [], [], []
    for i, (M, N, K) in enumerate(SHAPES):
        a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=20 + i, dist="int")
        As.append(a.to(d))
        Bs.append(b.to(d))
        refs.append(oracle.gemm(a, b)[0])
    outs = m.grouped_gemm(As, Bs, out_dtype=torch.float32, config=m.Config(mode=mode))
    assert m.default_workspace(d).status() == 0
    for i, (o, r) in enumerate(zip(outs, refs)):
        assert np.array_equal(to_np(o), r), (mode, SHAPES[i])


@pytest.mark.parametrize("tile_m", [128, 256])
def test_grouped_pair_tiles_exact(m, tile_m):
    """Grouped launch whose problems all allow the CTA-pair kernel."""
    d = dev()
    shapes = [(256, 1024, 1024), (300, 512, 2048), (1024, 768, 128), (512, 2048, 64), (777, 256, 4096)]
    As, Bs, refs = [], [], []
    for i, (M, N, K) in enumerate(shapes):
        a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=80 + i, dist="int")
        As.append(a.to(d))
        Bs.append(b.to(d))
        refs.append(oracle.gemm(a, b)[0])
    for mode in ("sk", "hybrid2", "dp"):
        outs = m.grouped_gemm(As, Bs, out_dtype=torch.float32, config=m.Config(mode=mode, tile_m=tile_m))
        assert m.default_workspace(d).status() == 0
        for i, (o, r) in enumerate(zip(outs, refs)):
            assert np.array_equal(to_np(o), r), (mode, tile_m, shapes[i])


def test_grouped_bound_and_graph(m):
    d = dev()
    shapes = workloads.grouped_shapes(count=12, seed=0, m_hi=1024)
    As, Bs, hosts = [], [], []
    for i, (M, N, K) in enumerate(shapes):
        a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=40 + i)
        As.append(a.to(d))
        Bs.append(b.to(d))
        hosts.append((a, b))
    outs = m.grouped_gemm(As, Bs)
    for o, (a, b) in zip(outs, hosts):
        assert_within_bound(o, a, b, out="bf16", what="grouped")
    # graph capture and replay give identical bits
    s = torch.cuda.Stream()
    outs2 = [torch.empty_like(o) for o in outs]
    with torch.cuda.stream(s):
        m.grouped_gemm(As, Bs, outs2)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            m.grouped_gemm(As, Bs, outs2)
    for o in outs2:
        o.zero_()
    g.replay()
    torch.cuda.synchronize()
    for o, o2 in zip(outs, outs2):
        assert torch.equal(o, o2)


def test_backward_fd_shape(m):
    """(64, 48, 80): GPU dA, dB vs the oracle gradient (which the CPU tests
    pin with FP64 finite differences)."""
    M, N, K = workloads.FD_SHAPE
    d = dev()
    a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=50)
    g = workloads.normal((M, N), seed=51).to(torch.bfloat16)
    dA, dB = m.gemm_backward(a.to(d), b.to(d), g.to(d))
    assert m.default_workspace(d).status() == 0
    # dA = G B^T ; dB = A^T G, each an ordinary product of the same values
    assert_within_bound(dA, g, b.t(), out="bf16", what="dA")
    assert_within_bound(dB, a.t(), g, out="bf16", what="dB")
    assert dA.stride() == a.stride() and dB.stride() == b.stride()


@pytest.mark.parametrize("tile_m", [128, 256])
@pytest.mark.parametrize("al,bl", [("row", "col"), ("row", "row"), ("col", "col"), ("col", "row")])
def test_backward_layouts_exact(m, al, bl, tile_m):
    M, N, K = 264, 392, 520
    d = dev()
    a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", a_layout=al, b_layout=bl, seed=52, dist="int")
    g = workloads.small_int((M, N), seed=53).to(torch.bfloat16)
    from gpu_common import same_strides
    dA, dB = m.gemm_backward(same_strides(a, d), same_strides(b, d), g.to(d), config=m.Config(tile_m=tile_m))
    rA, _ = oracle.gemm(g, b.t())
    rB, _ = oracle.gemm(a.t(), g)
    # exact integers that fit BF16 output: |values| <= 4 * 392 < 2^8? not in
    # general, so compare within the BF16 rounding of the exact result
    assert np.all(np.abs(to_np(dA) - rA) <= 2 ** -8 * np.abs(rA))
    assert np.all(np.abs(to_np(dB) - rB) <= 2 ** -8 * np.abs(rB))


def test_backward_from_another_thread(m):
    """The autograd engine calls backward from its own thread: the library
    must work from a thread other than the one that first used it."""
    import threading
    M, N, K = 128, 256, 192
    d = dev()
    a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=56)
    g = workloads.normal((M, N), seed=57).to(torch.bfloat16)
    res = {}

    def work():
        try:
            torch.cuda.set_device(d)
            res["out"] = m.gemm_backward(a.to(d), b.to(d), g.to(d))
            torch.cuda.synchronize()
        except Exception as e:   # surfaced below
            res["err"] = e

    t = threading.Thread(target=work)
    t.start()
    t.join()
    assert "err" not in res, res.get("err")
    dA, dB = res["out"]
    assert_within_bound(dA, g, b.t(), out="bf16", what="dA (thread)")
    assert_within_bound(dB, a.t(), g, out="bf16", what="dB (thread)")


def test_autograd_matches_oracle(m):
    M, N, K = 256, 384, 512
    d = dev()
    a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=54)
    g = workloads.normal((M, N), seed=55).to(torch.bfloat16)
    A = a.to(d).requires_grad_(True)
    Bm = b.to(d).requires_grad_(True)
    C = m.sk_matmul(A, Bm)
    C.backward(g.to(d))
    assert_within_bound(C, a, b, out="bf16", what="forward")
    assert_within_bound(A.grad, g, b.t(), out="bf16", what="dA")
    assert_within_bound(Bm.grad, a.t(), g, out="bf16", what="dB")


def _many_problems(count, seed, dtype="bf16"):
    shapes = workloads.grouped_shapes(count=count, seed=seed, m_lo=16, m_hi=512,
                                      nk_choices=(64, 128, 256, 512, 1024))
    d = dev()
    As, Bs, refs = [], [], []
    for i, (M, N, K) in enumerate(shapes):
        a, b = workloads.gemm_inputs(M, N, K, dtype=dtype, seed=1000 + 7 * seed + i, dist="int")
        As.append(a.to(d))
        Bs.append(b.to(d))
        refs.append(oracle.gemm(a, b)[0])
    return shapes, As, Bs, refs


def test_grouped_256_problems_graph(m):
    """256 uneven problems in ONE persistent launch: more than the kernel's
    parameter block carries, so the problem table (tensor maps included)
    goes to the workspace, written by copy kernels on the stream.  Captured
    in a CUDA graph and replayed; small-integer inputs make every result
    exact, so each problem is compared with the oracle in full."""
    d = dev()
    shapes, As, Bs, refs = _many_problems(256, seed=1)
    outs = [torch.empty(a.shape[0], b.shape[1], dtype=torch.float32, device=d) for a, b in zip(As, Bs)]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        m.grouped_gemm(As, Bs, outs)      # first call outside the capture (sizes s's workspace)
        torch.cuda.synchronize()
        for i, (o, r) in enumerate(zip(outs, refs)):
            assert np.array_equal(to_np(o), r), ("direct", i, shapes[i])
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            m.grouped_gemm(As, Bs, outs)
    for o in outs:
        o.fill_(float("nan"))
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        assert m.default_workspace(d).status() == 0
    for i, (o, r) in enumerate(zip(outs, refs)):
        assert np.array_equal(to_np(o), r), ("graph", i, shapes[i])


@pytest.mark.parametrize("tile_m,mode", [(128, "sk"), (256, "hybrid2"), (256, "dp")])
def test_grouped_many_problems_tiles_modes(m, tile_m, mode):
    """100 problems (table in the workspace) on both unit shapes and modes,
    and the workspace-size contract: one byte short is refused."""
    d = dev()
    shapes, As, Bs, refs = _many_problems(100, seed=2)
    cfg = m.Config(mode=mode, tile_m=tile_m)
    outs = m.grouped_gemm(As, Bs, out_dtype=torch.float32, config=cfg)
    assert m.default_workspace(d).status() == 0
    for i, (o, r) in enumerate(zip(outs, refs)):
        assert np.array_equal(to_np(o), r), (tile_m, mode, i, shapes[i])
    B = m.binding
    arr = (B.sk_problem * len(As))(*[m.make_problem(a, b, o) for a, b, o in zip(As, Bs, outs)])
    import ctypes
    need = ctypes.c_size_t(0)
    c = cfg.to_c()
    B.check(B.sk_workspace_size(arr, len(As), ctypes.byref(c), ctypes.byref(need)))
    small = m.Workspace(d, need.value - 256)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert B.sk_gemm_grouped(arr, len(As), ctypes.byref(c), small.ptr, small.nbytes, st) == \
        B.SK_ERR_WORKSPACE_TOO_SMALL


@pytest.mark.parametrize("f32k", ["ffma", "tf32x3"])
def test_grouped_many_problems_fp32(m, f32k):
    """FP32 groups beyond the parameter block, on both FP32 kernels."""
    d = dev()
    shapes, As, Bs, refs = _many_problems(80, seed=3, dtype="f32")
    outs = m.grouped_gemm(As, Bs, config=m.Config(mode="hybrid2", f32_kernel=f32k))
    assert m.default_workspace(d).status() == 0
    for i, (o, r) in enumerate(zip(outs, refs)):
        assert np.array_equal(to_np(o), r), (f32k, i, shapes[i])


def _backward_ws(m, a, b, d, copies):
    """A workspace with (copies=True) or without room for the K-major copies
    sk_gemm_backward makes of MN-major operands: the copies end the size the
    library asks for, so 256 bytes less holds the GEMMs' own bytes but not
    the copies."""
    import ctypes
    B = m.binding
    fwd = m.make_problem(a, b, torch.empty(a.shape[0], b.shape[1], dtype=torch.bfloat16, device=d))
    cfg = m.Config().to_c()
    n = ctypes.c_size_t(0)
    B.check(B.sk_gemm_backward_workspace_size(ctypes.byref(fwd), 1, 1, ctypes.byref(cfg), ctypes.byref(n)))
    return m.Workspace(d, n.value if copies else n.value - 256)


@pytest.mark.parametrize("al,bl", [("row", "col"), ("row", "row"), ("col", "col"), ("col", "row")])
def test_backward_copies_equal_in_place(m, al, bl):
    """The backward GEMMs on K-major copies of their MN-major operands (made
    by the library's transpose kernel in the workspace) give the same bits
    as the GEMMs reading the operands in place; ragged extents (M = 300 with
    a padded leading dimension) take the transpose's element-by-element
    edge path."""
    M, N, K = 300, 392, 1000
    d = dev()
    a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=58)
    g = workloads.normal((M, N), seed=59).to(torch.bfloat16).to(d)
    # A col-major: storage K x M with a leading dimension padded to 304
    A = (torch.empty_strided((M, K), (1, 304), dtype=torch.bfloat16, device=d).copy_(a) if al == "col"
         else a.to(d))
    Bm = (torch.empty_strided((K, N), (1, K), dtype=torch.bfloat16, device=d).copy_(b) if bl == "col"
          else b.contiguous().to(d))
    w_copy, w_plain = _backward_ws(m, A, Bm, d, True), _backward_ws(m, A, Bm, d, False)
    assert w_copy.nbytes > w_plain.nbytes
    dA1, dB1 = m.gemm_backward(A, Bm, g, workspace=w_copy)
    dA2, dB2 = m.gemm_backward(A, Bm, g, workspace=w_plain)
    assert w_copy.status() == 0 and w_plain.status() == 0
    assert torch.equal(dA1, dA2) and torch.equal(dB1, dB2)
    assert_within_bound(dA1, g.cpu(), b.t(), out="bf16", what="dA (copies)")
    assert_within_bound(dB1, a.t(), g.cpu(), out="bf16", what="dB (copies)")


@pytest.mark.parametrize("shape,ld_pad", [((64, 64), 0), ((4096, 11008), 0), ((300, 1000), 8), ((1, 8), 0),
                                          ((7, 13), 3), ((130, 72), 0), ((8192, 8), 0)])
def test_transpose16_equals_torch(m, shape, ld_pad):
    """The backward's transpose kernel: bit-exact against torch's transpose,
    aligned (16-byte vector path) and ragged or odd-pitch (element path)."""
    d = dev()
    R, C = shape
    base = torch.arange(R * (C + ld_pad), device=d, dtype=torch.int32).to(torch.int16).view(torch.bfloat16)
    x = base.view(R, C + ld_pad)[:, :C]
    y = m.transpose16(x)
    torch.cuda.synchronize()
    assert torch.equal(y.view(torch.int16), x.t().contiguous().view(torch.int16))


def test_backward_with_wide_tile_config(m):
    """An explicit 256 x 512 tile (single-problem launches only): the
    backward runs its two GEMMs as single launches."""
    M, N, K = 512, 1024, 768
    d = dev()
    a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=60)
    g = workloads.normal((M, N), seed=61).to(torch.bfloat16)
    dA, dB = m.gemm_backward(a.to(d), b.to(d), g.to(d), config=m.Config(tile_m=256, tile_n=512))
    assert m.default_workspace(d).status() == 0
    assert_within_bound(dA, g, b.t(), out="bf16", what="dA (256x512)")
    assert_within_bound(dB, a.t(), g, out="bf16", what="dB (256x512)")
