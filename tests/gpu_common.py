"""Helpers for the GPU parity tests: build/load the library, compare a GPU
result with the oracle element by element under the normwise bound."""
from __future__ import annotations

import numpy as np
import torch

import oracle


def sk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2407_00044_gb300 as m
    return m


def dev():
    return torch.device("cuda", torch.cuda.current_device())


def same_strides(t: torch.Tensor, device) -> torch.Tensor:
    """Copy to ``device`` keeping the storage order (row/column major)."""
    return torch.empty_strided(t.shape, t.stride(), dtype=t.dtype, device=device).copy_(t)


def to_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().float().cpu().numpy().astype(np.float64)


def assert_within_bound(got, A, B, *, alpha=1.0, beta=0.0, C0=None, out="f32", what=""):
    """|got - ref| <= 5e-5 * S (+ 5e-5 |beta C0|) (+ 2^-8 |ref| for BF16
    output), element by element, with ref and S from the FP64 oracle on the
    same (already rounded) inputs."""
    host = lambda x: x.cpu() if isinstance(x, torch.Tensor) else x   # noqa: E731
    ref, S = oracle.gemm(host(A), host(B), alpha=alpha, beta=beta,
                         C0=None if C0 is None else host(C0))
    g = to_np(got)
    bc0 = None if (C0 is None or beta == 0.0) else beta * oracle.to_f64(host(C0))
    tol = oracle.bound(S, ref, out, beta_c0=bc0)
    err = np.abs(g - ref)
    bad = ~(err <= tol)
    if bad.any():
        i, j = np.unravel_index(np.argmax(np.where(bad, err / np.maximum(tol, 1e-300), 0)), err.shape)
        raise AssertionError(f"{what}: {int(bad.sum())}/{bad.size} entries outside the bound; "
                             f"worst ({i},{j}) got {g[i, j]!r} ref {ref[i, j]!r} tol {tol[i, j]!r}")
    return float(np.max(err / np.maximum(S, 1e-300)))


def assert_sampled(C, A, B, *, out="bf16", tile_m=128, tile_n=256, n_rand=48, seed=0, what=""):
    """Check rows R x cols Q of a large product: the first and last tile rows
    and columns (the last one ragged when the size is not a tile multiple)
    plus random rows/cols, against the oracle on those rows/cols only."""
    M, N = C.shape
    g = np.random.default_rng(seed)
    rows = set(range(min(tile_m, M))) | set(range(max(0, (M - 1) // tile_m * tile_m), M))
    cols = set(range(min(tile_n, N))) | set(range(max(0, (N - 1) // tile_n * tile_n), N))
    rows |= set(g.integers(0, M, size=n_rand).tolist())
    cols |= set(g.integers(0, N, size=n_rand).tolist())
    r = torch.tensor(sorted(rows), device=C.device)
    q = torch.tensor(sorted(cols), device=C.device)
    a = A.index_select(0, r).cpu()
    b = B.index_select(1, q).cpu()
    got = C.index_select(0, r).index_select(1, q)
    return assert_within_bound(got, a, b, out=out, what=what)
