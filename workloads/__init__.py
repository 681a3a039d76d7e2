"""Seeded synthetic inputs and workload tables for the Stream-K GEMM.

This module is shared by the CUDA path's tests/benchmark and by the oracle's
tests.  It holds none of the GEMM's arithmetic: only random-number draws,
dtype casts done by library routines (torch), the shape tables of the
workloads, and the flop/byte accounting used to turn times into TFLOP/s and
GB/s (the accounting the paper's Results table uses: TFLOP/s = 2*M*N*K / t,
GB/s = (M*K + K*N + M*N) * bytes / t).

Every generator takes an explicit integer seed and draws from numpy's Philox
bit generator on the host, or from a seeded torch CUDA generator for the
large benchmark shapes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

# ---------------------------------------------------------------------------
# Workload tables (synthetic stand-ins; the paper measures no public dataset)
# ---------------------------------------------------------------------------

#: Plain FP32 Stream-K case: 128x128 tiles give 9 tiles, fewer than SMs.
FP32_SMALL = dict(M=384, N=384, K=2048, tile_m=128, tile_n=128)

#: BF16-input / FP32-accumulate / BF16-output shape sweep.  The first shape
#: is the paper's baseline problem (Results, Table 1: 3840x4096x4096).
BF16_SWEEP = [
    (3840, 4096, 4096),
    (1536, 1536, 8192),
    (8192, 8192, 8192),
    (2048, 7168, 1024),
    (128, 8192, 16384),
]

#: FP8 E4M3 per-tensor-scaled shapes.
FP8_SHAPES = [(8192, 8192, 8192), (4096, 14336, 4096)]

#: Autograd layer shape and the finite-difference shape.
AUTOGRAD_SHAPE = (8192, 11008, 4096)
FD_SHAPE = (64, 48, 80)

#: Shapes from the paper's Results section used as regression cases:
#: the irregular 1920x2000x2000 problem and the 480x512x512 problem that the
#: studied implementation got wrong.
PAPER_IRREGULAR = (1920, 2000, 2000)
PAPER_MEDIUM = (480, 512, 512)


def gemm_flops(M: int, N: int, K: int) -> int:
    """Algorithmic flop count of one GEMM: one multiply and one add per MAC."""
    return 2 * M * N * K


def gemm_bytes(M: int, N: int, K: int, a_bytes: float, b_bytes: float,
               c_bytes: float, read_c: bool = False) -> float:
    """Algorithmic bytes of one GEMM: read A and B once, write C once
    (and read C once more when beta != 0)."""
    b = M * K * a_bytes + K * N * b_bytes + M * N * c_bytes
    if read_c:
        b += M * N * c_bytes
    return b


# ---------------------------------------------------------------------------
# Host generators (numpy Philox)
# ---------------------------------------------------------------------------

def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def uniform(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> torch.Tensor:
    """float32 host tensor, i.i.d. uniform[lo, hi)."""
    a = _rng(seed).uniform(lo, hi, size=shape).astype(np.float32)
    return torch.from_numpy(a)


def normal(shape, seed: int) -> torch.Tensor:
    """float32 host tensor, i.i.d. N(0, 1)."""
    a = _rng(seed).standard_normal(size=shape).astype(np.float32)
    return torch.from_numpy(a)


def small_int(shape, seed: int, lo: int = -2, hi: int = 2) -> torch.Tensor:
    """float32 host tensor of integers drawn uniformly from [lo, hi]."""
    a = _rng(seed).integers(lo, hi + 1, size=shape).astype(np.float32)
    return torch.from_numpy(a)


def draw(shape, seed: int, dist: str) -> torch.Tensor:
    if dist == "uniform":
        return uniform(shape, seed)
    if dist == "normal":
        return normal(shape, seed)
    if dist == "int":
        return small_int(shape, seed)
    raise ValueError(f"unknown distribution {dist!r}")


def as_layout(x: torch.Tensor, layout: str) -> torch.Tensor:
    """Return the logical matrix ``x`` stored in 'row' or 'col' major order.

    A column-major R x C matrix is a contiguous C x R tensor viewed through
    ``.t()``; strides tell the binding which one it got.
    """
    if layout == "row":
        return x.contiguous()
    if layout == "col":
        return x.t().contiguous().t()
    raise ValueError(layout)


_TORCH_DTYPES = {
    "f32": torch.float32,
    "bf16": torch.bfloat16,
}


def gemm_inputs(M: int, N: int, K: int, *, dtype: str = "bf16",
                a_layout: str = "row", b_layout: str = "col",
                seed: int = 0, dist: str = "uniform"):
    """Seeded host operands A (M x K) and B (K x N) in the requested storage
    order, already rounded to ``dtype`` ('f32' or 'bf16') by torch's cast."""
    td = _TORCH_DTYPES[dtype]
    a = draw((M, K), 2 * seed + 0, dist).to(td)
    b = draw((K, N), 2 * seed + 1, dist).to(td)
    return as_layout(a, a_layout), as_layout(b, b_layout)


def grouped_shapes(count: int = 64, seed: int = 0,
                   m_lo: int = 64, m_hi: int = 4096,
                   nk_choices=(1024, 2048, 4096, 7168)):
    """Problem sizes of the grouped workload: M log-uniform in [m_lo, m_hi]
    (rounded to an integer), N and K each drawn from ``nk_choices``."""
    r = _rng(10_000 + seed)
    out = []
    for _ in range(count):
        m = int(round(math.exp(r.uniform(math.log(m_lo), math.log(m_hi)))))
        n = int(r.choice(nk_choices))
        k = int(r.choice(nk_choices))
        out.append((m, n, k))
    return out


# ---------------------------------------------------------------------------
# Device generators (seeded torch CUDA generator) for the large shapes
# ---------------------------------------------------------------------------

def device_uniform(shape, seed: int, device, dtype=torch.bfloat16) -> torch.Tensor:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    x = torch.rand(shape, generator=g, device=device, dtype=torch.float32)
    return (x.mul_(2.0).sub_(1.0)).to(dtype)


def device_normal(shape, seed: int, device, dtype=torch.float32) -> torch.Tensor:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return torch.randn(shape, generator=g, device=device, dtype=torch.float32).to(dtype)


@dataclass
class Problem:
    """One GEMM of a workload: sizes plus storage orders."""
    M: int
    N: int
    K: int
    a_layout: str = "row"
    b_layout: str = "col"
