"""HostGemmPipeline: GEMMs on pinned host operands with overlapped copies
give exactly what the device path gives, run after run."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from gpu_common import dev, sk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    return sk()


def test_host_pipeline_matches_oracle_over_runs(m):
    shapes = [(264, 392, 520), (1024, 768, 256), (130, 72, 8)]
    host, refs = [], []
    for i, (M, N, K) in enumerate(shapes):
        a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=140 + i, dist="int")
        ha = torch.empty(a.shape, dtype=a.dtype, pin_memory=True).copy_(a)
        hb = torch.empty_strided(b.shape, b.stride(), dtype=b.dtype, pin_memory=True).copy_(b)
        hc = torch.empty((M, N), dtype=torch.float32, pin_memory=True)
        host.append((ha, hb, hc))
        refs.append(oracle.gemm(a, b)[0])
    pipe = m.HostGemmPipeline(host, device=dev())
    for run in range(3):
        for _, _, hc in host:
            hc.fill_(float("nan"))
        pipe.run()
        torch.cuda.synchronize()
        for (_, _, hc), r, s in zip(host, refs, shapes):
            assert np.array_equal(hc.numpy().astype(np.float64), r), (run, s)
    assert m.default_workspace(dev()).status() == 0
    assert pipe.bytes_in == sum((M * K + K * N) * 2 for M, N, K in shapes)
    assert pipe.bytes_out == sum(M * N * 4 for M, N, K in shapes)


def test_host_pipeline_overlapped_runs(m):
    """Runs enqueued back to back without joining (consecutive steps
    overlap on the three streams) produce the same C; join() then orders
    the current stream after all of them."""
    shapes = [(512, 1024, 768), (264, 392, 520), (1100, 300, 1024)]
    host, refs = [], []
    for i, (M, N, K) in enumerate(shapes):
        a, b = workloads.gemm_inputs(M, N, K, dtype="bf16", seed=150 + i, dist="int")
        ha = torch.empty(a.shape, dtype=a.dtype, pin_memory=True).copy_(a)
        hb = torch.empty_strided(b.shape, b.stride(), dtype=b.dtype, pin_memory=True).copy_(b)
        hc = torch.full((M, N), float("nan"), dtype=torch.float32, pin_memory=True)
        host.append((ha, hb, hc))
        refs.append(oracle.gemm(a, b)[0])
    pipe = m.HostGemmPipeline(host, device=dev())
    for _ in range(4):
        pipe.run(join=False)
    pipe.join()
    done = torch.cuda.Event()
    done.record()
    done.synchronize()
    for (_, _, hc), r, s in zip(host, refs, shapes):
        assert np.array_equal(hc.numpy().astype(np.float64), r), s
    assert pipe.ws.status() == 0
