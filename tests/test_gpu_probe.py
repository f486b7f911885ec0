"""The measurement probes do exactly the work they state: the reduction
probe's adds (its timing is the denominator of the backward's
atomic-throughput fraction) and the FMA probe's chains (the denominator of
the compositing kernels' ALU fraction)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_06644_gb300 import build
    build.build()
    from paper_2510_06644_gb300 import gs
    return gs


@pytest.mark.parametrize("n_dst,n_threads,per", [(1000, 5000, 3), (4096, 4096, 8), (7, 1000, 2)])
def test_probe_adds_exactly(G, n_dst, n_threads, per):
    dst = torch.zeros(n_dst, dtype=torch.float32, device="cuda")
    G.gs_probe_red_f32(dst, n_threads, per)
    torch.cuda.synchronize()
    want = torch.zeros(n_dst, dtype=torch.float64)
    idx = torch.arange(n_threads) % n_dst
    want.index_add_(0, idx, torch.full((n_threads,), float(per), dtype=torch.float64))
    assert torch.equal(dst.cpu().double(), want)


@pytest.mark.parametrize("n_threads,iters", [(1, 1), (300, 7), (4096, 1000)])
def test_fma_probe_runs_every_chain(G, n_threads, iters):
    out = torch.full((n_threads,), -1.0, dtype=torch.float32, device="cuda")
    G.gs_probe_fma_f32(out, iters)
    torch.cuda.synchronize()
    assert torch.all(out.cpu() == float(28 + 8 * iters))
