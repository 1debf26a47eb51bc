"""The FMA-pipe probe that gives the plain kernels' roofline peak: it runs,
counts its operations, and its sink holds the chains' finite results."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def semax():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_07659_gb300 as m
    return m


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_fma_probe_runs_and_counts(semax, prec):
    sink, flops = semax.fma_probe(prec, blocks=40, iters=64)
    torch.cuda.synchronize()
    assert flops == 2 * (4 if prec == "f64" else 8) * 64 * 256 * 40
    assert sink.numel() == 40 * 256 and bool(torch.isfinite(sink).all())
    # thread t's chains start at (t + q) c; after 64 steps of a -> a b_q + c_q they are positive
    assert bool((sink > 0).all())
