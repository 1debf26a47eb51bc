"""The bounded staging waits of the tensor-core kernels report a timeout
through a status word (SEMAX_ETIMEOUT), without a GPU fault.

The waits give up only when a TMA bulk copy never completes, which no input
can cause.  To drive that path on ordinary inputs the poll limit of each
element's first wait is set to zero (semax_set_wait_polls): every CTA then
gives up at its first element, reports, writes NaN over its outputs, and
drains its copies in flight with the second wait, which keeps the default
limit, so no copy is outstanding when it exits.  The tests restore the
default limit before they return.
"""
import numpy as np
import pytest
import torch

import sem_inputs as si

pytestmark = pytest.mark.gpu

ETIMEOUT = -6


@pytest.fixture(scope="module")
def semax():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_07659_gb300 as m
    return m


@pytest.fixture
def zero_polls(semax):
    semax.set_wait_polls(0)
    try:
        yield
    finally:
        semax.set_wait_polls(-1)


def _mesh(N, E, seed):
    m = si.make_mesh(np.random.default_rng(seed), E, N)
    return m.u.cuda(), m.G.cuda(), m.D.cuda()


@pytest.mark.parametrize("N,E", [(7, 37), (7, 1000), (15, 5), (15, 400)])
def test_status_reports_timeout(semax, N, E):
    u, G, D = _mesh(N, E, 900 + N + E)
    ref = semax.sem_ax_f64tc(u, G, D)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    semax.set_wait_polls(0)
    try:
        w = semax.sem_ax_f64tc(u, G, D, status=status)
        torch.cuda.synchronize()
    finally:
        semax.set_wait_polls(-1)
    assert int(status.item()) == ETIMEOUT
    assert bool(torch.isnan(w).all())
    # the default limit again: no report, the result of the plain call bit for bit
    status.zero_()
    w = semax.sem_ax_f64tc(u, G, D, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.equal(w, ref)


@pytest.mark.parametrize("N,E", [(7, 64), (15, 9)])
def test_prepared_status_reports_timeout(semax, N, E, zero_polls):
    u, G, D = _mesh(N, E, 950 + N)
    gp = semax.f64tc_prepare(G)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    w = semax.sem_ax_f64tc_prepared(u, gp, D, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == ETIMEOUT
    assert bool(torch.isnan(w).all())


def test_other_orders_never_write_status(semax, zero_polls):
    """Orders without a tensor-core kernel run the double-float tile: no waits."""
    u, G, D = _mesh(5, 20, 960)
    status = torch.full((1,), 123, dtype=torch.int32, device="cuda")
    w = semax.sem_ax_f64tc(u, G, D, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 123
    assert bool(torch.isfinite(w).all())


def test_plan_status(semax):
    u7, G7, D7 = _mesh(7, 50, 970)
    u3, G3, D3 = _mesh(3, 40, 971)
    w7, w3 = torch.empty_like(u7), torch.empty_like(u3)
    semax.set_wait_polls(0)
    try:   # the limit is captured into the plan's graph at create
        plan = semax.Plan([(7, u7, G7, D7, w7), (3, u3, G3, D3, w3)], f64tc=True)
    finally:
        semax.set_wait_polls(-1)
    plan()
    assert plan.status() == ETIMEOUT
    assert plan.status() == 0                         # cleared by the read
    assert bool(torch.isnan(w7).all()) and bool(torch.isfinite(w3).all())
    plan.close()
    plan = semax.Plan([(7, u7, G7, D7, w7), (3, u3, G3, D3, w3)], f64tc=True)
    plan()
    assert plan.status() == 0
    assert torch.equal(w7, semax.sem_ax_f64tc(u7, G7, D7))
    plan.close()


def test_pcg_returns_timeout(semax, zero_polls):
    bm = si.box_mesh(2, 2, 2, 7, si.rng_for(5))
    G, B, D = si.box_operator_data(bm, device="cuda")
    gs = semax.GatherScatter(bm.l2g, bm.nglobal, bm.boundary)
    b = torch.ones_like(B)
    gs(b, mask=True)
    pcg = semax.PCG(G, D, gs, f64tc=True)
    x = torch.zeros_like(b)
    with pytest.raises(semax.SemaxError) as ex:
        pcg.solve(b, x, max_iter=20, rtol=1e-8)
    assert ex.value.status == ETIMEOUT
    pcg.close()
    gs.close()
