"""The Ax entry points neither synchronise with the host nor allocate device
memory: each one captures into a CUDA graph (a call that synchronised or
allocated would fail the capture), and replaying the graph reproduces the
eager call's result bit for bit."""
import numpy as np
import pytest
import torch

import sem_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def semax():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_07659_gb300 as m
    return m


def _captured_equals_eager(fn, like):
    eager = fn(torch.empty_like(like))
    torch.cuda.synchronize()
    w = torch.empty_like(like)
    fn(w)                                    # warm-up outside the capture (lazy attribute setup)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        fn(w)
    w.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    return torch.equal(w, eager)


def test_entry_points_capture_into_a_cuda_graph(semax):
    rng = np.random.default_rng(97)
    m7 = si.make_mesh(rng, 9, 7, device="cuda")
    m15 = si.make_mesh(rng, 3, 15, device="cuda")
    gp7, gp15 = semax.f64tc_prepare(m7.G), semax.f64tc_prepare(m15.G)
    u32, G32, D32 = m15.u.float(), m15.G.float(), m15.D.float()
    u7, G7, D7 = m7.u.float(), m7.G.float(), m7.D.float()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    cases = {
        "sem_ax": (lambda w: semax.sem_ax(m7.u, m7.G, m7.D, w), m7.u),
        "sem_ax_f64x": (lambda w: semax.sem_ax_f64x(m7.u, m7.G, m7.D, w), m7.u),
        "sem_ax_f64tc N=7": (lambda w: semax.sem_ax_f64tc(m7.u, m7.G, m7.D, w), m7.u),
        "sem_ax_f64tc N=15": (lambda w: semax.sem_ax_f64tc(m15.u, m15.G, m15.D, w), m15.u),
        "sem_ax_f64tc_prepared N=7": (lambda w: semax.sem_ax_f64tc_prepared(m7.u, gp7, m7.D, w), m7.u),
        "sem_ax_f64tc_prepared N=15": (lambda w: semax.sem_ax_f64tc_prepared(m15.u, gp15, m15.D, w), m15.u),
        "sem_ax_f32": (lambda w: semax.sem_ax_f32(u32, G32, D32, w), u32),
        "sem_ax_bf16x3": (lambda w: semax.sem_ax_bf16x3(u32, G32, D32, w, terms=6), u32),
        "sem_ax_f16x3 N=15": (lambda w: semax.sem_ax_f16x3(u32, G32, D32, w), u32),
        "sem_ax_f16x3 N=7": (lambda w: semax.sem_ax_f16x3(u7, G7, D7, w), u7),
        "sem_ax_f64tc_status N=7": (lambda w: semax.sem_ax_f64tc(m7.u, m7.G, m7.D, w, status=st), m7.u),
        "sem_ax_f64tc_prepared_status N=15": (lambda w: semax.sem_ax_f64tc_prepared(m15.u, gp15, m15.D, w, status=st),
                                              m15.u),
    }
    for name, (fn, like) in cases.items():
        assert _captured_equals_eager(fn, like), name
    assert int(st.item()) == 0


def test_batched_and_reduce_capture_with_preallocated_workspaces(semax):
    rng = np.random.default_rng(98)
    meshes = [si.make_mesh(rng, E, N, device="cuda") for N, E in [(3, 11), (7, 4), (15, 2)]]
    ws = [torch.empty_like(m.u) for m in meshes]
    groups = [(m.N, m.u, m.G, m.D, w) for m, w in zip(meshes, ws)]
    import ctypes
    import paper_1503_07659_gb300._lib as L
    arr, ng = semax._groups(groups)
    size = ctypes.c_size_t(0)
    L.check(L.lib().sem_ax_batched_workspace_size(arr, ng, ctypes.byref(size)), "workspace size")
    work = torch.empty(size.value, dtype=torch.uint8, device="cuda")
    semax.sem_ax_batched(groups, workspace=work)
    torch.cuda.synchronize()
    eager = [w.clone() for w in ws]
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        semax.sem_ax_batched(groups, workspace=work)
        semax.reduce(ws[1], eager[1], out=out)
    for w in ws:
        w.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(ws, eager))
    assert out[0].item() == 0.0 and out[1].item() == float(eager[1].abs().max())
