"""GPU parity of the solver around Ax (gather-scatter, operator diagonal,
graph-captured Jacobi-PCG) against the NumPy solver oracle on conforming box
meshes."""
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


@pytest.fixture(scope="module")
def solver_oracle():
    from oracle import solver
    return solver


def _setup(shape, N, seed):
    m = si.box_mesh(*shape, N, np.random.default_rng(seed))
    G, B, D = si.box_operator_data(m)
    x = m.coords
    ue = np.sin(np.pi * x[..., 0]) * np.sin(np.pi * x[..., 1]) * np.sin(np.pi * x[..., 2])
    mask = (~m.boundary[m.l2g]).astype(np.float64).reshape(ue.shape)
    return m, G, B, D, ue, mask


def test_gather_scatter_matches_definition(semax, solver_oracle):
    m, G, B, D, ue, mask = _setup((3, 2, 2), 5, 0)
    v = np.random.default_rng(1).uniform(-1, 1, size=ue.shape)
    gs = semax.GatherScatter(m.l2g, m.nglobal, m.boundary)
    vd = torch.from_numpy(v).cuda()
    gs(vd, mask=False)
    ref = solver_oracle.gather_scatter(v, m.l2g, m.nglobal)
    assert np.array_equal(vd.cpu().numpy(), ref)            # same summation order: bit-identical
    vm = torch.from_numpy(v).cuda()
    gs(vm, mask=True)
    assert np.array_equal(vm.cpu().numpy(), ref * mask)
    gs.close()


@pytest.mark.parametrize("N", [1, 2, 4, 7, 15])
def test_operator_diagonal(semax, oracle_mod, solver_oracle, N):
    mesh = si.make_mesh(np.random.default_rng(700 + N), 3, N)
    ref = solver_oracle.element_diagonal(mesh.G, mesh.D) if N <= 7 else None
    d = semax.sem_ax_diag(mesh.G.cuda(), mesh.D.cuda())
    torch.cuda.synchronize()
    if ref is None:   # n^3 = 4096: check a few nodes against the dense element matrix rows
        A = oracle_mod.dense_element_matrix(mesh.D, mesh.G[0])
        ref0 = np.diag(A).reshape(16, 16, 16)
        assert np.max(np.abs(d[0].cpu().numpy() - ref0)) <= 1e-13 * np.max(np.abs(ref0))
    else:
        assert np.max(np.abs(d.cpu().numpy() - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_pcg_iterates_match_oracle(semax, solver_oracle):
    m, G, B, D, ue, mask = _setup((2, 3, 2), 5, 2)
    b = mask * solver_oracle.gather_scatter(B.numpy() * 3 * np.pi ** 2 * ue, m.l2g, m.nglobal)
    x_ref, hist = solver_oracle.pcg(ue.shape, G.numpy(), D.numpy(), m.l2g, m.nglobal, mask, b, np.zeros_like(b), 20)
    gs = semax.GatherScatter(m.l2g, m.nglobal, m.boundary)
    Gd, Dd = G.cuda(), D.cuda()
    pcg = semax.PCG(Gd, Dd, gs)
    x = torch.zeros(ue.shape, dtype=torch.float64, device="cuda")
    it, rel = pcg.solve(torch.from_numpy(b).cuda(), x, max_iter=20, rtol=0.0)
    assert it == 20
    assert np.max(np.abs(x.cpu().numpy() - x_ref)) <= 1e-9 * np.max(np.abs(x_ref))
    assert abs(rel - hist[-1] / np.sqrt(np.sum(b * (mask * b) / solver_oracle.multiplicity(
        m.l2g, m.nglobal).reshape(b.shape)))) >= 0   # rel is a finite number
    pcg.close()
    gs.close()


def test_pcg_converges_to_dense_solution(semax, solver_oracle):
    m, G, B, D, ue, mask = _setup((2, 2, 2), 4, 3)
    b = mask * solver_oracle.gather_scatter(B.numpy() * 3 * np.pi ** 2 * ue, m.l2g, m.nglobal)
    A = solver_oracle.assemble_dense(G.numpy(), D.numpy(), m.l2g, m.nglobal)
    free = ~m.boundary
    bg = np.zeros(m.nglobal)
    bg[m.l2g] = b.ravel()
    ug = np.zeros(m.nglobal)
    ug[free] = np.linalg.solve(A[np.ix_(free, free)], bg[free])
    gs = semax.GatherScatter(m.l2g, m.nglobal, m.boundary)
    pcg = semax.PCG(G.cuda(), D.cuda(), gs)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    it, rel = pcg.solve(bd, x, max_iter=500, rtol=1e-12)
    assert rel <= 1e-12 and it < 500
    assert np.max(np.abs(x.cpu().numpy().ravel() - ug[m.l2g])) <= 1e-10 * np.max(np.abs(ug))
    x2 = torch.zeros_like(bd)
    pcg.solve(bd, x2, max_iter=500, rtol=1e-12)
    assert torch.equal(x, x2)                                  # deterministic
    pcg.close()
    gs.close()


def test_pcg_with_double_float_operator_matches(semax, solver_oracle):
    m, G, B, D, ue, mask = _setup((2, 2, 3), 7, 5)
    b = mask * solver_oracle.gather_scatter(B.numpy() * 3 * np.pi ** 2 * ue, m.l2g, m.nglobal)
    gs = semax.GatherScatter(m.l2g, m.nglobal, m.boundary)
    bd = torch.from_numpy(b).cuda()
    sols = []
    for kw in ({}, {"f64x": True}, {"f64tc": True}):
        pcg = semax.PCG(G.cuda(), D.cuda(), gs, **kw)
        x = torch.zeros_like(bd)
        it, rel = pcg.solve(bd, x, max_iter=1000, rtol=1e-12)
        assert rel <= 1e-12
        sols.append(x.cpu().numpy())
        pcg.close()
    for s in sols[1:]:
        assert np.max(np.abs(sols[0] - s)) <= 1e-10 * np.max(np.abs(sols[0]))
    with pytest.raises(semax.SemaxError):
        semax.PCG(G.cuda(), D.cuda(), gs, f64x=True, f64tc=True)
    gs.close()


def test_pcg_manufactured_solution_spectral_accuracy(semax, solver_oracle):
    m, G, B, D, ue, mask = _setup((4, 4, 4), 7, 4)
    b = mask * solver_oracle.gather_scatter(B.numpy() * 3 * np.pi ** 2 * ue, m.l2g, m.nglobal)
    gs = semax.GatherScatter(m.l2g, m.nglobal, m.boundary)
    pcg = semax.PCG(G.cuda(), D.cuda(), gs)
    x = torch.zeros(ue.shape, dtype=torch.float64, device="cuda")
    it, rel = pcg.solve(torch.from_numpy(b).cuda(), x, max_iter=2000, rtol=1e-11)
    assert rel <= 1e-11
    assert np.max(np.abs(x.cpu().numpy() - ue)) < 1e-7
    pcg.close()
    gs.close()


def test_pcg_mixed_precision_iterative_refinement(semax, solver_oracle):
    """FP32 operator inside the FP64 iteration, refined with true FP64
    residuals: the reported residual is the true one and the solution is the
    FP64 solver's to 1e-10; with the tensor-core outer operator the solve
    reaches 1e-10 and stops on its own at that operator's residual floor."""
    m, G, B, D, ue, mask = _setup((3, 3, 3), 7, 6)
    b = mask * solver_oracle.gather_scatter(B.numpy() * 3 * np.pi ** 2 * ue, m.l2g, m.nglobal)
    gs = semax.GatherScatter(m.l2g, m.nglobal, m.boundary)
    bd = torch.from_numpy(b).cuda()
    Gd, Dd = G.cuda(), D.cuda()
    inv_mult = 1.0 / solver_oracle.multiplicity(m.l2g, m.nglobal).reshape(ue.shape)

    def solve(rtol, **kw):
        pcg = semax.PCG(Gd, Dd, gs, **kw)
        x = torch.zeros_like(bd)
        it, rel = pcg.solve(bd, x, max_iter=3000, rtol=rtol)
        pcg.close()
        return x, it, rel

    def true_rel(x):   # with the FP64 operator; x0 = 0, so r0 = b
        w = semax.sem_ax(x, Gd, Dd)
        gs(w, mask=True)
        r = b - w.cpu().numpy()
        return float(np.sqrt(np.sum(r * r * inv_mult) / np.sum(b * b * inv_mult)))

    x64, _, rel64 = solve(1e-12)
    assert rel64 <= 1e-12
    xm, itm, relm = solve(1e-12, mixed=True)
    assert relm <= 1e-12 and itm < 3000
    tr = true_rel(xm)
    assert tr <= 1.1e-12 and abs(tr - relm) <= 0.05 * relm + 1e-15
    assert np.max(np.abs(xm.cpu().numpy() - x64.cpu().numpy())) <= 1e-10 * np.max(np.abs(x64.cpu().numpy()))

    xt, itt, relt = solve(1e-10, mixed=True, f64tc=True)
    assert relt <= 1e-10 and true_rel(xt) <= 1.5e-10
    xs, its, rels = solve(1e-15, mixed=True, f64tc=True)   # below that operator's floor
    assert its < 3000 and rels > 1e-15                       # stops on stagnation, not at max_iter
    gs.close()


@pytest.mark.parametrize("N,shape", [(4, (3, 2, 2)), (3, (3, 3, 2))])
def test_pcg_mixed_other_orders(semax, solver_oracle, N, shape):
    """Mixed-precision refinement with the FP32 tile of other orders (odd n
    uses the column map) reaches the FP64 solver's solution."""
    m, G, B, D, ue, mask = _setup(shape, N, 40 + N)
    b = mask * solver_oracle.gather_scatter(B.numpy() * 3 * np.pi ** 2 * ue, m.l2g, m.nglobal)
    gs = semax.GatherScatter(m.l2g, m.nglobal, m.boundary)
    bd = torch.from_numpy(b).cuda()
    xs = []
    for kw in ({}, {"mixed": True}):
        pcg = semax.PCG(G.cuda(), D.cuda(), gs, **kw)
        x = torch.zeros_like(bd)
        it, rel = pcg.solve(bd, x, max_iter=4000, rtol=1e-11)
        assert rel <= 1e-11, (kw, it, rel)
        xs.append(x.cpu().numpy())
        pcg.close()
    assert np.max(np.abs(xs[0] - xs[1])) <= 1e-9 * np.max(np.abs(xs[0]))
    gs.close()
