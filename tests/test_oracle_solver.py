"""Pins for the solver oracle (gather-scatter, diagonal, assembly, PCG) on
conforming box meshes: closed forms, a dense direct solve, and spectral
convergence to a manufactured solution."""
import numpy as np
import pytest

import sem_inputs as si
from oracle import solver


def _mesh(shape=(2, 2, 2), N=3, seed=0):
    m = si.box_mesh(*shape, N, np.random.default_rng(seed))
    G, B, D = si.box_operator_data(m)
    return m, G.numpy(), B.numpy(), D.numpy()


def test_gather_scatter_is_multiplicity_on_continuous_vectors():
    m, *_ = _mesh((3, 2, 2), 4)
    g = np.random.default_rng(1).uniform(size=m.nglobal)
    v = g[m.l2g]
    np.testing.assert_allclose(solver.gather_scatter(v, m.l2g, m.nglobal),
                               solver.multiplicity(m.l2g, m.nglobal) * v, rtol=1e-15)
    mult = solver.multiplicity(m.l2g, m.nglobal)
    assert set(np.unique(mult)) <= {1.0, 2.0, 4.0, 8.0}
    assert np.isclose(np.sum(1.0 / mult), m.nglobal)


def test_element_diagonal_closed_form_on_cube(oracle_mod):
    """On the cube (J = h/2 I): diag A_e = (h/2)(w_j w_k K_ii + ...) with K = D^T W D."""
    N, h = 4, 1.0
    cube = si.make_mesh(np.random.default_rng(2), 2, N, kind="cube", h=h)
    w = si.gll_weights(N)
    D = si.gll_diff_matrix(N)
    K = D.T @ np.diag(w) @ D
    kd = np.diag(K)
    ref = (h / 2) * (np.einsum("k,j,i->kji", w, w, kd) + np.einsum("k,j,i->kji", w, kd, w)
                     + np.einsum("k,j,i->kji", kd, w, w))
    dg = solver.element_diagonal(cube.G, cube.D)
    np.testing.assert_allclose(dg, np.broadcast_to(ref, dg.shape), rtol=1e-13)


def test_assembled_matrix_symmetric_with_constant_nullspace():
    m, G, B, D = _mesh((2, 2, 1), 3)
    A = solver.assemble_dense(G, D, m.l2g, m.nglobal)
    assert np.max(np.abs(A - A.T)) < 1e-13 * np.max(np.abs(A))
    assert np.max(np.abs(A @ np.ones(m.nglobal))) < 1e-12 * np.max(np.abs(A))


def _manufactured(m, B):
    """-lap u = f on [0,1]^3, u = sin(pi x) sin(pi y) sin(pi z), zero on the boundary."""
    x = m.coords
    ue = np.sin(np.pi * x[..., 0]) * np.sin(np.pi * x[..., 1]) * np.sin(np.pi * x[..., 2])
    f = 3 * np.pi ** 2 * ue
    mask = (~m.boundary[m.l2g]).astype(np.float64).reshape(ue.shape)
    b = mask * solver.gather_scatter(B * f, m.l2g, m.nglobal).reshape(ue.shape)
    return ue, b, mask


def test_dense_direct_solve_converges_spectrally():
    errs = []
    for N in (3, 5, 7):
        m, G, B, D = _mesh((2, 2, 2), N, seed=3)
        ue, b, mask = _manufactured(m, B)
        A = solver.assemble_dense(G, D, m.l2g, m.nglobal)
        free = ~m.boundary
        bg = np.zeros(m.nglobal)
        bg[m.l2g] = b.ravel()
        ug = np.zeros(m.nglobal)
        ug[free] = np.linalg.solve(A[np.ix_(free, free)], bg[free])
        errs.append(np.max(np.abs(ug[m.l2g] - ue.ravel())))
    assert errs[0] < 2e-2 and errs[1] < 5e-4 and errs[2] < 1e-5
    assert errs[2] < errs[1] / 10 < errs[0] / 100           # exponential in N


def test_pcg_oracle_reaches_the_dense_solution():
    m, G, B, D = _mesh((2, 2, 2), 5, seed=4)
    ue, b, mask = _manufactured(m, B)
    x, hist = solver.pcg(ue.shape, G, D, m.l2g, m.nglobal, mask, b, np.zeros_like(b), 200)
    A = solver.assemble_dense(G, D, m.l2g, m.nglobal)
    free = ~m.boundary
    bg = np.zeros(m.nglobal)
    bg[m.l2g] = b.ravel()
    ug = np.zeros(m.nglobal)
    ug[free] = np.linalg.solve(A[np.ix_(free, free)], bg[free])
    assert hist[-1] < 1e-10 * hist[0]
    assert np.max(np.abs(x.ravel() - ug[m.l2g])) < 1e-9 * np.max(np.abs(ug))
