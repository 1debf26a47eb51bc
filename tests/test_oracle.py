"""Pins for the CPU oracle and the input generators (no GPU).

Nothing here compares the oracle with itself.  Each test fixes a part through
mathematics that holds independently of the loop nest:

  part                         pin                                          catches
  ---------------------------  -------------------------------------------  -----------------------------
  GLL nodes / weights          3-point rule by hand (golden); exactness of  wrong node equation, weight
                               the rule to degree 2N-1                      formula
  D                            N=2 by hand (golden); D x^p = p x^{p-1} for  off-diagonal formula, sign of
                               p <= N; D_00 = -N(N+1)/4                     the diagonal
  1D stiffness D^T W D         N=1, N=2 closed forms (golden)               D, W together
  oracle on a cube             A = (h/2)(W(x)W(x)K + W(x)K(x)W + K(x)W(x)W)  wrong direction / index, D vs
                               (Kronecker closed form)                      D^T, dropped direction
  oracle on an affine element  u = a.x + c: u^T A u = |a|^2 vol exactly;    dropped / mis-signed cross
                               (Au) = 0 at interior nodes                   terms of G, G generator
  oracle on perturbed elements dense Kronecker-assembled A_e (independent   any term, index or transpose
                               formulation) times u_e                       error in the loop nest
  invariants                   A.1 = 0; v.Au = u.Av; u.Au >= 0; one zero    asymmetric transposed step
                               eigenvalue (constants)
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import sem_inputs as si

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frac_array(rows):
    return np.array([[float(Fraction(x)) for x in r] for r in rows])


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- GLL and D

def test_gll_three_point_rule_matches_hand_values():
    g = _golden("gll_N2.json")
    x = si.gll_nodes(2)
    w = si.gll_weights(2)
    D = si.gll_diff_matrix(2)
    np.testing.assert_allclose(x, [float(Fraction(v)) for v in g["nodes"]], atol=1e-16)
    np.testing.assert_allclose(w, [float(Fraction(v)) for v in g["weights"]], rtol=1e-15)
    np.testing.assert_allclose(D, _frac_array(g["D"]), atol=1e-15)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 7, 9, 11, 15])
def test_gll_quadrature_exact_to_degree_2N_minus_1(N):
    x, w = si.gll_nodes(N), si.gll_weights(N)
    assert np.all(np.diff(x) > 0) and x[0] == -1.0 and x[-1] == 1.0
    for p in range(2 * N):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.dot(w, x ** p) - exact) < 4e-15, (N, p)
    # degree 2N is NOT integrated exactly by an (N+1)-point Lobatto rule
    assert abs(np.dot(w, x ** (2 * N)) - 2.0 / (2 * N + 1)) > 1e-10


@pytest.mark.parametrize("N", [1, 2, 3, 5, 7, 9, 11, 15])
def test_D_differentiates_polynomials_up_to_degree_N(N):
    x, D = si.gll_nodes(N), si.gll_diff_matrix(N)
    for p in range(N + 1):
        f = x ** p
        df = p * x ** (p - 1) if p > 0 else np.zeros_like(x)
        tol = 100 * np.finfo(float).eps * N * N * max(1.0, np.max(np.abs(df)))
        assert np.max(np.abs(D @ f - df)) <= tol, (N, p)
    assert abs(D[0, 0] + N * (N + 1) / 4) < 1e-12 * N * N
    assert abs(D[N, N] - N * (N + 1) / 4) < 1e-12 * N * N
    # exact centro-antisymmetry (the generator enforces it bit for bit)
    assert np.array_equal(D, -D[::-1, ::-1])


@pytest.mark.parametrize("N", [1, 2])
def test_1d_stiffness_closed_form(N):
    K_ref = _frac_array(_golden("stiffness_1d.json")["K"][str(N)])
    D, w = si.gll_diff_matrix(N), si.gll_weights(N)
    np.testing.assert_allclose(D.T @ np.diag(w) @ D, K_ref, atol=1e-14)


# ---------------------------------------------------------------- geometry

def test_geometric_factor_is_spd_with_positive_jacobian():
    rng = np.random.default_rng(1)
    m = si.make_mesh(rng, 16, 5)
    assert (si.jacobian_determinants(m.X, 5) > 0).all()
    G = m.G.numpy()
    n = 6
    for e in range(4):
        for p in range(0, n ** 3, 17):
            k, j, i = np.unravel_index(p, (n, n, n))
            c = G[e, :, k, j, i]
            M = np.array([[c[0], c[1], c[2]], [c[1], c[3], c[4]], [c[2], c[4], c[5]]])
            assert np.all(np.linalg.eigvalsh(M) > 0)


def test_cube_geometric_factor_closed_form():
    # J = (h/2) I:  G_aa = (h/2) w_i w_j w_k, off-diagonal zero
    h = 1.0
    N = 4
    m = si.make_mesh(np.random.default_rng(2), 3, N, kind="cube", h=h)
    w = si.gll_weights(N)
    W3 = np.einsum("k,j,i->kji", w, w, w)
    G = m.G.numpy()
    for comp in (0, 3, 5):
        np.testing.assert_allclose(G[:, comp], np.broadcast_to((h / 2) * W3, G[:, comp].shape), rtol=1e-14)
    for comp in (1, 2, 4):
        assert np.max(np.abs(G[:, comp])) < 1e-15


# ---------------------------------------------------------------- oracle Ax

@pytest.mark.parametrize("N", [1, 2, 4, 7])
def test_oracle_cube_matches_kronecker_closed_form(oracle_mod, N):
    h = 1.0
    m = si.make_mesh(np.random.default_rng(3), 4, N, kind="cube", h=h)
    if N in (1, 2):   # hand-derived K, independent of the D generator
        K = _frac_array(_golden("stiffness_1d.json")["K"][str(N)])
        W = np.diag([float(Fraction(v)) for v in _golden("gll_N2.json")["weights"]]) if N == 2 else np.eye(2)
    else:
        D, w = si.gll_diff_matrix(N), si.gll_weights(N)
        K, W = D.T @ np.diag(w) @ D, np.diag(w)
    A = (h / 2) * (np.kron(W, np.kron(W, K)) + np.kron(W, np.kron(K, W)) + np.kron(K, np.kron(W, W)))
    w_or = oracle_mod.sem_ax(m.u, m.G, m.D)
    u = m.u.numpy().reshape(4, -1)
    ref = u @ A.T
    err = np.max(np.abs(w_or.reshape(4, -1) - ref)) / np.max(np.abs(ref))
    assert err < 1e-13


@pytest.mark.parametrize("N", [2, 3, 5, 7])
def test_oracle_affine_element_energy_and_interior_zero(oracle_mod, N):
    rng = np.random.default_rng(4)
    E = 6
    m = si.make_mesh(rng, E, N, kind="affine")
    n = N + 1
    xi = si.gll_nodes(N)
    # nodal coordinates of the affine map x = A_e xi (vertices X_v = A_e xi_v)
    A_e = np.einsum("eva,vb->eab", m.X, np.array(
        [[2 * (v & 1) - 1, 2 * ((v >> 1) & 1) - 1, 2 * ((v >> 2) & 1) - 1] for v in range(8)])) / 8.0
    t, s, r = np.meshgrid(xi, xi, xi, indexing="ij")
    ref = np.stack([r, s, t], -1)                     # [k][j][i][3]
    x = np.einsum("eab,kjib->ekjia", A_e, ref)        # [E][k][j][i][3]
    a = rng.uniform(-1, 1, size=(E, 3))
    c = rng.uniform(-1, 1, size=(E, 1, 1, 1))
    u = np.einsum("ekjia,ea->ekji", x, a) + c
    w = oracle_mod.sem_ax(u, m.G, m.D)
    vol = 8.0 * np.linalg.det(A_e)
    energy = np.einsum("ekji,ekji->e", u, w)
    np.testing.assert_allclose(energy, np.sum(a * a, 1) * vol, rtol=1e-12)
    interior = w[:, 1:-1, 1:-1, 1:-1]
    if interior.size:
        assert np.max(np.abs(interior)) < 1e-12 * np.max(np.abs(w))


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7])
def test_oracle_matches_dense_kronecker_operator(oracle_mod, N):
    m = si.make_mesh(np.random.default_rng(5), 3, N)
    w = oracle_mod.sem_ax(m.u, m.G, m.D)
    for e in range(3):
        A = oracle_mod.dense_element_matrix(m.D, m.G[e])
        ref = A @ m.u[e].numpy().ravel()
        err = np.max(np.abs(w[e].ravel() - ref)) / np.max(np.abs(ref))
        assert err < 1e-13, (N, e, err)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_dense_operator_symmetric_psd_with_constant_nullspace(oracle_mod, N):
    m = si.make_mesh(np.random.default_rng(6), 2, N)
    for e in range(2):
        A = oracle_mod.dense_element_matrix(m.D, m.G[e])
        assert np.max(np.abs(A - A.T)) < 1e-14 * np.max(np.abs(A))
        ev = np.linalg.eigvalsh(0.5 * (A + A.T))
        scale = ev[-1]
        assert ev[0] > -1e-13 * scale
        assert abs(ev[0]) < 1e-13 * scale and ev[1] > 1e-6 * scale


def test_oracle_invariants_on_perturbed_mesh(oracle_mod):
    m = si.make_mesh(np.random.default_rng(7), 40, 7)
    u = m.u.numpy()
    v = np.random.default_rng(8).uniform(-1, 1, size=u.shape)
    Au = oracle_mod.sem_ax(u, m.G, m.D)
    Av = oracle_mod.sem_ax(v, m.G, m.D)
    A1 = oracle_mod.sem_ax(np.ones_like(u), m.G, m.D)
    assert np.max(np.abs(A1)) <= 1e-12 * np.max(np.abs(Au))
    for e in range(40):
        vAu, uAv = np.dot(v[e].ravel(), Au[e].ravel()), np.dot(u[e].ravel(), Av[e].ravel())
        assert abs(vAu - uAv) <= 1e-12 * np.linalg.norm(v[e]) * np.linalg.norm(Au[e])
        assert np.dot(u[e].ravel(), Au[e].ravel()) > 0


def test_oracle_zero_elements(oracle_mod):
    D = si.gll_diff_matrix(3)
    w = oracle_mod.sem_ax(np.zeros((0, 4, 4, 4)), np.zeros((0, 6, 4, 4, 4)), D)
    assert w.shape == (0, 4, 4, 4)


def test_oracle_reduce_definitions(oracle_mod):
    a = np.array([1.0, -2.0, 3.5])
    b = np.array([1.5, -2.0, -4.0])
    mx, mb, dot = oracle_mod.reduce(a, b)
    assert mx == 7.5 and mb == 4.0 and dot == 1.5 + 4.0 - 14.0


def test_batched_order_mix_reaches_target():
    counts = si.batched_orders(si.rng_for(3))
    nodes = sum((N + 1) ** 3 * k for N, k in counts.items())
    assert 4_194_304 <= nodes < 4_194_304 + 16 ** 3
    assert set(counts) <= {3, 5, 7, 9, 11, 15}
    # geometric law: lower orders are drawn more often
    ks = [counts[N] for N in sorted(counts)]
    assert ks == sorted(ks, reverse=True)


# ---------------------------------------------------------------- Helmholtz form h1 A u + h2 B u

def test_mass_diagonal_closed_forms():
    """B = det(J) w_i w_j w_k: (h/2)^3 w_i w_j w_k on the cube; its sum is the
    element volume, exactly 8 det(A_e) for an affine element."""
    N = 5
    h = 0.7
    cube = si.make_mesh(np.random.default_rng(40), 3, N, kind="cube", h=h)
    w = si.gll_weights(N)
    B = si.mass_diagonal(cube.X, N).numpy()
    np.testing.assert_allclose(B, np.broadcast_to((h / 2) ** 3 * np.einsum("k,j,i->kji", w, w, w), B.shape),
                               rtol=1e-14)
    assert np.allclose(B.reshape(3, -1).sum(1), h ** 3, rtol=1e-14)
    aff = si.make_mesh(np.random.default_rng(41), 4, N, kind="affine")
    A_e = np.einsum("eva,vb->eab", aff.X, np.array(
        [[2 * (v & 1) - 1, 2 * ((v >> 1) & 1) - 1, 2 * ((v >> 2) & 1) - 1] for v in range(8)])) / 8.0
    Ba = si.mass_diagonal(aff.X, N).numpy().reshape(4, -1)
    np.testing.assert_allclose(Ba.sum(1), 8.0 * np.linalg.det(A_e), rtol=1e-13)


@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_oracle_helmholtz_matches_dense_and_reduces_to_ax(oracle_mod, N):
    m = si.make_mesh(np.random.default_rng(42 + N), 3, N)
    B = si.mass_diagonal(m.X, N)
    h1, h2 = 0.75, 3.5
    w = oracle_mod.sem_helmholtz(m.u, m.G, B, m.D, h1, h2)
    for e in range(3):
        H = h1 * oracle_mod.dense_element_matrix(m.D, m.G[e]) + h2 * np.diag(B[e].numpy().ravel())
        ref = H @ m.u[e].numpy().ravel()
        assert np.max(np.abs(w[e].ravel() - ref)) / np.max(np.abs(ref)) < 1e-13
        ev = np.linalg.eigvalsh(0.5 * (H + H.T))
        assert ev[0] > 0                                   # SPD once h2 > 0
    assert np.array_equal(oracle_mod.sem_helmholtz(m.u, m.G, B, m.D, 1.0, 0.0), oracle_mod.sem_ax(m.u, m.G, m.D))


def test_oracle_helmholtz_of_constant_is_mass(oracle_mod):
    """A 1 = 0, so H 1 = h2 B (and sums to h2 times the volume)."""
    m = si.make_mesh(np.random.default_rng(45), 6, 4)
    B = si.mass_diagonal(m.X, 4)
    one = np.ones_like(m.u.numpy())
    w = oracle_mod.sem_helmholtz(one, m.G, B, m.D, 2.0, 0.5)
    assert np.max(np.abs(w - 0.5 * B.numpy())) <= 1e-12 * np.max(np.abs(B.numpy()))
