"""CPU oracle for the solver built around Ax: direct stiffness summation
(gather-scatter), the operator's diagonal, dense assembly and Jacobi-
preconditioned conjugate gradients, all in float64 NumPy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Definitions:

* Q is the local-to-global Boolean map (E n^3 local nodes -> global nodes);
  direct stiffness summation is Q Q^T: every local value becomes the sum of
  the local values sharing its global node (Deville, Fischer & Mund 2002,
  Sec. 4.5).
* A vector is kept in local (element) form and is continuous when equal
  copies sit at shared nodes; the global inner product of two continuous
  vectors is sum_l a_l b_l / mult_l with mult_l the number of copies.
* PCG is Hestenes & Stiefel's conjugate gradient method with the Jacobi
  preconditioner diag(Q Q^T diag(A_L))^{-1}, homogeneous Dirichlet nodes held
  at zero by a mask.
"""
from __future__ import annotations

import numpy as np

from . import sem_ax, dense_element_matrix, _f64


def gather_scatter(v, l2g, nglobal: int) -> np.ndarray:
    """Q Q^T v for a local vector v (any shape with E n^3 entries)."""
    v = _f64(v)
    g = np.zeros(nglobal)
    np.add.at(g, l2g, v.ravel())
    return g[l2g].reshape(v.shape)


def multiplicity(l2g, nglobal: int) -> np.ndarray:
    return np.bincount(l2g, minlength=nglobal)[l2g].astype(np.float64)


def element_diagonal(G, D) -> np.ndarray:
    """diag(A_e) for every element, from the dense element matrices (small E)."""
    G, D = _f64(G), _f64(D)
    n = D.shape[0]
    return np.stack([np.diag(dense_element_matrix(D, G[e])).reshape(n, n, n) for e in range(G.shape[0])])


def assemble_dense(G, D, l2g, nglobal: int) -> np.ndarray:
    """Global stiffness Q A_L Q^T as a dense matrix (small meshes only)."""
    G, D = _f64(G), _f64(D)
    n3 = D.shape[0] ** 3
    A = np.zeros((nglobal, nglobal))
    for e in range(G.shape[0]):
        idx = l2g[e * n3:(e + 1) * n3]
        A[np.ix_(idx, idx)] += dense_element_matrix(D, G[e])
    return A


def pcg(u_shape, G, D, l2g, nglobal, mask, b, x0, iters: int, inv_diag=None):
    """`iters` Jacobi-PCG iterations on continuous local vectors.

    mask: 1 at free nodes, 0 at Dirichlet nodes (local form).  b: continuous
    right-hand side (already summed and masked).  Returns (x, residual norms
    sqrt(r.r) after each iteration)."""
    mult = multiplicity(l2g, nglobal).reshape(u_shape)
    mask = _f64(mask).reshape(u_shape)
    if inv_diag is None:
        dg = gather_scatter(element_diagonal(G, D), l2g, nglobal).reshape(u_shape)
        inv_diag = np.where(mask > 0, 1.0 / dg, 0.0)

    def A(v):
        return mask * gather_scatter(sem_ax(v, G, D), l2g, nglobal).reshape(u_shape)

    def dot(a, c):
        return float(np.sum(a * c / mult))

    x = _f64(x0).reshape(u_shape).copy()
    r = _f64(b).reshape(u_shape) - A(x)
    z = inv_diag * r
    p = z.copy()
    rz = dot(r, z)
    hist = []
    for _ in range(iters):
        w = A(p)
        alpha = rz / dot(p, w)
        x += alpha * p
        r -= alpha * w
        z = inv_diag * r
        rz_new = dot(r, z)
        hist.append(np.sqrt(dot(r, r)))
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, np.array(hist)
