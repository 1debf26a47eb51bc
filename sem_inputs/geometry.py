"""Seeded synthetic hexahedral geometry and the geometric factors G.

Each element is the image of the reference cube [-1,1]^3 under a trilinear map
x(r,s,t) = sum_v X_v N_v(r,s,t) through 8 vertices X_v, with
N_v = (1 + r_v r)(1 + s_v s)(1 + t_v t) / 8.  The vertices come from a random
affine map perturbed by 10%:

    A_e = (h/2) (I + 0.1 M_e),  M_e ~ U(-1,1)^{3x3}
    X_v = A_e xi_v + delta_v,   delta_v ~ 0.1 (h/2) U(-1,1)^3

so the map is trilinear, not affine, once delta is nonzero.  At every GLL node
(xi_i, xi_j, xi_k) (r = xi_i along the fastest index i) the Jacobian
J[a][b] = d x_a / d xi_b is formed and

    G = det(J) w_i w_j w_k J^{-1} J^{-T}                         (3x3, SPD)

is stored as six components in the order (rr, rs, rt, ss, st, tt), layout
[E][6][k][j][i] (component-major within an element).  This is the textbook
weak-form Laplacian metric (Deville, Fischer & Mund 2002, Sec. 4.4): the
element stiffness is the sum over a, b of D_a^T diag(G_ab) D_b.

Random draws use numpy's PCG64 generator; the arithmetic runs in float64 torch
ops on whatever device the caller names, so large meshes can be built where
they are used.  Nothing here applies the operator.
"""
from __future__ import annotations

import numpy as np
import torch

from .gll import gll_nodes, gll_weights

# component order of the symmetric 3x3 factor
G_COMPONENTS = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))

# reference-cube vertices, v = a + 2 b + 4 c  ->  (+-1, +-1, +-1)
_VERTS = np.array([[2 * (v & 1) - 1, 2 * ((v >> 1) & 1) - 1, 2 * ((v >> 2) & 1) - 1]
                   for v in range(8)], dtype=np.float64)


def draw_geometry(rng: np.random.Generator, E: int, h: float = 1.0,
                  affine_perturb: float = 0.1, vertex_perturb: float = 0.1):
    """Draw the per-element affine matrices A (E,3,3) and vertex offsets
    delta (E,8,3).  Draw order: all M_e first, then all delta."""
    M = rng.uniform(-1.0, 1.0, size=(E, 3, 3))
    delta = rng.uniform(-1.0, 1.0, size=(E, 8, 3))
    A = (h / 2.0) * (np.eye(3)[None] + affine_perturb * M)
    delta = vertex_perturb * (h / 2.0) * delta
    return A, delta


def vertices(A: np.ndarray, delta: np.ndarray) -> np.ndarray:
    """X[e, v, a] = (A_e xi_v)_a + delta[e, v, a]."""
    return np.einsum("eab,vb->eva", A, _VERTS) + delta


def _shape_gradients(N: int) -> np.ndarray:
    """dN[p, v, d]: derivative of N_v along reference direction d at GLL node
    p = (k*n + j)*n + i, i.e. (r, s, t) = (xi_i, xi_j, xi_k)."""
    xi = gll_nodes(N)
    n = N + 1
    t, s, r = np.meshgrid(xi, xi, xi, indexing="ij")  # [k][j][i]
    rst = np.stack([r.ravel(), s.ravel(), t.ravel()], axis=1)  # (n^3, 3)
    f = 1.0 + rst[:, None, :] * _VERTS[None, :, :]  # (n^3, 8, 3): 1 + xi_v,d * x_d
    dN = np.empty((n ** 3, 8, 3))
    dN[:, :, 0] = _VERTS[None, :, 0] * f[:, :, 1] * f[:, :, 2] / 8.0
    dN[:, :, 1] = f[:, :, 0] * _VERTS[None, :, 1] * f[:, :, 2] / 8.0
    dN[:, :, 2] = f[:, :, 0] * f[:, :, 1] * _VERTS[None, :, 2] / 8.0
    return dN


def _node_weights(N: int) -> np.ndarray:
    w = gll_weights(N)
    return np.einsum("k,j,i->kji", w, w, w).reshape(-1)  # (n^3,)


def geometric_factors(X: np.ndarray, N: int, device="cpu", chunk: int = 8192) -> torch.Tensor:
    """G [E, 6, n, n, n] float64 on `device` from vertices X [E, 8, 3].

    Raises ValueError if det(J) <= 0 at any node (a folded element)."""
    n = N + 1
    E = X.shape[0]
    dev = torch.device(device)
    dN = torch.from_numpy(_shape_gradients(N)).to(dev)            # (p, v, d)
    wq = torch.from_numpy(_node_weights(N)).to(dev)               # (p,)
    G = torch.empty((E, 6, n ** 3), dtype=torch.float64, device=dev)
    Xt = torch.from_numpy(np.ascontiguousarray(X)).to(dev)
    for e0 in range(0, E, chunk):
        Xc = Xt[e0:e0 + chunk]                                    # (c, v, a)
        J = torch.einsum("cva,pvd->cpad", Xc, dN)                 # (c, p, a, d)
        a, b, c_ = J[..., 0, 0], J[..., 0, 1], J[..., 0, 2]
        d, e, f = J[..., 1, 0], J[..., 1, 1], J[..., 1, 2]
        g, h, i = J[..., 2, 0], J[..., 2, 1], J[..., 2, 2]
        # adjugate: J^{-1} = adj / det
        adj = torch.stack([
            torch.stack([e * i - f * h, c_ * h - b * i, b * f - c_ * e], -1),
            torch.stack([f * g - d * i, a * i - c_ * g, c_ * d - a * f], -1),
            torch.stack([d * h - e * g, b * g - a * h, a * e - b * d], -1),
        ], -2)                                                    # (c, p, 3, 3)
        det = a * adj[..., 0, 0] + b * adj[..., 1, 0] + c_ * adj[..., 2, 0]
        if bool((det <= 0).any()):
            raise ValueError("non-positive Jacobian determinant")
        # det * w * J^{-1} J^{-T} = w * adj adj^T / det
        scale = wq[None, :] / det
        for m, (p, q) in enumerate(G_COMPONENTS):
            G[e0:e0 + chunk, m] = scale * (adj[..., p, :] * adj[..., q, :]).sum(-1)
    return G.view(E, 6, n, n, n)


def mass_diagonal(X: np.ndarray, N: int, device="cpu", chunk: int = 8192) -> torch.Tensor:
    """B [E, n, n, n] = det(J) w_i w_j w_k at every GLL node: the diagonal of
    the GLL-collocated mass matrix (Deville, Fischer & Mund 2002, Sec. 4.4)."""
    n = N + 1
    E = X.shape[0]
    dev = torch.device(device)
    dN = torch.from_numpy(_shape_gradients(N)).to(dev)
    wq = torch.from_numpy(_node_weights(N)).to(dev)
    B = torch.empty((E, n ** 3), dtype=torch.float64, device=dev)
    Xt = torch.from_numpy(np.ascontiguousarray(X)).to(dev)
    for e0 in range(0, E, chunk):
        J = torch.einsum("cva,pvd->cpad", Xt[e0:e0 + chunk], dN)
        det = (J[..., 0, 0] * (J[..., 1, 1] * J[..., 2, 2] - J[..., 1, 2] * J[..., 2, 1])
               - J[..., 0, 1] * (J[..., 1, 0] * J[..., 2, 2] - J[..., 1, 2] * J[..., 2, 0])
               + J[..., 0, 2] * (J[..., 1, 0] * J[..., 2, 1] - J[..., 1, 1] * J[..., 2, 0]))
        B[e0:e0 + chunk] = det * wq[None, :]
    return B.view(E, n, n, n)


def jacobian_determinants(X: np.ndarray, N: int) -> np.ndarray:
    """det(J) at every node, (E, n^3), float64 on the host (for checks)."""
    dN = _shape_gradients(N)
    J = np.einsum("eva,pvd->epad", X, dN)
    return np.linalg.det(J)
