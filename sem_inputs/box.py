"""Conforming hexahedral box meshes for solver tests and benchmarks.

Ex x Ey x Ez elements of order N on [0, 1]^3.  The global vertex grid has its
interior vertices jittered (shared by every element that touches them, so the
trilinear maps agree on shared faces and the mesh stays conforming); boundary
vertices stay on their faces.  Global GLL node numbering is the tensor grid
(Ex N + 1) x (Ey N + 1) x (Ez N + 1), x fastest; element e = ex + Ex (ey + Ey ez)
maps its local node (k, j, i) to global (ex N + i, ey N + j, ez N + k).

Nothing here applies the operator or solves anything.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from .gll import gll_nodes, gll_diff_matrix
from .geometry import geometric_factors, mass_diagonal, _VERTS


@dataclass
class BoxMesh:
    N: int
    shape: tuple[int, int, int]
    X: np.ndarray              # (E, 8, 3) element vertices
    l2g: np.ndarray            # (E * n^3,) int64 global node of each local node
    nglobal: int
    boundary: np.ndarray       # (nglobal,) bool, on the domain boundary
    coords: np.ndarray         # (E, n, n, n, 3) physical coordinates of the local nodes

    @property
    def E(self) -> int:
        return self.X.shape[0]

    @property
    def n(self) -> int:
        return self.N + 1


def box_mesh(Ex: int, Ey: int, Ez: int, N: int, rng: np.random.Generator, jitter: float = 0.1) -> BoxMesh:
    n = N + 1
    vx, vy, vz = np.meshgrid(np.arange(Ex + 1) / Ex, np.arange(Ey + 1) / Ey, np.arange(Ez + 1) / Ez,
                             indexing="ij")
    V = np.stack([vx, vy, vz], -1)                                   # [ix, iy, iz, 3]
    h = np.array([1.0 / Ex, 1.0 / Ey, 1.0 / Ez])
    d = rng.uniform(-1.0, 1.0, size=V.shape) * jitter * h / 2
    d[0, :, :, :] = d[-1, :, :, :] = 0
    d[:, 0, :, :] = d[:, -1, :, :] = 0
    d[:, :, 0, :] = d[:, :, -1, :] = 0
    V = V + d
    E = Ex * Ey * Ez
    X = np.empty((E, 8, 3))
    l2g = np.empty((E, n, n, n), dtype=np.int64)
    gx, gy, gz = Ex * N + 1, Ey * N + 1, Ez * N + 1
    kk, jj, ii = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    for ez in range(Ez):
        for ey in range(Ey):
            for ex in range(Ex):
                e = ex + Ex * (ey + Ey * ez)
                for v in range(8):
                    a, b, c = v & 1, (v >> 1) & 1, (v >> 2) & 1
                    X[e, v] = V[ex + a, ey + b, ez + c]
                l2g[e] = (ex * N + ii) + gx * ((ey * N + jj) + gy * (ez * N + kk))
    g = np.arange(gx * gy * gz)
    gi, gj, gk = g % gx, (g // gx) % gy, g // (gx * gy)
    boundary = (gi == 0) | (gi == gx - 1) | (gj == 0) | (gj == gy - 1) | (gk == 0) | (gk == gz - 1)
    xi = gll_nodes(N)
    t, s, r = np.meshgrid(xi, xi, xi, indexing="ij")
    rst = np.stack([r, s, t], -1)                                    # [k][j][i][3]
    Nv = np.prod(1.0 + rst[..., None, :] * _VERTS[None, None, None], axis=-1) / 8.0   # [k][j][i][v]
    coords = np.einsum("kjiv,eva->ekjia", Nv, X)
    return BoxMesh(N=N, shape=(Ex, Ey, Ez), X=X, l2g=l2g.reshape(-1), nglobal=int(gx * gy * gz),
                   boundary=boundary, coords=coords)


def box_operator_data(m: BoxMesh, device="cpu"):
    """(G, B, D) for the box mesh: geometric factors, mass diagonal, D."""
    G = geometric_factors(m.X, m.N, device=device)
    B = mass_diagonal(m.X, m.N, device=device)
    D = torch.from_numpy(gll_diff_matrix(m.N)).to(device)
    return G, B, D
