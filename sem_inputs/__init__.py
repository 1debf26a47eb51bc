"""Seeded synthetic inputs for the spectral-element Ax operator.

This package is shared by the CPU oracle's tests, the GPU parity tests and the
benchmark.  It produces inputs only (GLL data, D, geometric factors G, the
field u, and the order mix of the batched workload); it contains none of the
operator's arithmetic.

Workloads (all synthetic, seed = numpy.random.default_rng([1503, 7659, c])):

  c=0  N=7,  E=512      FP64            (small: oracle finishes in well under 1 s)
  c=1  N=7,  E=32768    FP64            (16.8M nodes, ~1.07 GB per call)
  c=2  N=15, E=8192     FP32 / BF16x3   (33.5M nodes; FP32 storage of u, G)
  c=3  N in {3,5,7,9,11,15}, geometric order mix, ~4.19M nodes, FP64, batched
  c=4  N=7,  E=262144   FP64 and FP32   (134M nodes)
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from .gll import gll_nodes, gll_weights, gll_diff_matrix, legendre
from .geometry import (G_COMPONENTS, draw_geometry, vertices, geometric_factors,
                       jacobian_determinants, mass_diagonal)
from .box import BoxMesh, box_mesh, box_operator_data

SEED_BASE = (1503, 7659)

# per-workload element count and order; c=3 is the batched mix
WORKLOADS = {
    0: dict(N=7, E=512),
    1: dict(N=7, E=32768),
    2: dict(N=15, E=8192),
    3: dict(orders=(3, 5, 7, 9, 11, 15), target_nodes=4_194_304, ratio=0.7),
    4: dict(N=7, E=262144),
}


def rng_for(c: int, extra: int | None = None) -> np.random.Generator:
    seed = [*SEED_BASE, c] if extra is None else [*SEED_BASE, c, extra]
    return np.random.default_rng(seed)


@dataclass
class Mesh:
    """One group of E elements of order N: u [E,n,n,n], G [E,6,n,n,n], D [n,n]."""
    N: int
    E: int
    u: torch.Tensor
    G: torch.Tensor
    D: torch.Tensor
    X: np.ndarray = field(repr=False, default=None)  # vertices (E, 8, 3)

    @property
    def n(self) -> int:
        return self.N + 1

    @property
    def dofs(self) -> int:
        return self.E * self.n ** 3


def make_mesh(rng: np.random.Generator, E: int, N: int, device="cpu",
              kind: str = "perturbed", h: float = 1.0) -> Mesh:
    """Draw geometry then u ~ U(-1,1) for E elements of order N.

    kind: "perturbed" (affine x (I + 0.1 M) plus 10% vertex jitter: trilinear),
          "affine"    (no vertex jitter), or "cube" (J = (h/2) I exactly).
    """
    n = N + 1
    A, delta = draw_geometry(rng, E, h=h)
    if kind == "affine":
        delta = np.zeros_like(delta)
    elif kind == "cube":
        A = np.broadcast_to((h / 2.0) * np.eye(3), (E, 3, 3)).copy()
        delta = np.zeros_like(delta)
    elif kind != "perturbed":
        raise ValueError(kind)
    X = vertices(A, delta)
    G = geometric_factors(X, N, device=device)
    u = torch.from_numpy(rng.uniform(-1.0, 1.0, size=(E, n, n, n))).to(device)
    D = torch.from_numpy(gll_diff_matrix(N)).to(device)
    return Mesh(N=N, E=E, u=u, G=G, D=D, X=X)


def batched_orders(rng: np.random.Generator, orders=(3, 5, 7, 9, 11, 15),
                   target_nodes: int = 4_194_304, ratio: float = 0.7) -> dict[int, int]:
    """Element count per order for the uneven-order workload.

    Each element's order index m (into the ascending `orders`) is i.i.d. with
    P(m) proportional to ratio**m (a geometric law truncated to the list);
    elements are drawn until the node count sum (N+1)^3 reaches target_nodes.
    """
    p = ratio ** np.arange(len(orders))
    p = p / p.sum()
    idx = rng.choice(len(orders), size=target_nodes // 64 + 1, p=p)
    nodes = np.cumsum((np.asarray(orders)[idx] + 1) ** 3)
    stop = int(np.searchsorted(nodes, target_nodes)) + 1
    counts = np.bincount(idx[:stop], minlength=len(orders))
    return {N: int(k) for N, k in zip(orders, counts) if k > 0}


def make_workload(c: int, device="cpu", E: int | None = None) -> list[Mesh]:
    """Meshes of workload c (a list with one Mesh, or one per order for c=3).

    E overrides the element count (for reduced-size cases of the same recipe)."""
    spec = WORKLOADS[c]
    rng = rng_for(c)
    if c == 3:
        counts = batched_orders(rng, spec["orders"], spec["target_nodes"], spec["ratio"])
        return [make_mesh(rng, k, N, device=device) for N, k in sorted(counts.items())]
    return [make_mesh(rng, spec["E"] if E is None else E, spec["N"], device=device)]


def per_element_g_scale(G: torch.Tensor) -> torch.Tensor:
    """Power-of-two scale s_e = 2^ceil(log2 max|G_e|) per element (exact to
    apply and to undo in binary floating point)."""
    m = G.abs().reshape(G.shape[0], -1).amax(dim=1)
    return torch.exp2(torch.ceil(torch.log2(m)))


__all__ = [
    "SEED_BASE", "WORKLOADS", "Mesh", "make_mesh", "make_workload", "batched_orders",
    "rng_for", "per_element_g_scale", "gll_nodes", "gll_weights", "gll_diff_matrix",
    "legendre", "G_COMPONENTS", "draw_geometry", "vertices", "geometric_factors",
    "jacobian_determinants", "mass_diagonal", "BoxMesh", "box_mesh", "box_operator_data",
]
