"""CPU oracle for the spectral-element Ax operator.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg import this package; the library never does, and the two share
no code.  Everything here is float64 on the host:

* ``sem_ax``  -- the plain C loop nest in sem_ax_oracle.c (the operator's
  definition written out; OpenMP over elements, no FMA contraction);
* ``sem_helmholtz`` -- h1 A u + h2 B u, the same loop nest plus the diagonal
  mass term;
* ``dense_element_matrix`` -- the same operator assembled as a dense
  n^3 x n^3 matrix from Kronecker products, an independent formulation used to
  pin the loop nest on small elements;
* ``reduce`` -- max|a-b|, max|b| and the dot product a.b, by their definitions.

Which pin fixes which part is listed in the oracle tests (tests/test_oracle.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sem_ax_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libsemax_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc -O2 -ffp-contract=off -fopenmp) if stale."""
    with _lock:
        if (not force and os.path.exists(_OUT)
                and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
            return _OUT
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                        "-std=c11", "-o", tmp, _SRC], check=True)
        os.replace(tmp, _OUT)
        return _OUT


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_sem_ax.restype = ctypes.c_int
        lib.oracle_sem_ax.argtypes = [ctypes.c_int64, ctypes.c_int] + [ctypes.c_void_p] * 4 + [ctypes.c_int]
        lib.oracle_sem_helmholtz.restype = ctypes.c_int
        lib.oracle_sem_helmholtz.argtypes = ([ctypes.c_int64, ctypes.c_int] + [ctypes.c_void_p] * 4 +
                                             [ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_int])
        _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    if hasattr(a, "detach"):  # torch tensor
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(a, dtype=np.float64)


def sem_ax(u, G, D, nthreads: int = 0, return_threads: bool = False):
    """w = Ax for u [E,n,n,n], G [E,6,n,n,n], D [n,n] (float64 on the host)."""
    u, G, D = _f64(u), _f64(G), _f64(D)
    n = D.shape[0]
    E = u.shape[0] if u.size else 0
    assert u.shape == (E, n, n, n) and G.shape == (E, 6, n, n, n) and D.shape == (n, n)
    w = np.empty_like(u)
    used = _load().oracle_sem_ax(E, n - 1, u.ctypes.data, G.ctypes.data, D.ctypes.data,
                                 w.ctypes.data, int(nthreads))
    if used < 0:
        raise RuntimeError("oracle_sem_ax failed")
    return (w, used) if return_threads else w


def sem_helmholtz(u, G, B, D, h1: float, h2: float, nthreads: int = 0):
    """w = h1 A u + h2 B u (B [E,n,n,n] the diagonal mass), float64 on the host."""
    u, G, B, D = _f64(u), _f64(G), _f64(B), _f64(D)
    n = D.shape[0]
    E = u.shape[0] if u.size else 0
    assert B.shape == u.shape
    w = np.empty_like(u)
    if _load().oracle_sem_helmholtz(E, n - 1, u.ctypes.data, G.ctypes.data, B.ctypes.data, D.ctypes.data,
                                    float(h1), float(h2), w.ctypes.data, int(nthreads)) < 0:
        raise RuntimeError("oracle_sem_helmholtz failed")
    return w


def dense_element_matrix(D, G_e) -> np.ndarray:
    """A_e = sum_{a,b in r,s,t} D_a^T diag(G_ab) D_b as a dense n^3 x n^3 matrix,
    with D_r = I (x) I (x) D, D_s = I (x) D (x) I, D_t = D (x) I (x) I acting on
    the flat node index (k*n + j)*n + i.  G_e is [6,n,n,n] in the component
    order (rr, rs, rt, ss, st, tt)."""
    D, G_e = _f64(D), _f64(G_e)
    n = D.shape[0]
    I = np.eye(n)
    Dd = [np.kron(I, np.kron(I, D)), np.kron(I, np.kron(D, I)), np.kron(D, np.kron(I, I))]
    comp = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (1, 1): 3, (1, 2): 4, (2, 2): 5}
    A = np.zeros((n ** 3, n ** 3))
    for a in range(3):
        for b in range(3):
            g = G_e[comp[(min(a, b), max(a, b))]].reshape(-1)
            A += Dd[a].T @ (g[:, None] * Dd[b])
    return A


def reduce(a, b) -> tuple[float, float, float]:
    """(max|a-b|, max|b|, sum a*b) over all entries, in float64."""
    a = _f64(a).ravel()
    b = _f64(b).ravel()
    if a.size == 0:
        return 0.0, 0.0, 0.0
    return float(np.max(np.abs(a - b))), float(np.max(np.abs(b))), float(np.dot(a, b))
