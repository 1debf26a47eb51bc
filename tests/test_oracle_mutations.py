"""Plant plausible mistakes in a copy of the C oracle (on the CPU) and check
that the pins catch each one: a dropped term, a wrong sign, a wrong index and
a transposed operand.  The planted copy is compiled to a temporary directory;
the committed oracle is never touched."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import sem_inputs as si

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "sem_ax_oracle.c")

MUTATIONS = {
    "gradient uses D^T along r": ("a += D[i * n + l] * u[(k * n + j) * n + l];",
                                  "a += D[l * n + i] * u[(k * n + j) * n + l];"),
    "wrong index along s": ("b += D[j * n + l] * u[(k * n + l) * n + i];",
                            "b += D[j * n + l] * u[(l * n + k) * n + i];"),
    "dropped cross term rs": ("ur[p] = Grr[p] * r + Grs[p] * s + Grt[p] * t;",
                              "ur[p] = Grr[p] * r + Grt[p] * t;"),
    "mis-signed cross term st": ("ut[p] = Grt[p] * r + Gst[p] * s + Gtt[p] * t;",
                                 "ut[p] = Grt[p] * r - Gst[p] * s + Gtt[p] * t;"),
    "G component swap": ("us[p] = Grs[p] * r + Gss[p] * s + Gst[p] * t;",
                         "us[p] = Grt[p] * r + Gss[p] * s + Gst[p] * t;"),
    "transposed step uses D along t": ("acc += D[l * n + k] * ut[(l * n + j) * n + i];",
                                       "acc += D[k * n + l] * ut[(l * n + j) * n + i];"),
    "dropped t direction in transpose": ("for (int l = 0; l < n; ++l) acc += D[l * n + k] * ut[(l * n + j) * n + i];",
                                         ""),
}


def _compile(tmp_path, name, src):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                    "-o", str(so), str(c)], check=True)
    lib = ctypes.CDLL(str(so))
    lib.oracle_sem_ax.restype = ctypes.c_int
    lib.oracle_sem_ax.argtypes = [ctypes.c_int64, ctypes.c_int] + [ctypes.c_void_p] * 4 + [ctypes.c_int]
    return lib


def _run(lib, u, G, D):
    u, G, D = (np.ascontiguousarray(x, dtype=np.float64) for x in (u, G, D))
    w = np.empty_like(u)
    assert lib.oracle_sem_ax(u.shape[0], D.shape[0] - 1, u.ctypes.data, G.ctypes.data,
                             D.ctypes.data, w.ctypes.data, 1) >= 0
    return w


def _pins_pass(lib, oracle_mod):
    """The dense-Kronecker pin and the affine energy pin, as in test_oracle."""
    ok = True
    m = si.make_mesh(np.random.default_rng(5), 2, 3)
    w = _run(lib, m.u.numpy(), m.G.numpy(), m.D.numpy())
    for e in range(2):
        ref = oracle_mod.dense_element_matrix(m.D, m.G[e]) @ m.u[e].numpy().ravel()
        ok &= np.max(np.abs(w[e].ravel() - ref)) / np.max(np.abs(ref)) < 1e-13
    m = si.make_mesh(np.random.default_rng(7), 4, 3)
    u = m.u.numpy()
    v = np.random.default_rng(8).uniform(-1, 1, size=u.shape)
    Au, Av = _run(lib, u, m.G.numpy(), m.D.numpy()), _run(lib, v, m.G.numpy(), m.D.numpy())
    ok &= abs(np.dot(v.ravel(), Au.ravel()) - np.dot(u.ravel(), Av.ravel())) <= 1e-12 * np.linalg.norm(v) * np.linalg.norm(Au)
    return bool(ok)


def test_unmutated_copy_passes(tmp_path, oracle_mod):
    assert _pins_pass(_compile(tmp_path, "orig", open(SRC).read()), oracle_mod)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, oracle_mod, name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor not found"
    lib = _compile(tmp_path, "mut", src.replace(old, new))
    assert not _pins_pass(lib, oracle_mod)


def test_planted_helmholtz_mistake_is_caught(tmp_path, oracle_mod):
    """The mass term applied to w instead of u, or with h1 and h2 swapped,
    fails the dense Helmholtz pin."""
    src = open(SRC).read()
    anchor = "w[p] = h1 * w[p] + h2 * B[p] * u[p];"
    assert src.count(anchor) == 1
    m = si.make_mesh(np.random.default_rng(46), 2, 3)
    B = si.mass_diagonal(m.X, 3).numpy()
    for idx, bad in enumerate(("w[p] = h1 * w[p] + h2 * B[p] * w[p];", "w[p] = h2 * w[p] + h1 * B[p] * u[p];")):
        lib = _compile(tmp_path, f"helm{idx}", src.replace(anchor, bad))
        lib.oracle_sem_helmholtz.restype = ctypes.c_int
        lib.oracle_sem_helmholtz.argtypes = ([ctypes.c_int64, ctypes.c_int] + [ctypes.c_void_p] * 4 +
                                             [ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_int])
        u, G, D = (np.ascontiguousarray(x.numpy()) for x in (m.u, m.G, m.D))
        w = np.empty_like(u)
        lib.oracle_sem_helmholtz(2, 3, u.ctypes.data, G.ctypes.data, B.ctypes.data, D.ctypes.data,
                                 0.75, 3.5, w.ctypes.data, 1)
        H = 0.75 * oracle_mod.dense_element_matrix(m.D, m.G[0]) + 3.5 * np.diag(B[0].ravel())
        ref = H @ u[0].ravel()
        assert np.max(np.abs(w[0].ravel() - ref)) / np.max(np.abs(ref)) > 1e-6
