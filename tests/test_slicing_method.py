"""CPU check of the exact digit-slicing method behind the tensor-core
FP64-accurate form, independent of the GPU and of its arithmetic order.

The method, in exact arithmetic: each operand of a contraction (u, D, and
the intermediate [wr ws wt] = G grad u) is rounded to balanced digits
against one power-of-two scale per element (D: one for the matrix), the
digit products of the kept levels are summed exactly, and the levels are
combined.  The kernels use five base-1024 digits whose leading digit takes
one bit less, so that no digit exceeds 512 (FP16 operands, levels 0..4
kept); six base-256 digits (BF16 operands, levels 0..5) are the
alternative the first form used.  This test evaluates that model in float64 (rounding
each operand at the last digit and dropping the levels above the kept ones,
which is what the digits represent) and compares it with the FP64 oracle:
the model's error is the method's own error floor, which the GPU parity
tests' bound (2e-13 of ||w||_inf) must exceed.  One digit fewer in either
system must miss the FP64 requirement.
"""
import numpy as np
import pytest

import sem_inputs as si


def _scale(x, axis=None):
    """Smallest power of two strictly above max |x| (over axis)."""
    m = np.max(np.abs(x), axis=axis, keepdims=axis is not None)
    m = np.where(m > 0, m, 1.0)
    return 2.0 ** (np.floor(np.log2(m)) + 1)


def _expand(x, s, ndig, bits=8, head=0):
    """The ndig balanced base-2^bits digits of x / s as integer-valued
    arrays, the leading digit taking bits - head bits."""
    M = np.round(x / s * 2.0 ** (bits * ndig - head)).astype(np.int64)
    half, mask = 1 << (bits - 1), (1 << bits) - 1
    d = []
    for _ in range(ndig - 1):
        lo = ((M + half) & mask) - half
        d.append(lo)
        M = (M - lo) >> bits
    d.append(M)
    return d[::-1]   # most significant first


def _contract(Dd, sD, ud, su, ndig, path, bits=8, head=0):
    """sum_l D[.,l] u[..l..] from digit expansions with levels p + q <= ndig - 1."""
    out = 0.0
    for p in range(ndig):
        for q in range(ndig):
            if p + q > ndig - 1:
                continue
            w = 2.0 ** (-(bits * (p + q + 2) - 2 * head))
            out = out + np.einsum(path, Dd[p].astype(np.float64), ud[q].astype(np.float64)) * w
    return out * sD * su


def _slice_ax(u, G, D, ndig, bits=8, head=0):
    E = u.shape[0]
    kw = dict(bits=bits, head=head)
    sD = float(_scale(D))
    Dd = _expand(D, sD, ndig, **kw)
    su = _scale(u.reshape(E, -1), axis=1).reshape(E, 1, 1, 1)
    ud = _expand(u, su, ndig, **kw)
    ur = _contract(Dd, sD, ud, su, ndig, "il,ekjl->ekji", **kw)
    us = _contract(Dd, sD, ud, su, ndig, "jl,ekli->ekji", **kw)
    ut = _contract(Dd, sD, ud, su, ndig, "kl,elji->ekji", **kw)
    g = [G[:, a] for a in range(6)]
    wr = g[0] * ur + g[1] * us + g[2] * ut
    ws = g[1] * ur + g[3] * us + g[4] * ut
    wt = g[2] * ur + g[4] * us + g[5] * ut
    sw = np.maximum(np.maximum(_scale(wr.reshape(E, -1), axis=1), _scale(ws.reshape(E, -1), axis=1)),
                    _scale(wt.reshape(E, -1), axis=1)).reshape(E, 1, 1, 1)
    xr, xs, xt = (_expand(a, sw, ndig, **kw) for a in (wr, ws, wt))
    return (_contract(Dd, sD, xr, sw, ndig, "li,ekjl->ekji", **kw)
            + _contract(Dd, sD, xs, sw, ndig, "lj,ekli->ekji", **kw)
            + _contract(Dd, sD, xt, sw, ndig, "lk,elji->ekji", **kw))


def _rel(w, ref):
    return float(np.max(np.abs(w - ref)) / np.max(np.abs(ref)))


@pytest.fixture(scope="module")
def mesh():
    return si.make_mesh(np.random.default_rng(90), 12, 7)


@pytest.fixture(scope="module")
def mesh16():
    return si.make_mesh(np.random.default_rng(91), 2, 15)


B10 = dict(bits=10, head=1)   # the kernels' digit system


def test_digit_expansion_is_balanced_and_exact(mesh, mesh16):
    for m in (mesh, mesh16):
        u = m.u.numpy()
        s = _scale(u)
        d = _expand(u, s, 5, **B10)
        assert all(np.abs(x).max() <= 512 for x in d)
        val = sum(x.astype(np.float64) * 2.0 ** -(10 * (k + 1) - 1) for k, x in enumerate(d)) * s
        assert np.max(np.abs(val - u)) <= 2.0 ** -50 * s


def test_level_sums_fit_the_fp32_significand(mesh, mesh16):
    """Order 7 (K = 8): every level sums at most five digit pairs of
    magnitude <= 512 x 512, below 2^24, so all five FP32 accumulators are
    exact.  Order 15 (K = 16): levels 0..2 (at most three pairs) are."""
    for m, levels in ((mesh, 5), (mesh16, 3)):
        D = m.D.numpy()
        u = m.u.numpy()
        Dd, ud = _expand(D, float(_scale(D)), 5, **B10), _expand(u, _scale(u), 5, **B10)
        for L in range(levels):
            acc = 0
            for p in range(L + 1):
                acc = acc + np.einsum("il,ekjl->ekji", np.abs(Dd[p]), np.abs(ud[L - p]))
            assert acc.max() < 2 ** 24


@pytest.mark.parametrize("which", ["mesh", "mesh16"])
def test_five_digits_meet_the_fp64_bound_and_four_do_not(oracle_mod, request, which):
    m = request.getfixturevalue(which)
    u, G, D = m.u.numpy(), m.G.numpy(), m.D.numpy()
    ref = oracle_mod.sem_ax(u, G, D)
    e5 = _rel(_slice_ax(u, G, D, 5, **B10), ref)
    e4 = _rel(_slice_ax(u, G, D, 4, **B10), ref)
    assert e5 <= 2e-13          # the GPU tests' typical bound sits above the method's floor
    assert e4 > 1e-12           # one digit fewer misses the FP64 requirement


def test_base256_system_needs_six_digits(oracle_mod, mesh):
    """The BF16 alternative (base-256 digits, no headroom bit): six digits
    reach the same floor, five do not."""
    u, G, D = mesh.u.numpy(), mesh.G.numpy(), mesh.D.numpy()
    ref = oracle_mod.sem_ax(u, G, D)
    assert _rel(_slice_ax(u, G, D, 6), ref) <= 2e-13
    assert _rel(_slice_ax(u, G, D, 5), ref) > 1e-12


def test_constant_field_floor(oracle_mod, mesh):
    """A 1 = 0 up to the five-digit truncation of D's rows (~1e-13 of ||A u||)."""
    u1 = np.full(mesh.u.shape, 3.25)
    w1 = _slice_ax(u1, mesh.G.numpy(), mesh.D.numpy(), 5, **B10)
    wr = oracle_mod.sem_ax(mesh.u.numpy(), mesh.G.numpy(), mesh.D.numpy())
    assert np.max(np.abs(w1)) <= 1e-12 * np.max(np.abs(wr))
