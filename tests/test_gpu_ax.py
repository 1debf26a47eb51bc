"""GPU parity of the plain Ax forms against the FP64 CPU oracle, through the
C ABI (via the ctypes binding).

Error measure: ||w - w_ref||_inf / ||w_ref||_inf over the whole output.
Tolerances: FP64 1e-12 (the requirement); FP32 compute 1e-5; BF16 splits:
terms=6 1e-5, terms=3 5e-5 (its products keep ~16 significant bits, unit
error 2^-16 ~ 1.5e-5 before accumulation).
"""
import numpy as np
import pytest
import torch

import sem_inputs as si

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-12
TOL_F32 = 1e-5
TOL_BF16 = {6: 1e-5, 3: 5e-5}


@pytest.fixture(scope="module")
def semax():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_07659_gb300 as m
    return m


def rel_err(w, ref):
    w = w.detach().cpu().double().numpy() if hasattr(w, "detach") else w
    return float(np.max(np.abs(w - ref)) / np.max(np.abs(ref)))


def to_dev(mesh, dtype=torch.float64):
    return (mesh.u.to("cuda", dtype), mesh.G.to("cuda", dtype), mesh.D.to("cuda", dtype))


# ---------------------------------------------------------------- FP64

def test_f64_small_workload_full(semax, oracle_mod):
    m = si.make_workload(0)[0]                       # N=7, E=512
    ref = oracle_mod.sem_ax(m.u, m.G, m.D)
    u, G, D = to_dev(m)
    w = semax.sem_ax(u, G, D)
    torch.cuda.synchronize()
    assert rel_err(w, ref) <= TOL_F64


@pytest.mark.parametrize("N", list(range(1, 16)))
@pytest.mark.parametrize("E", [1, 5, 37])
def test_f64_every_order_ragged(semax, oracle_mod, N, E):
    m = si.make_mesh(np.random.default_rng(100 + N), E, N)
    ref = oracle_mod.sem_ax(m.u, m.G, m.D)
    u, G, D = to_dev(m)
    w = semax.sem_ax(u, G, D)
    torch.cuda.synchronize()
    assert rel_err(w, ref) <= TOL_F64


def test_f64_full_size_sampled(semax, oracle_mod):
    """N=7, E=32768 (the 1.07 GB workload) in the benchmark's launch; the
    oracle checks a seeded 2% sample of elements (Ax is element-local, so a
    sampled element's output is exact to check)."""
    m = si.make_workload(1, device="cuda")[0]
    w = semax.sem_ax(m.u, m.G, m.D)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(11).choice(m.E, size=m.E // 50, replace=False))
    it = torch.from_numpy(idx).cuda()
    ref = oracle_mod.sem_ax(m.u[it].cpu(), m.G[it].cpu(), m.D.cpu())
    assert rel_err(w[it], ref) <= TOL_F64
    assert torch.isfinite(w).all()


@pytest.mark.parametrize("N", [3, 7, 15])
def test_f64_general_D_takes_the_generic_path(semax, oracle_mod, N):
    """A D that is not centro-antisymmetric (any caller's matrix) must still
    give the exact operator: the even/odd tile falls back per CTA."""
    m = si.make_mesh(np.random.default_rng(400 + N), 9, N)
    D = m.D.clone()
    D[0, 1] += 0.125
    ref = oracle_mod.sem_ax(m.u, m.G, D)
    u, G, Dd = m.u.cuda(), m.G.cuda(), D.cuda()
    w = semax.sem_ax(u, G, Dd)
    w32 = semax.sem_ax_f32(u.float(), G.float(), Dd.float())
    torch.cuda.synchronize()
    assert rel_err(w, ref) <= TOL_F64
    assert rel_err(w32, ref) <= TOL_F32


def test_pinned_host_arrays_stream_over_the_link(semax, oracle_mod):
    """u, G, D and w in pinned host memory: the kernel reads and writes them
    in place (coherent host access), bit-identical to device-resident arrays."""
    m = si.make_mesh(np.random.default_rng(77), 33, 7)
    u_h, G_h, D_h = m.u.pin_memory(), m.G.pin_memory(), m.D.pin_memory()
    w_h = torch.full_like(u_h, float("nan")).pin_memory()
    semax.sem_ax(u_h, G_h, D_h, w_h)
    w_d = semax.sem_ax(u_h.cuda(), G_h.cuda(), D_h.cuda())
    torch.cuda.synchronize()
    assert torch.equal(w_h, w_d.cpu())
    assert rel_err(w_h, oracle_mod.sem_ax(m.u, m.G, m.D)) <= TOL_F64
    w32 = torch.empty_like(u_h, dtype=torch.float32).pin_memory()
    semax.sem_ax_f32(u_h.float().pin_memory(), G_h.float().pin_memory(), D_h.float().pin_memory(), w32)
    torch.cuda.synchronize()
    assert torch.equal(w32, semax.sem_ax_f32(u_h.float().cuda(), G_h.float().cuda(), D_h.float().cuda()).cpu())


def test_f64_empty_and_guard_band(semax, oracle_mod):
    m = si.make_mesh(np.random.default_rng(3), 7, 5)
    u, G, D = to_dev(m)
    n3 = 6 ** 3
    buf = torch.full((7 * n3 + 2 * 64,), float("nan"), dtype=torch.float64, device="cuda")
    w = buf[64:64 + 7 * n3].view(7, 6, 6, 6)
    semax.sem_ax(u, G, D, w)
    semax.sem_ax(u[:0], G[:0], D, buf[:0].view(0, 6, 6, 6))     # E = 0 is a no-op
    torch.cuda.synchronize()
    assert torch.isnan(buf[:64]).all() and torch.isnan(buf[64 + 7 * n3:]).all()
    assert rel_err(w, oracle_mod.sem_ax(m.u, m.G, m.D)) <= TOL_F64


def test_f64_invariants_on_gpu(semax):
    """A.1 = 0 and symmetry v.Au = u.Av, with the FP64 reducer."""
    m = si.make_mesh(np.random.default_rng(9), 64, 7, device="cuda")
    v = torch.rand_like(m.u) * 2 - 1
    one = torch.ones_like(m.u)
    Au, Av, A1 = (semax.sem_ax(x, m.G, m.D) for x in (m.u, v, one))
    r = semax.reduce(v, Au).cpu().numpy()
    s = semax.reduce(m.u, Av).cpu().numpy()
    z = semax.reduce(A1, torch.zeros_like(A1)).cpu().numpy()
    assert abs(r[2] - s[2]) <= 1e-12 * torch.linalg.norm(v).item() * torch.linalg.norm(Au).item()
    assert z[0] <= 1e-12 * semax.reduce(Au, torch.zeros_like(Au)).cpu().numpy()[0]
    assert semax.reduce(m.u, Au).cpu().numpy()[2] > 0


# ---------------------------------------------------------------- Helmholtz form

@pytest.mark.parametrize("N", [1, 2, 3, 4, 7, 8, 15])
@pytest.mark.parametrize("E", [1, 19])
def test_helmholtz_against_oracle(semax, oracle_mod, N, E):
    m = si.make_mesh(np.random.default_rng(600 + N), E, N)
    B = si.mass_diagonal(m.X, N)
    h1, h2 = 0.625, 7.25
    ref = oracle_mod.sem_helmholtz(m.u, m.G, B, m.D, h1, h2)
    u, G, D = to_dev(m)
    w = semax.sem_ax_helmholtz(u, G, B.cuda(), D, h1, h2)
    torch.cuda.synchronize()
    assert rel_err(w, ref) <= TOL_F64


def test_helmholtz_reduces_to_ax_and_mass(semax):
    m = si.make_mesh(np.random.default_rng(610), 40, 7, device="cuda")
    B = si.mass_diagonal(m.X, 7, device="cuda")
    w_ax = semax.sem_ax(m.u, m.G, m.D)
    w_h = semax.sem_ax_helmholtz(m.u, m.G, B, m.D, 1.0, 0.0)
    w_m = semax.sem_ax_helmholtz(torch.ones_like(m.u), m.G, B, m.D, 3.0, 2.0)
    torch.cuda.synchronize()
    assert torch.equal(w_ax, w_h)
    assert (w_m - 2.0 * B).abs().max().item() <= 1e-12 * B.abs().max().item()


def test_helmholtz_full_size_sampled(semax, oracle_mod):
    m = si.make_workload(1, device="cuda")[0]
    B = si.mass_diagonal(m.X, m.N, device="cuda")
    w = semax.sem_ax_helmholtz(m.u, m.G, B, m.D, 1.0, 0.1)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(17).choice(m.E, size=m.E // 50, replace=False))
    it = torch.from_numpy(idx).cuda()
    ref = oracle_mod.sem_helmholtz(m.u[it].cpu(), m.G[it].cpu(), B[it].cpu(), m.D.cpu(), 1.0, 0.1)
    assert rel_err(w[it], ref) <= TOL_F64


@pytest.mark.parametrize("N,E", [(7, 1), (7, 37), (7, 3000), (15, 1), (15, 40), (5, 20)])
def test_helmholtz_f64tc_against_oracle(semax, oracle_mod, N, E):
    """A u on tensor cores (N = 7 and 15; the FP64 form otherwise), the mass term in FP64."""
    m = si.make_mesh(np.random.default_rng(620 + N + E), E, N)
    B = si.mass_diagonal(m.X, N)
    h1, h2 = 0.625, 7.25
    ref = oracle_mod.sem_helmholtz(m.u, m.G, B, m.D, h1, h2)
    u, G, D = to_dev(m)
    w = semax.sem_ax_helmholtz_f64tc(u, G, B.cuda(), D, h1, h2)
    torch.cuda.synchronize()
    assert rel_err(w, ref) <= TOL_F64


@pytest.mark.parametrize("N", [7, 15])
def test_helmholtz_f64tc_reduces_to_f64tc_and_mass(semax, N):
    m = si.make_mesh(np.random.default_rng(630 + N), 40, N, device="cuda")
    B = si.mass_diagonal(m.X, N, device="cuda")
    w_ax = semax.sem_ax_f64tc(m.u, m.G, m.D)
    w_h = semax.sem_ax_helmholtz_f64tc(m.u, m.G, B, m.D, 1.0, 0.0)
    one = torch.ones_like(m.u)
    w_1 = semax.sem_ax_f64tc(one, m.G, m.D)
    w_m = semax.sem_ax_helmholtz_f64tc(one, m.G, B, m.D, 3.0, 2.0)
    w_b = semax.sem_ax_helmholtz_f64tc(one, m.G, B, m.D, 0.0, 2.0)
    torch.cuda.synchronize()
    assert torch.equal(w_ax, w_h)                  # h1 = 1, h2 = 0: the tensor-core Ax bit for bit
    assert torch.equal(w_b, 2.0 * B)               # h1 = 0: the mass term alone, exact
    # one fused multiply-add per node: h2 B u + h1 (A u) with a single rounding, and here
    # h2 B u = 2 B is exact, so it equals the two-step sum bit for bit
    assert torch.equal(w_m, 3.0 * w_1 + 2.0 * B)
    # A annihilates constants (D applied to a constant is zero): what is left is rounding
    assert w_1.abs().max().item() <= 1e-12 * semax.sem_ax_f64tc(m.u, m.G, m.D).abs().max().item()


@pytest.mark.parametrize("wl", [1, 2])   # N = 7, E = 32768 and N = 15, E = 8192
def test_helmholtz_f64tc_full_size_sampled(semax, oracle_mod, wl):
    m = si.make_workload(wl, device="cuda")[0]
    B = si.mass_diagonal(m.X, m.N, device="cuda")
    w = semax.sem_ax_helmholtz_f64tc(m.u, m.G, B, m.D, 1.0, 0.1)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(18).choice(m.E, size=m.E // 50, replace=False))
    it = torch.from_numpy(idx).cuda()
    ref = oracle_mod.sem_helmholtz(m.u[it].cpu(), m.G[it].cpu(), B[it].cpu(), m.D.cpu(), 1.0, 0.1)
    assert rel_err(w[it], ref) <= TOL_F64


# ---------------------------------------------------------------- FP64-accurate double-float form

@pytest.mark.parametrize("N", list(range(1, 16)))
@pytest.mark.parametrize("E", [1, 6, 37])
def test_f64x_every_order_ragged(semax, oracle_mod, N, E):
    m = si.make_mesh(np.random.default_rng(500 + N), E, N)
    ref = oracle_mod.sem_ax(m.u, m.G, m.D)
    u, G, D = to_dev(m)
    w = semax.sem_ax_f64x(u, G, D)
    torch.cuda.synchronize()
    assert rel_err(w, ref) <= TOL_F64


def test_f64x_full_size_sampled(semax, oracle_mod):
    m = si.make_workload(1, device="cuda")[0]
    w = semax.sem_ax_f64x(m.u, m.G, m.D)
    w64 = semax.sem_ax(m.u, m.G, m.D)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(14).choice(m.E, size=m.E // 50, replace=False))
    it = torch.from_numpy(idx).cuda()
    ref = oracle_mod.sem_ax(m.u[it].cpu(), m.G[it].cpu(), m.D.cpu())
    assert rel_err(w[it], ref) <= TOL_F64
    r = semax.reduce(w, w64).cpu().numpy()
    assert r[0] / r[1] <= TOL_F64                      # whole output against the FP64 kernel


@pytest.mark.parametrize("scale", [1e-30, 1e-3, 1.0, 1e30])
def test_f64x_is_scale_invariant(semax, oracle_mod, scale):
    """Per-element power-of-two scaling keeps the double-float form accurate
    for inputs far outside the float range's comfortable middle."""
    m = si.make_mesh(np.random.default_rng(15), 12, 7)
    u = m.u * scale
    ref = oracle_mod.sem_ax(u, m.G, m.D)
    w = semax.sem_ax_f64x(u.cuda(), m.G.cuda(), m.D.cuda())
    torch.cuda.synchronize()
    assert rel_err(w, ref) <= TOL_F64


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_nonfinite_input_stays_in_its_element(semax, oracle_mod, bad):
    """A NaN or Inf in one element's u makes that element's output non-finite
    (as in the definition) and leaves every other element exact, in the FP64,
    double-float and FP32 forms."""
    m = si.make_mesh(np.random.default_rng(20), 6, 7)
    u = m.u.clone()
    u[3, 2, 5, 1] = bad
    ref = oracle_mod.sem_ax(np.delete(u.numpy(), 3, 0), np.delete(m.G.numpy(), 3, 0), m.D)
    for fn, dt, tol in ((semax.sem_ax, torch.float64, TOL_F64), (semax.sem_ax_f64x, torch.float64, TOL_F64),
                        (semax.sem_ax_f32, torch.float32, TOL_F32)):
        w = fn(u.to("cuda", dt), m.G.to("cuda", dt), m.D.to("cuda", dt))
        torch.cuda.synchronize()
        wc = w.double().cpu().numpy()
        assert not np.isfinite(wc[3]).all()
        assert rel_err(np.delete(wc, 3, 0), ref) <= tol


def test_f64x_general_D_falls_back(semax, oracle_mod):
    m = si.make_mesh(np.random.default_rng(16), 5, 7)
    D = m.D.clone()
    D[2, 3] += 0.25
    ref = oracle_mod.sem_ax(m.u, m.G, D)
    w = semax.sem_ax_f64x(m.u.cuda(), m.G.cuda(), D.cuda())
    torch.cuda.synchronize()
    assert rel_err(w, ref) <= TOL_F64


# ---------------------------------------------------------------- FP32

@pytest.mark.parametrize("N,E", [(7, 300), (15, 20), (3, 77), (10, 9)])
def test_f32_against_f64_oracle(semax, oracle_mod, N, E):
    m = si.make_mesh(np.random.default_rng(200 + N), E, N)
    ref = oracle_mod.sem_ax(m.u, m.G, m.D)
    u, G, D = to_dev(m, torch.float32)
    w = semax.sem_ax_f32(u, G, D)
    torch.cuda.synchronize()
    assert rel_err(w, ref) <= TOL_F32


@pytest.mark.parametrize("E", [1, 5, 37, 1000, 5000])
def test_f32_order7_against_oracle(semax, oracle_mod, E):
    """Order 7 in FP32: ragged counts, more elements than one wave of CTAs,
    and a general D that is not centro-antisymmetric (the generic tile)."""
    m = si.make_mesh(np.random.default_rng(1400 + E), E, 7)
    ref = oracle_mod.sem_ax(m.u, m.G, m.D)
    u, G, D = to_dev(m, torch.float32)
    w = semax.sem_ax_f32(u, G, D)
    torch.cuda.synchronize()
    assert rel_err(w, ref) <= TOL_F32
    Dg = m.D + 0.05 * torch.from_numpy(np.random.default_rng(1401).standard_normal((8, 8)))
    refg = oracle_mod.sem_ax(m.u, m.G, Dg)
    wg = semax.sem_ax_f32(u, G, Dg.float().cuda())
    torch.cuda.synchronize()
    assert rel_err(wg, refg) <= TOL_F32


def test_f32_power_of_two_scale_is_exact(semax):
    m = si.make_mesh(np.random.default_rng(5), 40, 7, device="cuda")
    u, G, D = (x.float() for x in (m.u, m.G, m.D))
    s = si.per_element_g_scale(G).float()
    w0 = semax.sem_ax_f32(u, G, D)
    w1 = semax.sem_ax_f32(u, (G / s.view(-1, 1, 1, 1, 1)).contiguous(), D, G_scale=s)
    torch.cuda.synchronize()
    assert torch.equal(w0, w1)


# ---------------------------------------------------------------- BF16 splits on tensor cores

@pytest.mark.parametrize("terms", [3, 6])
@pytest.mark.parametrize("E", [1, 7, 300])
def test_bf16_split_against_f64_oracle(semax, oracle_mod, terms, E):
    m = si.make_mesh(np.random.default_rng(300 + E), E, 15)
    ref = oracle_mod.sem_ax(m.u, m.G, m.D)
    u, G, D = to_dev(m, torch.float32)
    w = semax.sem_ax_bf16x3(u, G, D, terms=terms)
    torch.cuda.synchronize()
    err = rel_err(w, ref)
    assert err <= TOL_BF16[terms], err


@pytest.mark.parametrize("terms", [3, 6])
def test_bf16_split_scaled_matches_unscaled(semax, terms):
    m = si.make_mesh(np.random.default_rng(8), 33, 15, device="cuda")
    u, G, D = (x.float() for x in (m.u, m.G, m.D))
    s = si.per_element_g_scale(G).float()
    w0 = semax.sem_ax_bf16x3(u, G, D, terms=terms)
    w1 = semax.sem_ax_bf16x3(u, (G / s.view(-1, 1, 1, 1, 1)).contiguous(), D, G_scale=s, terms=terms)
    torch.cuda.synchronize()
    assert torch.equal(w0, w1)


# ---------------------------------------------------------------- FP16 splits (3 products) on tensor cores
#
# Tolerance: two FP16 pieces keep ~22 bits of each scaled operand (x - x0 -
# x1 <= 2^-22 |x|, and 2^-25 of the group's largest absolute below FP16's
# normal range), the dropped product x1 y1 weighs <= 2^-22, and the FP32
# accumulation and the FP32 geometric-factor multiply add ~2^-24 per step:
# about 1e-6 of ||w||_inf after the cancellation of the Laplacian's terms.
# The test holds it to TOL_F16 = 1e-5 (the bar the split forms are held to)
# and the typical error to 3e-6.

TOL_F16, TYPICAL_F16 = 1e-5, 3e-6


@pytest.mark.parametrize("N,E", [(15, 1), (15, 7), (15, 300), (7, 1), (7, 37), (7, 5000)])
def test_f16_split_against_f64_oracle(semax, oracle_mod, N, E):
    m = si.make_mesh(np.random.default_rng(1300 + E + N), E, N)
    ref = oracle_mod.sem_ax(m.u, m.G, m.D)
    u, G, D = to_dev(m, torch.float32)
    w = semax.sem_ax_f16x3(u, G, D)
    torch.cuda.synchronize()
    err = rel_err(w, ref)
    assert err <= TOL_F16 and err <= TYPICAL_F16, err


@pytest.mark.parametrize("N", [7, 15])
@pytest.mark.parametrize("us,gs", [(2.0 ** 40, 1.0), (2.0 ** -50, 1.0), (1.0, 2.0 ** 30), (2.0 ** -20, 2.0 ** -25)])
def test_f16_split_is_scale_invariant(semax, N, us, gs):
    """Power-of-two scales of u and G scale the result exactly: the operands
    are rescaled to [1, 2) before the FP16 split, so the pieces are the same."""
    m = si.make_mesh(np.random.default_rng(1350), 9, N, device="cuda")
    u, G, D = (x.float() for x in (m.u, m.G, m.D))
    w0 = semax.sem_ax_f16x3(u, G, D)
    w1 = semax.sem_ax_f16x3((u * us).contiguous(), (G * gs).contiguous(), D)
    torch.cuda.synchronize()
    assert torch.equal(w1, w0 * (us * gs))


@pytest.mark.parametrize("N", [7, 15])
def test_f16_split_zero_and_scaled_g(semax, oracle_mod, N):
    """An all-zero element, an element with zero u in one plane, and the
    per-element G scale give the unscaled result bit for bit."""
    m = si.make_mesh(np.random.default_rng(1360), 11, N)
    u = m.u.clone()
    u[2] = 0.0
    u[4, 7] = 0.0
    ref = oracle_mod.sem_ax(u, m.G, m.D)
    ud, G, D = u.float().cuda(), m.G.float().cuda(), m.D.float().cuda()
    w0 = semax.sem_ax_f16x3(ud, G, D)
    s = si.per_element_g_scale(G).float()
    w1 = semax.sem_ax_f16x3(ud, (G / s.view(-1, 1, 1, 1, 1)).contiguous(), D, G_scale=s)
    torch.cuda.synchronize()
    assert torch.equal(w0, w1)
    assert bool((w0[2] == 0).all())
    assert rel_err(w0, ref) <= TYPICAL_F16


def test_f16_split_general_d_order7(semax, oracle_mod):
    """The order-7 form takes any D (no symmetry is used)."""
    m = si.make_mesh(np.random.default_rng(1365), 40, 7)
    Dg = m.D + 0.05 * torch.from_numpy(np.random.default_rng(1366).standard_normal((8, 8)))
    ref = oracle_mod.sem_ax(m.u, m.G, Dg)
    w = semax.sem_ax_f16x3(m.u.float().cuda(), m.G.float().cuda(), Dg.float().cuda())
    torch.cuda.synchronize()
    assert rel_err(w, ref) <= TOL_F16


def test_f16_split_rejects_other_orders(semax):
    m = si.make_mesh(np.random.default_rng(1370), 2, 5, device="cuda")
    with pytest.raises(semax.SemaxError):
        semax.sem_ax_f16x3(m.u.float(), m.G.float(), m.D.float())


def _geo_inputs(m):
    X = torch.from_numpy(m.X).float().cuda().contiguous()
    xq = torch.cat([torch.from_numpy(si.gll_nodes(m.N)), torch.from_numpy(si.gll_weights(m.N))]).float().cuda()
    return X, xq


@pytest.mark.parametrize("terms", [3, 6])
@pytest.mark.parametrize("E", [1, 5, 130])
def test_bf16_geo_against_f64_oracle(semax, oracle_mod, terms, E):
    """G recomputed from FP32 vertices inside the kernel; the oracle uses the
    FP64 G of the same (FP64) vertices."""
    m = si.make_mesh(np.random.default_rng(800 + E), E, 15)
    ref = oracle_mod.sem_ax(m.u, m.G, m.D)
    X, xq = _geo_inputs(m)
    w = semax.sem_ax_bf16x3_geo(m.u.float().cuda(), X, xq, m.D.float().cuda(), terms=terms)
    torch.cuda.synchronize()
    err = rel_err(w, ref)
    assert err <= TOL_BF16[terms], err


def test_bf16_geo_matches_stored_g_form(semax):
    """Recomputed and stored (FP32-rounded) geometric factors agree to FP32
    rounding, so the two forms agree far inside the BF16 split's error."""
    m = si.make_mesh(np.random.default_rng(810), 64, 15, device="cuda")
    X, xq = _geo_inputs(m)
    u, D = m.u.float(), m.D.float()
    a = semax.sem_ax_bf16x3_geo(u, X, xq, D, terms=6)
    b = semax.sem_ax_bf16x3(u, m.G.float(), D, terms=6)
    torch.cuda.synchronize()
    assert ((a - b).abs().max() / b.abs().max()).item() <= 2e-6


def test_bf16_rejects_other_orders(semax):
    m = si.make_mesh(np.random.default_rng(1), 2, 7, device="cuda")
    with pytest.raises(semax.SemaxError, match="UNSUPPORTED_N"):
        semax.sem_ax_bf16x3(m.u.float(), m.G.float(), m.D.float())


def test_mixed_full_size_sampled(semax, oracle_mod):
    """N=15, E=8192 in FP32 and both BF16 variants, checked on a 1% sample
    with the oracle on the FP64 originals; FP64 residual on the GPU too."""
    m = si.make_workload(2, device="cuda")[0]
    u, G, D = (x.float() for x in (m.u, m.G, m.D))
    idx = np.sort(np.random.default_rng(12).choice(m.E, size=82, replace=False))
    it = torch.from_numpy(idx).cuda()
    ref = oracle_mod.sem_ax(m.u[it].cpu(), m.G[it].cpu(), m.D.cpu())
    ref_t = torch.from_numpy(ref).cuda()
    for name, fn, tol in [("f32", lambda: semax.sem_ax_f32(u, G, D), TOL_F32),
                          ("bf16x3", lambda: semax.sem_ax_bf16x3(u, G, D, terms=3), TOL_BF16[3]),
                          ("bf16x6", lambda: semax.sem_ax_bf16x3(u, G, D, terms=6), TOL_BF16[6])]:
        w = fn()
        torch.cuda.synchronize()
        assert rel_err(w[it], ref) <= tol, name
        red = semax.reduce(w[it].contiguous(), ref_t).cpu().numpy()
        assert abs(red[0] / red[1] - rel_err(w[it], ref)) <= 1e-12, name


# ---------------------------------------------------------------- maximum sizes

@pytest.fixture(scope="module")
def big_n16():
    """E = 140000 elements of order 15 (573M nodes): G's element offsets pass
    2^31 values (e * 6 * 4096 > 2^31 from e = 87382 on).  Built by tiling a
    64-element seeded mesh, u from a seeded generator."""
    base = si.make_mesh(np.random.default_rng(900), 64, 15, device="cuda")
    E = 140000
    reps = (E + 63) // 64
    G = base.G.repeat(reps, 1, 1, 1, 1)[:E].contiguous()
    gen = torch.Generator(device="cuda").manual_seed(901)
    u = torch.rand((E, 16, 16, 16), generator=gen, dtype=torch.float64, device="cuda") * 2 - 1
    return base, u, G


def _check_tail(w, u, base, oracle_mod, tol):
    E = u.shape[0]
    idx = np.array([0, 87381, 87382, 100000, E - 2, E - 1])
    it = torch.from_numpy(idx).cuda()
    Gs = base.G[it.remainder(64)].cpu()
    ref = oracle_mod.sem_ax(u[it].cpu(), Gs, base.D.cpu())
    got = w[it].double().cpu().numpy()
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= tol


def test_max_size_f64_and_f64x(semax, oracle_mod, big_n16):
    base, u, G = big_n16
    w = semax.sem_ax(u, G, base.D)
    torch.cuda.synchronize()
    _check_tail(w, u, base, oracle_mod, TOL_F64)
    semax.sem_ax_f64x(u, G, base.D, w)
    torch.cuda.synchronize()
    _check_tail(w, u, base, oracle_mod, TOL_F64)


def test_max_size_f32_and_bf16(semax, oracle_mod, big_n16):
    base, u64, G64 = big_n16
    u, G, D = u64.float(), G64.float(), base.D.float()
    w = semax.sem_ax_f32(u, G, D)
    torch.cuda.synchronize()
    _check_tail(w, u64, base, oracle_mod, TOL_F32)
    semax.sem_ax_bf16x3(u, G, D, w, terms=6)
    torch.cuda.synchronize()
    _check_tail(w, u64, base, oracle_mod, TOL_BF16[6])
