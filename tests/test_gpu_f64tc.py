"""GPU parity of the tensor-core FP64-accurate form (exact digit slicing on
FP16 tensor cores, sem_ax_f64tc) against the FP64 CPU oracle, through the C
ABI.

Error measure: ||w - w_ref||_inf / ||w_ref||_inf over the whole output.

Tolerance.  Each operand keeps 5 base-1024 digits (truncation 2^-50 of its
element's scale), the tensor-core level sums are exact (order 7; at order 15
the two lowest levels may round by a unit at weights 2^-30 and 2^-40), the
level sums and the geometric-factor multiply run in double-float (~2^-47 per
operation, G split to 47 bits), and the dropped digit levels weigh < 2^-48.
About ten such terms pass through two contractions with n-term sums (the
gradient's worst case is n max|D| max|u|), so the bound is of order
10 * 16 * 2^-47 ~ 1e-12 of the element's scale, and typically 1e-14 to
1e-13.  The test holds it to TOL_TC = 1e-12, the FP64 requirement; the
typical error is checked to stay below 2e-13.
"""
import numpy as np
import pytest
import torch

import sem_inputs as si

pytestmark = pytest.mark.gpu

TOL_TC = 1e-12
TYPICAL_TC = 2e-13


@pytest.fixture(scope="module")
def semax():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_07659_gb300 as m
    return m


def rel_err(w, ref):
    w = w.detach().cpu().double().numpy() if hasattr(w, "detach") else w
    return float(np.max(np.abs(w - ref)) / np.max(np.abs(ref)))


def run(semax, u, G, D):
    w = semax.sem_ax_f64tc(u.cuda(), G.cuda(), D.cuda())
    torch.cuda.synchronize()
    return w


@pytest.mark.parametrize("E", [1, 3, 77, 300])
def test_f64tc_ragged_against_oracle(semax, oracle_mod, E):
    m = si.make_mesh(np.random.default_rng(700 + E), E, 7)
    ref = oracle_mod.sem_ax(m.u, m.G, m.D)
    err = rel_err(run(semax, m.u, m.G, m.D), ref)
    assert err <= TOL_TC
    assert err <= TYPICAL_TC


def test_f64tc_integer_inputs_are_exact(semax, oracle_mod):
    """With small-integer u, G and D every digit product, level sum and
    double-float step is exact, so the result equals the exact (integer)
    FP64 value bit for bit.  This pins the exactness of the FP32
    accumulation inside the tensor-core products, on which the method rests."""
    rng = np.random.default_rng(71)
    E = 40
    u = torch.from_numpy(rng.integers(-100, 101, size=(E, 8, 8, 8)).astype(np.float64))
    G = torch.from_numpy(rng.integers(0, 17, size=(E, 6, 8, 8, 8)).astype(np.float64))
    D = torch.from_numpy(rng.integers(-8, 9, size=(8, 8)).astype(np.float64))
    ref = oracle_mod.sem_ax(u, G, D)
    w = run(semax, u, G, D).cpu().numpy()
    assert np.array_equal(w, ref)


def test_f64tc_full_size_sampled(semax, oracle_mod):
    m = si.make_workload(1, device="cuda")[0]
    w = semax.sem_ax_f64tc(m.u, m.G, m.D)
    w64 = semax.sem_ax(m.u, m.G, m.D)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(24).choice(m.E, size=m.E // 50, replace=False))
    it = torch.from_numpy(idx).cuda()
    ref = oracle_mod.sem_ax(m.u[it].cpu(), m.G[it].cpu(), m.D.cpu())
    assert rel_err(w[it], ref) <= TYPICAL_TC
    r = semax.reduce(w, w64).cpu().numpy()
    assert r[0] / r[1] <= TYPICAL_TC                   # whole output against the FP64 kernel


@pytest.mark.parametrize("us,gs", [(1e-300, 1.0), (1e30, 1e-30), (1.0, 1e250), (2.0 ** -1000, 2.0 ** 900)])
def test_f64tc_is_scale_invariant(semax, oracle_mod, us, gs):
    """u and G far outside the float range: the per-element scale of u and
    the per-node scale of G keep the result accurate."""
    m = si.make_mesh(np.random.default_rng(72), 9, 7)
    u, G = m.u * us, m.G * gs
    ref = oracle_mod.sem_ax(u, G, m.D)
    assert rel_err(run(semax, u, G, m.D), ref) <= TYPICAL_TC


def test_f64tc_general_D(semax, oracle_mod):
    """Any D works (no even/odd symmetry is used)."""
    m = si.make_mesh(np.random.default_rng(73), 11, 7)
    D = m.D.clone()
    D[2, 3] += 0.25
    D[5] *= 3.0
    ref = oracle_mod.sem_ax(m.u, m.G, D)
    assert rel_err(run(semax, m.u, m.G, D), ref) <= TYPICAL_TC


def test_f64tc_zero_and_constant_fields(semax):
    m = si.make_mesh(np.random.default_rng(74), 5, 7)
    w0 = run(semax, torch.zeros_like(m.u), m.G, m.D)
    assert torch.count_nonzero(w0).item() == 0
    w1 = run(semax, torch.full_like(m.u, 3.25), m.G, m.D)
    wr = run(semax, m.u, m.G, m.D)
    # A 1 = 0 up to the rounding of D's row sums
    assert w1.abs().max().item() <= 1e-12 * wr.abs().max().item()


def test_f64tc_zero_geometric_factor_nodes(semax, oracle_mod):
    """Nodes whose six G entries are all zero, and an element with G = 0:
    zero entries are split into zero, not into a value of the node's scale."""
    m = si.make_mesh(np.random.default_rng(78), 7, 7)
    G = m.G.clone()
    G[2, :, 3, 4, 5] = 0.0
    G[2, :, 0, 0, 0] = 0.0
    G[5] = 0.0
    ref = oracle_mod.sem_ax(m.u, G, m.D)
    w = run(semax, m.u, G, m.D)
    assert rel_err(w, ref) <= TYPICAL_TC
    assert torch.count_nonzero(w[5]).item() == 0


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
@pytest.mark.parametrize("where", ["u", "G"])
def test_f64tc_nonfinite_input_poisons_only_its_element(semax, oracle_mod, bad, where):
    m = si.make_mesh(np.random.default_rng(75), 6, 7)
    u, G = m.u.clone(), m.G.clone()
    if where == "u":
        u[3, 2, 5, 1] = bad
    else:
        G[3, 4, 1, 1, 6] = bad
    ref = oracle_mod.sem_ax(np.delete(u.numpy(), 3, 0), np.delete(G.numpy(), 3, 0), m.D)
    w = run(semax, u, G, m.D).cpu().numpy()
    assert np.isnan(w[3]).all()
    assert rel_err(np.delete(w, 3, 0), ref) <= TYPICAL_TC


@pytest.mark.parametrize("E", [1, 3, 20])
def test_f64tc_order15_against_oracle(semax, oracle_mod, E):
    m = si.make_mesh(np.random.default_rng(900 + E), E, 15)
    ref = oracle_mod.sem_ax(m.u, m.G, m.D)
    err = rel_err(run(semax, m.u, m.G, m.D), ref)
    assert err <= TYPICAL_TC


def test_f64tc_order15_integer_inputs_are_exact(semax, oracle_mod):
    rng = np.random.default_rng(91)
    E = 6
    u = torch.from_numpy(rng.integers(-100, 101, size=(E, 16, 16, 16)).astype(np.float64))
    G = torch.from_numpy(rng.integers(0, 17, size=(E, 6, 16, 16, 16)).astype(np.float64))
    D = torch.from_numpy(rng.integers(-8, 9, size=(16, 16)).astype(np.float64))
    ref = oracle_mod.sem_ax(u, G, D)
    w = run(semax, u, G, D).cpu().numpy()
    assert np.array_equal(w, ref)


def test_f64tc_order15_edge_inputs(semax, oracle_mod):
    """Scaled inputs, a general D, zero G nodes and elements, zero and
    constant fields, and a NaN that poisons only its element, at order 15."""
    m = si.make_mesh(np.random.default_rng(92), 5, 15)
    for us, gs in ((1e-300, 1.0), (1.0, 1e250), (2.0 ** -1000, 2.0 ** 900)):
        u, G = m.u * us, m.G * gs
        assert rel_err(run(semax, u, G, m.D), oracle_mod.sem_ax(u, G, m.D)) <= TYPICAL_TC
    D = m.D.clone()
    D[2, 3] += 0.25
    assert rel_err(run(semax, m.u, m.G, D), oracle_mod.sem_ax(m.u, m.G, D)) <= TYPICAL_TC
    G = m.G.clone()
    G[1, :, 3, 4, 5] = 0.0
    G[3] = 0.0
    w = run(semax, m.u, G, m.D)
    assert rel_err(w, oracle_mod.sem_ax(m.u, G, m.D)) <= TYPICAL_TC
    assert torch.count_nonzero(w[3]).item() == 0
    assert torch.count_nonzero(run(semax, torch.zeros_like(m.u), m.G, m.D)).item() == 0
    w1 = run(semax, torch.full_like(m.u, 3.25), m.G, m.D)
    assert w1.abs().max().item() <= 1e-12 * run(semax, m.u, m.G, m.D).abs().max().item()
    u = m.u.clone()
    u[2, 5, 1, 7] = float("nan")
    w = run(semax, u, m.G, m.D).cpu().numpy()
    assert np.isnan(w[2]).all()
    ref = oracle_mod.sem_ax(np.delete(u.numpy(), 2, 0), np.delete(m.G.numpy(), 2, 0), m.D)
    assert rel_err(np.delete(w, 2, 0), ref) <= TYPICAL_TC


def test_f64tc_order15_unbalanced_geometric_factor(semax, oracle_mod):
    """Nodes whose (ss, st, tt) and (rr, rs, rt) differ in scale by far more
    than the common-scale path takes (2^80, 2^-70, one group zero), in whole
    elements and in some nodes of an element: every element still matches
    the oracle to its own scale."""
    m = si.make_mesh(np.random.default_rng(94), 5, 15)
    G = m.G.clone()
    G[0, 3:] *= 2.0 ** 80                   # second half far above the first
    G[1, :3, ::2] *= 2.0 ** -70             # first half far below, in every other plane
    G[2, :3, :, 5] = 0.0                    # first half zero in one row of every plane
    G[3, 3:, 7, :, 2:9] = 0.0               # second half zero in part of a plane
    ref = oracle_mod.sem_ax(m.u, G, m.D)
    w = run(semax, m.u, G, m.D).cpu().numpy()
    for e in range(m.E):
        assert rel_err(w[e], ref[e]) <= TYPICAL_TC, e


def test_f64tc_order15_full_size_sampled(semax, oracle_mod):
    m = si.make_workload(2, device="cuda")[0]
    w = semax.sem_ax_f64tc(m.u, m.G, m.D)
    w64 = semax.sem_ax(m.u, m.G, m.D)
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(93).choice(m.E, size=m.E // 256, replace=False))
    it = torch.from_numpy(idx).cuda()
    ref = oracle_mod.sem_ax(m.u[it].cpu(), m.G[it].cpu(), m.D.cpu())
    assert rel_err(w[it], ref) <= TYPICAL_TC
    r = semax.reduce(w, w64).cpu().numpy()
    assert r[0] / r[1] <= TYPICAL_TC


@pytest.mark.parametrize("N,E", [(3, 20), (4, 9), (11, 3)])
def test_f64tc_other_orders_use_the_double_float_form(semax, oracle_mod, N, E):
    m = si.make_mesh(np.random.default_rng(760 + N), E, N)
    ref = oracle_mod.sem_ax(m.u, m.G, m.D)
    assert rel_err(run(semax, m.u, m.G, m.D), ref) <= TOL_TC


def test_f64tc_preserves_inputs_and_honours_stream(semax, oracle_mod):
    m = si.make_mesh(np.random.default_rng(77), 50, 7)
    u, G, D = m.u.cuda(), m.G.cuda(), m.D.cuda()
    u0, G0 = u.clone(), G.clone()
    s = torch.cuda.Stream()
    w = torch.empty_like(u)
    with torch.cuda.stream(s):
        semax.sem_ax_f64tc(u, G, D, w, stream=s)
    s.synchronize()
    assert torch.equal(u, u0) and torch.equal(G, G0)
    assert rel_err(w, oracle_mod.sem_ax(m.u, m.G, m.D)) <= TYPICAL_TC


def test_f64tc_max_size_offsets_past_2_31(semax, oracle_mod):
    """E = 720000 elements of order 7 (369M nodes, 23 GB): G's element offsets
    pass 2^31 values from e = 699051 on (e * 6 * 512).  Built by tiling a
    64-element seeded mesh; checked against the oracle on elements on both
    sides of that point and at the end, and against the FP64 kernel whole."""
    base = si.make_mesh(np.random.default_rng(79), 64, 7, device="cuda")
    E = 720000
    G = base.G.repeat((E + 63) // 64, 1, 1, 1, 1)[:E].contiguous()
    gen = torch.Generator(device="cuda").manual_seed(80)
    u = torch.rand((E, 8, 8, 8), generator=gen, dtype=torch.float64, device="cuda") * 2 - 1
    w = semax.sem_ax_f64tc(u, G, base.D)
    torch.cuda.synchronize()
    idx = np.array([0, 699050, 699051, 710000, E - 2, E - 1])
    it = torch.from_numpy(idx).cuda()
    ref = oracle_mod.sem_ax(u[it].cpu(), base.G[it.remainder(64)].cpu(), base.D.cpu())
    assert rel_err(w[it], ref) <= TYPICAL_TC
    w64 = semax.sem_ax(u, G, base.D)
    r = semax.reduce(w, w64).cpu().numpy()
    assert r[0] / r[1] <= TYPICAL_TC


def test_f64tc_order15_max_size_offsets_past_2_31(semax, oracle_mod):
    """E = 90000 elements of order 15 (369M nodes, 24 GB): G's element
    offsets pass 2^31 values from e = 87382 on (e * 6 * 4096), in the
    persistent kernel whose CTAs walk the elements with a stride of the SM
    count.  Checked against the oracle on elements on both sides of that
    point and at the end, and against the FP64 kernel whole."""
    base = si.make_mesh(np.random.default_rng(81), 16, 15, device="cuda")
    E = 90000
    G = base.G.repeat((E + 15) // 16, 1, 1, 1, 1)[:E].contiguous()
    gen = torch.Generator(device="cuda").manual_seed(82)
    u = torch.rand((E, 16, 16, 16), generator=gen, dtype=torch.float64, device="cuda") * 2 - 1
    w = semax.sem_ax_f64tc(u, G, base.D)
    torch.cuda.synchronize()
    idx = np.array([0, 87381, 87382, 88000, E - 2, E - 1])
    it = torch.from_numpy(idx).cuda()
    ref = oracle_mod.sem_ax(u[it].cpu(), base.G[it.remainder(16)].cpu(), base.D.cpu())
    assert rel_err(w[it], ref) <= TYPICAL_TC
    w64 = semax.sem_ax(u, G, base.D)
    r = semax.reduce(w, w64).cpu().numpy()
    assert r[0] / r[1] <= TYPICAL_TC


def test_f64tc_prepared_equals_f64tc_bit_for_bit(semax, oracle_mod):
    """The geometric factor prepared once gives sem_ax_f64tc's result bit for
    bit: on a ragged mesh, at the bench size, with zero nodes and elements,
    scaled G, a non-finite entry, and for a second u on the same Gp."""
    m = si.make_mesh(np.random.default_rng(95), 37, 7, device="cuda")
    Gp = semax.f64tc_prepare(m.G)
    torch.cuda.synchronize()
    assert Gp.numel() == 37 * 24592
    w = semax.sem_ax_f64tc_prepared(m.u, Gp, m.D)
    assert torch.equal(w, semax.sem_ax_f64tc(m.u, m.G, m.D))
    assert rel_err(w, oracle_mod.sem_ax(m.u.cpu(), m.G.cpu(), m.D.cpu())) <= TYPICAL_TC
    u2 = torch.rand_like(m.u) - 0.5
    assert torch.equal(semax.sem_ax_f64tc_prepared(u2, Gp, m.D), semax.sem_ax_f64tc(u2, m.G, m.D))
    G = m.G.clone()
    G[3] = 0.0
    G[5, :, 1, 2, 3] = 0.0
    G[7] *= 2.0 ** 700
    G[9] *= 2.0 ** -900
    G[11, 2, 4, 4, 4] = float("inf")
    G[13, :, 2, 2, 2] *= 2.0 ** -60    # one node far below the rest of its element (per-node vs per-element scale)
    Gp2 = semax.f64tc_prepare(G)
    w2 = semax.sem_ax_f64tc_prepared(m.u, Gp2, m.D)
    ref = semax.sem_ax_f64tc(m.u, G, m.D)
    keep = torch.arange(37, device=w2.device) != 11
    assert torch.equal(w2[keep], ref[keep])
    assert torch.isnan(w2[11]).all() and torch.isnan(ref[11]).all()
    big = si.make_workload(1, device="cuda")[0]
    Gpb = semax.f64tc_prepare(big.G)
    assert torch.equal(semax.sem_ax_f64tc_prepared(big.u, Gpb, big.D), semax.sem_ax_f64tc(big.u, big.G, big.D))


def test_f64tc_prepared_order15_equals_f64tc_bit_for_bit(semax, oracle_mod):
    """Order 15: the prepared halves give sem_ax_f64tc's result bit for bit,
    ragged, with zero, far-apart-scale and non-finite G, and at the bench size."""
    m = si.make_mesh(np.random.default_rng(96), 21, 15, device="cuda")
    G = m.G.clone()
    G[2] = 0.0
    G[4, 3:] *= 2.0 ** 80
    G[6, :3, ::2] *= 2.0 ** -70
    G[8, 5, 1, 2, 3] = float("nan")
    for GG in (m.G, G):
        Gp = semax.f64tc_prepare(GG)
        assert Gp.numel() == 21 * 196624
        w = semax.sem_ax_f64tc_prepared(m.u, Gp, m.D)
        ref = semax.sem_ax_f64tc(m.u, GG, m.D)
        keep = torch.arange(21, device=w.device) != (8 if GG is G else -1)
        assert torch.equal(w[keep], ref[keep])
    assert torch.isnan(w[8]).all()
    big = si.make_workload(2, device="cuda")[0]
    Gpb = semax.f64tc_prepare(big.G)
    assert torch.equal(semax.sem_ax_f64tc_prepared(big.u, Gpb, big.D), semax.sem_ax_f64tc(big.u, big.G, big.D))


def test_energy_norm_on_the_gpu(semax, oracle_mod):
    """u^T A u with the FP64 reduction on the GPU: equal to the oracle's energy
    for the FP64 and both FP64-accurate forms, and positive for random u."""
    m = si.make_mesh(np.random.default_rng(81), 40, 7)
    ref = oracle_mod.sem_ax(m.u, m.G, m.D)
    e_ref = float(np.sum(m.u.numpy() * ref))
    assert e_ref > 0
    u = m.u.cuda()
    for fn in (semax.sem_ax, semax.sem_ax_f64x, semax.sem_ax_f64tc):
        w = fn(u, m.G.cuda(), m.D.cuda())
        e = float(semax.reduce(u.reshape(-1), w.reshape(-1)).cpu().numpy()[2])
        assert abs(e - e_ref) <= 1e-12 * e_ref


def test_f64tc_back_to_back_calls_read_the_previous_output(semax):
    """The order-7 kernel starts as a programmatic dependent of the previous
    kernel in its stream (its CTAs may be resident during that kernel's last
    wave) and reads no global memory before that kernel has completed.  A
    chain of calls, each reading the previous call's output, issued with no
    synchronisation in between, must give what the same chain gives with a
    synchronisation after every call; also alternating with the prepared
    form and with a torch kernel that rewrites the input in between."""
    m = si.make_workload(1, device="cuda")[0]   # N = 7, E = 32768: many waves per call
    Gp = semax.f64tc_prepare(m.G)
    scale = 1.0 / 64.0                          # an exact rescaling between calls
    bufs = [m.u.clone()] + [torch.empty_like(m.u) for _ in range(4)]
    torch.cuda.synchronize()
    for q in range(4):                          # unsynchronised chain, one call straight after another
        if q % 2 == 0:
            semax.sem_ax_f64tc(bufs[q], m.G, m.D, bufs[q + 1])
        else:
            semax.sem_ax_f64tc_prepared(bufs[q], Gp, m.D, bufs[q + 1])
    torch.cuda.synchronize()
    x = m.u.clone()
    for q in range(4):                          # the same chain, synchronised
        x = semax.sem_ax_f64tc(x, m.G, m.D) if q % 2 == 0 else semax.sem_ax_f64tc_prepared(x, Gp, m.D)
        torch.cuda.synchronize()
        assert torch.equal(bufs[q + 1], x), q
    # w = A u then u overwritten in place by A's output in the same stream
    u = m.u.clone()
    for _ in range(3):
        semax.sem_ax_f64tc_prepared(u, Gp, m.D, bufs[0])
        u.copy_(bufs[0]).mul_(scale)
    torch.cuda.synchronize()
    x = m.u.clone()
    for _ in range(3):
        x = semax.sem_ax_f64tc_prepared(x, Gp, m.D) * scale
        torch.cuda.synchronize()
    assert torch.equal(u, x)
