"""GPU tests of the batched (uneven-order, one persistent launch) form, its
graph-captured plans and tuner, and the FP64 reducer."""
import json

import numpy as np
import pytest
import torch

import sem_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def semax():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1503_07659_gb300 as m
    return m


@pytest.fixture(scope="module")
def mix():
    """The uneven-order workload (~4.19M nodes, N in {3,5,7,9,11,15}) on the GPU."""
    return si.make_workload(3, device="cuda")


def _groups(meshes, ws):
    return [(m.N, m.u, m.G, m.D, w) for m, w in zip(meshes, ws)]


def test_batched_equals_per_order_plain_launches(semax, mix):
    plain = [semax.sem_ax(m.u, m.G, m.D) for m in mix]
    ws = [torch.full_like(m.u, float("nan")) for m in mix]
    semax.sem_ax_batched(_groups(mix, ws))
    torch.cuda.synchronize()
    for m, a, b in zip(mix, plain, ws):
        assert torch.equal(a, b), m.N      # same tile arithmetic: bit-identical


def test_batched_against_oracle_sampled(semax, mix, oracle_mod):
    ws = [torch.empty_like(m.u) for m in mix]
    semax.sem_ax_batched(_groups(mix, ws))
    torch.cuda.synchronize()
    rng = np.random.default_rng(13)
    for m, w in zip(mix, ws):
        idx = np.sort(rng.choice(m.E, size=min(m.E, 40), replace=False))
        it = torch.from_numpy(idx).cuda()
        ref = oracle_mod.sem_ax(m.u[it].cpu(), m.G[it].cpu(), m.D.cpu())
        err = np.max(np.abs(w[it].cpu().numpy() - ref)) / np.max(np.abs(ref))
        assert err <= 1e-12, (m.N, err)


def test_batched_ragged_small_groups(semax, oracle_mod):
    rng = np.random.default_rng(21)
    meshes = [si.make_mesh(rng, E, N, device="cuda") for N, E in [(1, 3), (4, 1), (15, 2), (6, 11), (4, 5)]]
    ws = [torch.empty_like(m.u) for m in meshes]
    semax.sem_ax_batched(_groups(meshes, ws))
    torch.cuda.synchronize()
    for m, w in zip(meshes, ws):
        ref = oracle_mod.sem_ax(m.u.cpu(), m.G.cpu(), m.D.cpu())
        assert np.max(np.abs(w.cpu().numpy() - ref)) / np.max(np.abs(ref)) <= 1e-12


def test_plan_graph_and_tuner_cache(semax, mix, tmp_path):
    plain = [semax.sem_ax(m.u, m.G, m.D) for m in mix]
    cache = tmp_path / "tune.json"
    ws = [torch.empty_like(m.u) for m in mix]
    tuned = semax.Plan(_groups(mix, ws), tune=True, cache_path=str(cache))
    data = json.loads(cache.read_text())
    assert {e["N"] for e in data["entries"]} == {m.N for m in mix}
    for w in ws:
        w.fill_(float("nan"))
    tuned()
    tuned()                      # the graph can be replayed
    torch.cuda.synchronize()
    for m, a, b in zip(mix, plain, ws):   # the tuned mapping may round differently
        assert (a - b).abs().max().item() <= 1e-12 * a.abs().max().item(), m.N
    # a second plan reads the cache and makes the same choices
    again = semax.Plan(_groups(mix, ws), tune=False, cache_path=str(cache))
    for e in data["entries"]:
        assert again.config(e["N"]) == (e["epb"], e["map"]) == tuned.config(e["N"])
    tuned.close()
    again.close()


def test_plan_with_double_float_tiles(semax, mix, oracle_mod):
    """SEMAX_PLAN_F64X: every (even n) group through the double-float tile in
    the one persistent launch equals the plain sem_ax_f64x call bit for bit,
    and the oracle to 1e-12."""
    ws = [torch.full_like(m.u, float("nan")) for m in mix]
    plan = semax.Plan(_groups(mix, ws), f64x=True)
    plan()
    torch.cuda.synchronize()
    rng = np.random.default_rng(19)
    for m, w in zip(mix, ws):
        assert plan.config(m.N)[1] == 3
        assert torch.equal(w, semax.sem_ax_f64x(m.u, m.G, m.D)), m.N
        idx = np.sort(rng.choice(m.E, size=min(m.E, 30), replace=False))
        it = torch.from_numpy(idx).cuda()
        ref = oracle_mod.sem_ax(m.u[it].cpu(), m.G[it].cpu(), m.D.cpu())
        assert np.max(np.abs(w[it].cpu().numpy() - ref)) / np.max(np.abs(ref)) <= 1e-12, m.N
    plan.close()


def test_plan_f64x_with_odd_orders_and_tuning(semax, oracle_mod):
    rng = np.random.default_rng(23)
    meshes = [si.make_mesh(rng, E, N, device="cuda") for N, E in [(2, 7), (7, 5), (4, 9), (15, 2)]]
    ws = [torch.empty_like(m.u) for m in meshes]
    plan = semax.Plan(_groups(meshes, ws), tune=True, f64x=True)
    plan()
    torch.cuda.synchronize()
    for m, w in zip(meshes, ws):
        assert plan.config(m.N)[1] == (3 if (m.N + 1) % 2 == 0 else plan.config(m.N)[1])
        ref = oracle_mod.sem_ax(m.u.cpu(), m.G.cpu(), m.D.cpu())
        assert np.max(np.abs(w.cpu().numpy() - ref)) / np.max(np.abs(ref)) <= 1e-12, m.N
    plan.close()


@pytest.mark.parametrize("f64x", [False, True])
def test_plan_with_tensor_core_orders(semax, mix, f64x):
    """SEMAX_PLAN_F64TC: the groups of order 7 and 15 run sem_ax_f64tc beside
    the persistent launch (forked streams in the captured graph) and equal
    that call bit for bit; with SEMAX_PLAN_F64X as well, the other groups of
    even n are launched apart too and equal sem_ax_f64x bit for bit; every
    other group equals the plan without the flag, bit for bit, so the forks
    and joins change nothing else.  Replays agree."""
    ws = [torch.full_like(m.u, float("nan")) for m in mix]
    plan = semax.Plan(_groups(mix, ws), f64x=f64x, f64tc=True)
    plan()
    torch.cuda.synchronize()
    ws0 = [torch.full_like(m.u, float("nan")) for m in mix]
    base = semax.Plan(_groups(mix, ws0), f64x=f64x)
    base()
    torch.cuda.synchronize()
    for m, w, w0 in zip(mix, ws, ws0):
        if m.N in (7, 15):
            assert plan.config(m.N) == (1, 4)
            assert torch.equal(w, semax.sem_ax_f64tc(m.u, m.G, m.D)), m.N
        else:
            assert plan.config(m.N) == base.config(m.N)
            assert torch.equal(w, w0), m.N
            if f64x and (m.N + 1) % 2 == 0:   # launched apart: sem_ax_f64x's kernel
                assert torch.equal(w, semax.sem_ax_f64x(m.u, m.G, m.D)), m.N
    first = [w.clone() for w in ws]
    plan()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(first, ws))
    plan.close()
    base.close()


def test_plan_tensor_core_orders_only_and_tuning(semax, oracle_mod):
    """A plan whose groups all take the tensor-core kernels has no
    persistent launch; with tuning, only the other orders are timed."""
    rng = np.random.default_rng(29)
    tc = [si.make_mesh(rng, E, N, device="cuda") for N, E in [(7, 9), (15, 3), (7, 1)]]
    ws = [torch.empty_like(m.u) for m in tc]
    plan = semax.Plan(_groups(tc, ws), f64tc=True)
    plan()
    torch.cuda.synchronize()
    for m, w in zip(tc, ws):
        ref = oracle_mod.sem_ax(m.u.cpu(), m.G.cpu(), m.D.cpu())
        assert np.max(np.abs(w.cpu().numpy() - ref)) / np.max(np.abs(ref)) <= 2e-13, m.N
    plan.close()
    mixed = tc + [si.make_mesh(rng, E, N, device="cuda") for N, E in [(3, 20), (5, 6)]]
    ws = [torch.empty_like(m.u) for m in mixed]
    plan = semax.Plan(_groups(mixed, ws), tune=True, f64x=True, f64tc=True)
    plan()
    torch.cuda.synchronize()
    for m, w in zip(mixed, ws):
        ref = oracle_mod.sem_ax(m.u.cpu(), m.G.cpu(), m.D.cpu())
        assert np.max(np.abs(w.cpu().numpy() - ref)) / np.max(np.abs(ref)) <= 1e-12, m.N
    assert plan.config(7)[1] == 4 and plan.config(3)[1] == 3 and plan.config(5)[1] == 3
    plan.close()


@pytest.mark.parametrize("count", [1, 1000, 3 * 1024 * 1024 + 7])
def test_reduce_against_definition(semax, oracle_mod, count):
    g = torch.Generator(device="cpu").manual_seed(count)
    a = (torch.rand(count, generator=g, dtype=torch.float64) - 0.5)
    b = (torch.rand(count, generator=g, dtype=torch.float64) - 0.5)
    mx, mb, dot = oracle_mod.reduce(a.numpy(), b.numpy())
    out = semax.reduce(a.cuda(), b.cuda()).cpu().numpy()
    assert out[0] == mx and out[1] == mb
    assert abs(out[2] - dot) <= 1e-13 * max(1.0, float(np.sum(np.abs(a.numpy() * b.numpy()))))
    out32 = semax.reduce(a.float().cuda(), b.cuda()).cpu().numpy()
    mx32, _, _ = oracle_mod.reduce(a.float().double().numpy(), b.numpy())
    assert out32[0] == mx32
    again = semax.reduce(a.cuda(), b.cuda()).cpu().numpy()
    assert np.array_equal(out, again)                # fixed partition: deterministic


def test_reduce_propagates_nan(semax):
    a = torch.zeros(5000, dtype=torch.float64, device="cuda")
    a[1234] = float("nan")
    out = semax.reduce(a, torch.zeros_like(a)).cpu().numpy()
    assert np.isnan(out[0]) and np.isnan(out[2])


@pytest.mark.parametrize("mapping", [0, 1, 2])
def test_every_mapping_through_cached_plan(semax, oracle_mod, tmp_path, mapping):
    """Force each thread mapping (node, column, even/odd line) through a
    hand-written tuning cache and check the plan against the oracle."""
    rng = np.random.default_rng(31 + mapping)
    meshes = [si.make_mesh(rng, E, N, device="cuda") for N, E in [(3, 40), (4, 9), (7, 13), (15, 3)]]
    ws = [torch.empty_like(m.u) for m in meshes]
    cache = tmp_path / "forced.json"
    semax.Plan(_groups(meshes, ws), tune=True, cache_path=str(cache)).close()  # device name as the library reads it
    dev = json.loads(cache.read_text())["device"]
    entries = []
    for m in meshes:
        n = m.N + 1
        mp = mapping if (mapping != 2 or n % 2 == 0) else 1
        epb = 1 if n >= 12 else 2        # n = 16 tiles of 2 elements exceed shared memory
        entries.append(f'{{"N": {m.N}, "prec": "f64", "epb": {epb}, "map": {mp}, "us": 0.0}}')
    cache.write_text('{"device": "%s", "entries": [\n  %s\n]}\n' % (dev, ",\n  ".join(entries)))
    plan = semax.Plan(_groups(meshes, ws), tune=False, cache_path=str(cache))
    plan()
    torch.cuda.synchronize()
    for m, w in zip(meshes, ws):
        n = m.N + 1
        assert plan.config(m.N)[1] == (mapping if (mapping != 2 or n % 2 == 0) else 1)
        ref = oracle_mod.sem_ax(m.u.cpu(), m.G.cpu(), m.D.cpu())
        assert np.max(np.abs(w.cpu().numpy() - ref)) / np.max(np.abs(ref)) <= 1e-12, (m.N, mapping)
    plan.close()


def test_plan_more_groups_apart_than_branches(semax):
    """With SEMAX_PLAN_F64X and SEMAX_PLAN_F64TC every even-n group runs in a
    launch of its own, dealt to at most eight graph branches: twelve such
    groups (orders 1 to 15, some twice, uneven sizes) plus groups of even N
    that stay in the persistent launch; each equals its own call bit for
    bit, and a replay gives the same bits."""
    rng = np.random.default_rng(47)
    spec = [(1, 30), (3, 17), (5, 9), (7, 40), (9, 5), (11, 3), (13, 2), (15, 2), (7, 3), (3, 1), (11, 6), (5, 21),
            (2, 11), (4, 7)]
    meshes = [si.make_mesh(rng, E, N, device="cuda") for N, E in spec]
    ws = [torch.full_like(m.u, float("nan")) for m in meshes]
    plan = semax.Plan(_groups(meshes, ws), f64x=True, f64tc=True)
    plan()
    torch.cuda.synchronize()
    first = [w.clone() for w in ws]
    for m, w in zip(meshes, ws):
        if (m.N + 1) % 2 == 0:
            assert torch.equal(w, semax.sem_ax_f64tc(m.u, m.G, m.D)), m.N   # sem_ax_f64x's kernel off 7, 15
            assert plan.config(m.N)[1] == (4 if m.N in (7, 15) else 3)
        else:
            assert torch.isfinite(w).all(), m.N
    plan()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(first, ws))
    plan.close()


def test_plan_with_prepared_tensor_core_orders(semax, mix):
    """SEMAX_PLAN_F64TC_PREPARED: the groups of order 7 and 15 run on their G
    split once at plan creation, bit for bit sem_ax_f64tc; the other groups
    equal the plan without the flag; G's values are read at creation, so a
    later change to G does not reach the plan."""
    ws = [torch.full_like(m.u, float("nan")) for m in mix]
    Gs = [m.G.clone() for m in mix]
    plan = semax.Plan([(m.N, m.u, G, m.D, w) for m, G, w in zip(mix, Gs, ws)], f64x=True, f64tc=True,
                      f64tc_prepared=True)
    plan()
    torch.cuda.synchronize()
    ws0 = [torch.full_like(m.u, float("nan")) for m in mix]
    base = semax.Plan(_groups(mix, ws0), f64x=True, f64tc=True)
    base()
    torch.cuda.synchronize()
    for m, w, w0 in zip(mix, ws, ws0):
        assert torch.equal(w, w0), m.N
        if m.N in (7, 15):
            assert torch.equal(w, semax.sem_ax_f64tc(m.u, m.G, m.D)), m.N
    first = [w.clone() for w in ws]
    for G in Gs:
        G.mul_(2.0)
    plan()
    torch.cuda.synchronize()
    for m, w, w1 in zip(mix, ws, first):
        if m.N in (7, 15):
            assert torch.equal(w, w1), m.N              # prepared at creation: unchanged
        else:
            assert torch.equal(w, 2.0 * w1), m.N        # read at execution: doubled (exact)
    plan.close()
    base.close()
