"""Ensembles of independent grids of uneven sizes (ns3d_batch_*): the sequential, graph and
persistent schedules and every tile variant give bitwise identical results, equal to
per-instance contexts, and one instance matches the oracle; the autotuner picks a variant,
caches it and leaves the caller's states untouched."""
import json
import os

import numpy as np
import pytest

from paper_2211_16718_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SIZES = [(16, 16, 16), (24, 20, 12), (12, 24, 16), (32, 32, 32), (20, 12, 24)]


@pytest.fixture(scope="module")
def ns3d():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2211_16718_gb300 import build as B
    B.build()
    from paper_2211_16718_gb300 import ns3d as N
    N.lib()
    return N


def _ensemble(ns3d, rk=0, precision=0):
    states, params, dts = [], [], []
    for i, (nx, ny, nz) in enumerate(SIZES):
        u = I.random_smooth(nx, ny, nz, seed=20 + i, amp=0.1, mach=0.4)
        mu = 0.0 if i == 2 else 2e-3 * (i + 1)
        params.append(ns3d.default_params(nx, ny, nz, mu_eff=mu, rk=rk, precision=precision))
        states.append(u)
        dts.append(0.01 + 0.002 * i)
    return states, params, dts


def _run_batch(ns3d, states, params, dts, schedule, nsteps, variant=None):
    import torch
    b = ns3d.Batch(params)
    ud = [torch.from_numpy(u.copy()).cuda() for u in states]
    b.set_states(ud)
    b.set_dt(dts)
    if variant is not None:
        b.set_variant(variant)
    b.step(nsteps, schedule)
    b.check()
    out = [t.cpu().numpy() for t in ud]
    info = b.info()
    b.close()
    return out, info


@pytest.mark.parametrize("rk", [0, 1])
def test_schedules_agree_bitwise_with_contexts(ns3d, rk):
    import torch
    states, params, dts = _ensemble(ns3d, rk=rk)
    ref = []
    for u, p, dt in zip(states, params, dts):
        s = ns3d.Solver(p.nx, p.ny, p.nz, mu_eff=p.mu_eff, rk=rk)
        ud = torch.from_numpy(u.copy()).cuda()
        s.rk_step(ud, dt, 3)
        ref.append(ud.cpu().numpy())
        s.close()
    for schedule in ("sequential", "graph", "persistent"):
        out, info = _run_batch(ns3d, states, params, dts, schedule, 3)
        for a, r in zip(out, ref):
            assert np.array_equal(a, r), schedule
    assert info["persistent_ctas_per_sm"] >= 1


def test_one_instance_matches_oracle(ns3d, oracle):
    states, params, dts = _ensemble(ns3d)
    out, _ = _run_batch(ns3d, states, params, dts, "persistent", 2)
    i = 3
    p = params[i]
    ref = oracle.rk_step(oracle.Params(p.nx, p.ny, p.nz, mu_eff=p.mu_eff), states[i], dts[i], 2)
    assert np.abs(out[i] - ref).max() / np.abs(ref).max() <= 1e-10


def test_tile_variants_bitwise_identical(ns3d):
    import torch
    states, params, dts = _ensemble(ns3d)
    outs = [_run_batch(ns3d, states, params, dts, "graph", 2, variant=v)[0] for v in range(3)]
    for v in (1, 2):
        for a, r in zip(outs[v], outs[0]):
            assert np.array_equal(a, r)
    u = states[3]
    p = params[3]
    s = ns3d.Solver(p.nx, p.ny, p.nz, mu_eff=p.mu_eff)
    rs = []
    for v in range(3):
        ns3d.set_solver_variant(s, v)
        rs.append(s.rhs(torch.from_numpy(u.copy()).cuda()).cpu().numpy())
    assert np.array_equal(rs[0], rs[1]) and np.array_equal(rs[0], rs[2])


def test_strict_mode_persistent(ns3d):
    states, params, dts = _ensemble(ns3d, precision=2)
    a, _ = _run_batch(ns3d, states, params, dts, "persistent", 2)
    b, _ = _run_batch(ns3d, states, params, dts, "sequential", 2)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_autotune_caches_and_keeps_states(ns3d, tmp_path):
    """Per grid size the fastest tile shape of its own timings, then the branch count; one
    cache line per size plus one for the branches; a second call reads them back."""
    import torch
    states, params, dts = _ensemble(ns3d)
    states = states + [s.copy() for s in states[:2]]  # two sizes with two instances each
    params = params + params[:2]
    dts = dts + dts[:2]
    cache = str(tmp_path / "tune.jsonl")
    b = ns3d.Batch(params)
    ud = [torch.from_numpy(u.copy()).cuda() for u in states]
    b.set_states(ud)
    b.set_dt(dts)
    t = b.autotune(cache)
    sizes = [(p.nx, p.ny, p.nz, p.mu_eff > 0) for p in params]
    for i, v in enumerate(t["variants"]):
        ms = t["ms_variants"][i]
        assert 0 <= v < 3 and all(m > 0 for m in ms) and ms[v] == min(ms)
        for j in range(len(params)):
            if sizes[j] == sizes[i]:
                assert t["variants"][j] == v
    timed = [m for m in t["ms_branches"] if m > 0]
    counts = [k for k in (1, 2, 4, 8) if k <= len(params)]
    assert len(timed) == len(counts) and t["ms_branches"][t["branches"] - 1] == min(timed)
    for tt, u in zip(ud, states):
        assert np.array_equal(tt.cpu().numpy(), u)
    lines = [json.loads(line) for line in open(cache)]
    assert len(lines) == len(set(sizes)) + 1
    assert sum("branches" in ln for ln in lines) == 1
    t2 = b.autotune(cache)
    assert t2["variants"] == t["variants"] and t2["branches"] == t["branches"]
    assert all(m == -1.0 for row in t2["ms_variants"] for m in row) and all(m == -1.0 for m in t2["ms_branches"])
    assert len(open(cache).readlines()) == len(lines)
    b.close()


@pytest.mark.parametrize("branches", [1, 3, 8])
def test_mixed_instance_variants_and_branches_bitwise(ns3d, branches):
    """Per-instance tile shapes and any branch count give the bits of per-instance contexts."""
    import torch
    states, params, dts = _ensemble(ns3d)
    ref = []
    for u, p, dt in zip(states, params, dts):
        s = ns3d.Solver(p.nx, p.ny, p.nz, mu_eff=p.mu_eff)
        ud = torch.from_numpy(u.copy()).cuda()
        s.rk_step(ud, dt, 2)
        ref.append(ud.cpu().numpy())
        s.close()
    for schedule in ("sequential", "graph"):
        b = ns3d.Batch(params)
        ud = [torch.from_numpy(u.copy()).cuda() for u in states]
        b.set_states(ud)
        b.set_dt(dts)
        for i in range(len(params)):
            b.set_instance_variant(i, (i + branches) % 3)
        b.set_branches(branches)
        b.step(2, schedule)
        b.check()
        assert b.schedule_info() == {"variants": [(i + branches) % 3 for i in range(len(params))],
                                     "branches": branches}
        for t, r in zip(ud, ref):
            assert np.array_equal(t.cpu().numpy(), r), schedule
        b.close()


def test_ensemble_of_the_benchmark_sizes(ns3d, oracle):
    """The ensemble sizes of the benchmark (32^3 .. 128^3 decaying turbulence, two instances
    per size, dt from CFL 0.4 each), autotuned, 2 graph-scheduled RK4 steps: one instance of
    each size against the oracle (1e-10 relative after the steps), the other bitwise against
    its own context."""
    import torch
    sizes = [32, 48, 64, 96, 128]
    mu = I.hit_mu_eff()
    states = [I.isotropic_turbulence(n, seed=k) for k in range(2) for n in sizes]
    params = [ns3d.default_params(u.shape[-1], u.shape[-1], u.shape[-1], mu_eff=mu) for u in states]
    b = ns3d.Batch(params)
    ud = [torch.from_numpy(u.copy()).cuda() for u in states]
    b.set_states(ud)
    dts = b.set_dt_from_cfl(0.4)
    b.autotune(None)
    b.step(2, "graph")
    b.check()
    out = [t.cpu().numpy() for t in ud]
    b.close()
    for i, (u, p, dt) in enumerate(zip(states, params, dts)):
        n = p.nx
        if i < len(sizes):
            ref = oracle.rk_step(oracle.Params(n, n, n, mu_eff=mu), u, dt, 2)
            assert np.abs(out[i] - ref).max() / np.abs(ref).max() <= 1e-10, n
        else:
            s = ns3d.Solver(n, n, n, mu_eff=mu)
            x = torch.from_numpy(u.copy()).cuda()
            s.rk_step(x, dt, 2)
            assert np.array_equal(out[i], x.cpu().numpy()), n
            s.close()


def test_batch_stats_match_contexts(ns3d):
    import torch
    states, params, dts = _ensemble(ns3d)
    b = ns3d.Batch(params)
    ud = [torch.from_numpy(u.copy()).cuda() for u in states]
    b.set_states(ud)
    b.set_dt(dts)
    st = b.stats().cpu().numpy()
    for i, (u, p) in enumerate(zip(states, params)):
        s = ns3d.Solver(p.nx, p.ny, p.nz, mu_eff=p.mu_eff)
        out = torch.zeros(ns3d.NS3D_STATS_NDOUBLE, dtype=torch.float64, device="cuda")
        s.stats_async(torch.from_numpy(u.copy()).cuda(), out)
        assert np.array_equal(st[i, :10], out.cpu().numpy()[:10])
    b.close()


def test_batch_dt_from_cfl_equals_contexts(ns3d):
    """ns3d_batch_set_dt_from_cfl gives each instance the time step its own context computes
    (ns3d_dt_from_cfl, the same kernels: the same bits) and applies it."""
    import torch
    states, params, _ = _ensemble(ns3d)
    b = ns3d.Batch(params)
    ud = [torch.from_numpy(u.copy()).cuda() for u in states]
    b.set_states(ud)
    dts = b.set_dt_from_cfl(0.4)
    ref = []
    for u, p in zip(states, params):
        s = ns3d.Solver(p.nx, p.ny, p.nz, mu_eff=p.mu_eff)
        ref.append(s.dt_from_cfl(torch.from_numpy(u.copy()).cuda(), 0.4))
        s.close()
    assert dts == ref
    b.step(1, "graph")
    out = [t.cpu().numpy() for t in ud]
    exp, _ = _run_batch(ns3d, states, params, ref, "graph", 1)
    assert all(np.array_equal(a, e) for a, e in zip(out, exp))
    with pytest.raises(ns3d.Ns3dError):
        b.set_dt_from_cfl(-1.0)
    b.close()


def test_batch_rejects_bad_input(ns3d):
    p = ns3d.default_params(8, 8, 8)
    q = ns3d.default_params(8, 8, 8, precision=ns3d.NS3D_FP32_BULK)
    with pytest.raises(ns3d.Ns3dError):
        ns3d.Batch([p, q])
    b = ns3d.Batch([p])
    with pytest.raises(ns3d.Ns3dError):
        b.step(1, "graph")  # no states yet
    b.close()
