"""Batched solves (rk_solve_batch) and problem memory management: a batch of
independent problems gives exactly what each problem gives alone, failures
stay with their problem, and a released problem whose recycle space is
restored continues bit-identically (checkpoint / resume of the sequence)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from problems.configs import config4_problem  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as g
    g.build()
    from paper_1501_03358_gb300 import Context
    c = Context()
    yield c
    c.close()


def small_set(n, max_edge=40):
    return [config4_problem(p, max_edge=max_edge, min_edge=12) for p in range(n)]


KW = dict(tol=1e-8, m=30, k=8, mode="hybrid", hybrid_switch=2, max_matvec=3000)


def test_batch_equals_alone(ctx):
    from paper_1501_03358_gb300 import Problem, solve_batch
    cfgs = small_set(6)
    alone = [Problem(ctx, c.grid, torch.from_numpy(c.coef)) for c in cfgs]
    batch = [Problem(ctx, c.grid, torch.from_numpy(c.coef)) for c in cfgs]
    for t in range(4):  # steps 0-1 rGCROT, 2-3 rBiCGStab with the frozen space
        bs = [torch.from_numpy(c.rhs(t)).cuda() for c in cfgs]
        precision = "mixed" if t % 2 else "fp64"
        xs, infos = solve_batch(batch, bs, nthreads=3, precision=precision, **KW)
        for i, p in enumerate(alone):
            xa, ia = p.solve(bs[i], precision=precision, **KW)
            assert infos[i]["status"] == ia["status"] == 0, (t, i, infos[i], ia)
            assert infos[i]["matvecs"] == ia["matvecs"]
            assert infos[i]["mode_used"] == ia["mode_used"]
            assert torch.equal(xs[i], xa), (t, i)
            assert infos[i]["recycle_dim"] == ia["recycle_dim"]
    for p in alone + batch:
        p.close()


def test_batch_failure_stays_with_its_problem(ctx):
    from paper_1501_03358_gb300 import Problem, solve_batch
    from paper_1501_03358_gb300.native import RKError, RK_E_INVALID
    cfgs = small_set(3)
    probs = [Problem(ctx, c.grid, torch.from_numpy(c.coef)) for c in cfgs]
    bs = [torch.from_numpy(c.rhs(0)).cuda() for c in cfgs]
    bs[1][5] = float("nan")
    xs, infos = solve_batch(probs, bs, **KW)
    assert infos[1]["status"] == RK_E_INVALID
    assert infos[0]["status"] == 0 and infos[2]["status"] == 0
    with pytest.raises(RKError):
        solve_batch(probs, bs, check_status=True, **KW)
    with pytest.raises(RKError):  # the same problem twice in one batch
        solve_batch([probs[0], probs[0]], [bs[0], bs[0]], **KW)
    for p in probs:
        p.close()


def test_release_and_restore_is_exact(ctx):
    from paper_1501_03358_gb300 import Problem
    c = small_set(1, max_edge=32)[0]
    kw = dict(KW, mode="rGCROT")
    a = Problem(ctx, c.grid, torch.from_numpy(c.coef))
    b = Problem(ctx, c.grid, torch.from_numpy(c.coef))
    rhs = [torch.from_numpy(c.rhs(t)).cuda() for t in range(3)]
    for t in range(2):
        a.solve(rhs[t], **kw)
        b.solve(rhs[t], **kw)
    full = b.memory()
    blob = b.export_recycle().cpu()
    U, C = b.get_recycle()
    b.release()
    assert b.memory() < full
    assert b.stats()["recycle_dim"] == 0
    # the FP64 copy restores the space to double rounding; the blob exactly
    c2 = Problem(ctx, c.grid, torch.from_numpy(c.coef))
    c2.set_recycle(U, C)
    U2, C2 = c2.get_recycle()
    assert torch.allclose(U2, U, rtol=2.0 ** -52, atol=0) and torch.allclose(C2, C, rtol=2.0 ** -52, atol=0)
    c2.close()
    b.import_recycle(blob)
    xa, ia = a.solve(rhs[2], **kw)
    xb, ib = b.solve(rhs[2], **kw)
    assert ia["matvecs"] == ib["matvecs"]
    assert torch.equal(xa, xb)
    a.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_phase_equals_alone_and_thread_pool(ctx, precision, tmp_path, monkeypatch):
    """The batched rBiCGStab phase: twelve uneven problems (7- and 19-band),
    each with its own recycle space, advance together in one launch per
    iteration phase over a (problem, block) work list, with launch shapes
    picked by the autotuner (cached to the RK_TUNE_CACHE file); every solve
    equals, bit for bit, the same solve alone and the same batch on the
    thread-pool executor (the default; the batched phase is selected with
    RK_BATCHED_BICG=1), in matrix-vector products, restarts and x."""
    import json
    import oracle
    from paper_1501_03358_gb300 import Problem, solve_batch
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("RK_TUNE_CACHE", str(cache))
    cfgs = small_set(10, max_edge=40)
    from problems import make_config
    cfgs += [make_config(1, size=14), make_config(1, size=9)]  # 7-band problems in the same batch
    kw = dict(tol=1e-8, k=8, mode="rBiCGStab", max_matvec=3000, precision=precision)
    sets = []
    for c in cfgs:
        op = oracle.Stencil(c.grid, c.coef)
        _, U, C, _ = oracle.rgcrot(op, c.rhs(0), tol=1e-9, m=20, k=8, max_matvec=400)
        sets.append((torch.from_numpy(U.T.copy()).cuda(), torch.from_numpy(C.T.copy()).cuda()))
    def fresh():
        ps = [Problem(ctx, c.grid, torch.from_numpy(c.coef)) for c in cfgs]
        for p, (U, C) in zip(ps, sets):
            p.set_recycle(U, C)
        return ps
    alone, batch, pool = fresh(), fresh(), fresh()
    for t in (1, 2):
        bs = [torch.from_numpy(c.rhs(t)).cuda() for c in cfgs]
        ref = [p.solve(b, **kw) for p, b in zip(alone, bs)]
        monkeypatch.setenv("RK_BATCHED_BICG", "1")
        xs, infos = solve_batch(batch, bs, nthreads=4, **kw)
        monkeypatch.delenv("RK_BATCHED_BICG", raising=False)
        xp, ip = solve_batch(pool, bs, nthreads=4, **kw)
        for i in range(len(cfgs)):
            xa, ia = ref[i]
            assert ia["status"] == 0 and infos[i]["status"] == 0 and ip[i]["status"] == 0, (i, t)
            for inf in (infos[i], ip[i]):
                assert inf["matvecs"] == ia["matvecs"] and inf["restarts"] == ia["restarts"], (i, t)
                assert inf["mode_used"] == ia["mode_used"] == 2
            assert torch.equal(xs[i], xa) and torch.equal(xp[i], xa), (i, t)
    tuned = json.loads(cache.read_text())
    assert any(k.startswith("bicg-n12") for k in tuned)
    for p in alone + batch + pool:
        p.close()


def test_continuous_serving_with_eviction_matches_direct_sequences(ctx):
    """Continuous admission: requests for four problems arrive while others
    are being solved (three slots, each its own stream), under a budget that
    holds the operators and only about two problems' solve footprints, so
    problems are evicted (recycle space spilled to host memory) and restored
    while other slots run. Each request's x equals, bit for bit, the same
    problem's sequence solved alone, in both phases of the hybrid."""
    from paper_1501_03358_gb300 import Problem
    from paper_1501_03358_gb300.serving import Server
    cfgs = small_set(4, max_edge=36)
    kw = dict(KW)  # hybrid: steps 0-1 rGCROT, 2-3 rBiCGStab
    steps = 4
    direct, base, foot = {}, [], []
    for i, c in enumerate(cfgs):
        p = Problem(ctx, c.grid, torch.from_numpy(c.coef))
        base.append(p.memory())
        foot.append(p.footprint(**kw))
        direct[i] = [p.solve(torch.from_numpy(c.rhs(t)).cuda(), **kw) for t in range(steps)]
        p.close()
    budget = sum(base) + 2 * max(f - b for f, b in zip(foot, base))
    srv = Server(ctx, budget, kw, slots=3)
    for i, c in enumerate(cfgs):
        srv.add(i, c.grid, torch.from_numpy(c.coef))
    rhs = {(i, t): torch.from_numpy(c.rhs(t)).cuda() for i, c in enumerate(cfgs) for t in range(steps)}
    torch.cuda.synchronize()
    # staggered arrivals: the next step of every problem is submitted while
    # the slots are still busy with the previous ones
    order = [(i, t) for t in range(steps) for i in range(len(cfgs))]
    k = 0
    while k < len(order) or srv.queue or srv.in_flight():
        if k < len(order):
            srv.submit(order[k][0], rhs[order[k]])
            k += 1
        srv.poll()
        if k >= len(order) or srv.in_flight() >= 3:
            srv.wait_any(timeout=5.0)
    srv.drain()
    assert len(srv.done) == len(order)
    assert srv.evictions > 0 and srv.restores > 0
    assert srv.max_in_flight >= 2
    seen = {i: 0 for i in range(len(cfgs))}
    for r in sorted(srv.done, key=lambda r: r.rid):
        t = seen[r.name]
        seen[r.name] += 1
        xd, idd = direct[r.name][t]
        assert r.info["status"] == 0
        assert r.info["mode_used"] == idd["mode_used"]
        assert r.info["matvecs"] == idd["matvecs"], (r.name, t)
        assert torch.equal(r.x, xd), (r.name, t)
    srv.close()


def test_footprint_bounds_the_memory_of_a_first_solve(ctx):
    """rk_problem_footprint before any solve bounds the bytes the problem
    holds after it (the admission figure of the serving loop), for every
    mode and precision."""
    from paper_1501_03358_gb300 import Problem
    c = small_set(1, max_edge=30)[0]
    for kw in (dict(KW), dict(KW, mode="rGCROT", precision="mixed"), dict(KW, mode="rBiCGStab", precision="df"),
               dict(KW, mode="rGCROT", precond="subdomain", precond_side="left")):
        p = Problem(ctx, c.grid, torch.from_numpy(c.coef))
        f = p.footprint(**kw)
        for t in range(3):
            p.solve(torch.from_numpy(c.rhs(t)).cuda(), **kw)
            assert p.memory() <= f, kw
        p.close()
