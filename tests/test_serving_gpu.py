"""Serving (continuous batching) on the GPU: every request's result is bitwise
the result of solving it alone, whatever else shares its rounds; admission
respects the HBM budget; cancellation and error paths behave."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


def _request_data(K, G, C, snapshot):
    cfg = synth.workloads.serve_snapshot_config(snapshot, K, G, max(C, 8))
    wl = synth.make_workload(cfg, cells=np.arange(C))
    return wl


def _padded(J):
    from paper_0907_3768_gb300 import padded_rows

    return padded_rows(torch.from_numpy(J).cuda())


def _mix():
    """Requests over four grids / three grain sets and all three precisions."""
    from paper_0907_3768_gb300 import Context

    # both GEMM orientations within each tensor-core precision: G <= 128 grain-major, G = 240 cell-major
    shapes = [(100, 48, "bf16x3"), (350, 96, "fp32"), (500, 240, "fp16x3"), (200, 96, "bf16x3"),
              (100, 240, "bf16x3"), (200, 48, "fp16x3")]
    ctxs, reqs = {}, []
    rng = np.random.default_rng(11)
    for i in range(10):
        K, G, prec = shapes[i % len(shapes)]
        C = int(np.exp(rng.uniform(np.log(300), np.log(40000))))
        wl = _request_data(K, G, C, snapshot=i % 5)
        key = (K, G, prec, i % 5)
        if key not in ctxs:
            ctxs[key] = Context.from_workload(wl, precision=prec)
        reqs.append((ctxs[key], _padded(wl.J), torch.from_numpy(wl.n).cuda()))
    return ctxs, reqs


def test_results_identical_alone_and_in_the_mix():
    from paper_0907_3768_gb300 import Server

    ctxs, reqs = _mix()
    alone = []
    for ctx, J, n in reqs:
        out = ctx.solve(J, n)
        torch.cuda.synchronize()
        alone.append({k: v.clone() for k, v in out.items() if k in ("T", "L", "resid", "flags")})
    with Server(hbm_budget_bytes=8 << 30, max_inflight=6) as srv:
        tickets = [ctx.submit(srv, J, n) for ctx, J, n in reqs]
        for t, _ in tickets:
            srv.wait(t, 60000.0)
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["rounds"] >= 1 and st["p99_ms"] >= st["p50_ms"] > 0.0
    for (t, out), ref in zip(tickets, alone):
        for k in ("T", "L", "resid", "flags"):
            assert torch.equal(out[k], ref[k]), k
    for c in ctxs.values():
        assert c.check() == 0
        c.close()


def test_admission_by_footprint_and_ebusy():
    from paper_0907_3768_gb300 import DustError, Server, _lib

    ctxs, reqs = _mix()
    # budget for roughly one large request at a time: all still complete
    with Server(hbm_budget_bytes=600 << 20, max_inflight=32) as srv:
        ok = []
        for ctx, J, n in reqs:
            try:
                ok.append(ctx.submit(srv, J, n))
            except DustError as e:
                assert e.code == _lib.DUST_EBUSY
        for t, _ in ok:
            srv.wait(t, 60000.0)
        st = srv.stats()
        assert st["completed"] == len(ok) and st["hbm_in_use"] == 0
    # a request larger than the whole budget can never be admitted
    ctx, J, n = reqs[-1]
    with Server(hbm_budget_bytes=1 << 20, max_inflight=2) as srv:
        with pytest.raises(DustError) as e:
            ctx.submit(srv, J, n)
        assert e.value.code == _lib.DUST_EBUSY
    for c in ctxs.values():
        c.close()


def test_cancel_poll_and_unknown_tickets():
    from paper_0907_3768_gb300 import DustError, Server, _lib

    ctxs, reqs = _mix()
    with Server(hbm_budget_bytes=8 << 30, max_inflight=1) as srv:
        subs = [ctx.submit(srv, J, n) for ctx, J, n in reqs[:4]]
        srv.cancel(subs[-1][0])           # still queued behind max_inflight = 1
        for t, _ in subs[:3]:
            srv.wait(t, 60000.0)
        state, _ = srv.poll(subs[-1][0])
        assert state == "cancelled"
        with pytest.raises(DustError) as e:
            srv.poll(subs[0][0])          # released by its wait
        assert e.value.code == _lib.DUST_ENOTFOUND
        st = srv.stats()
        assert st["completed"] == 3 and st["cancelled"] == 1
    for c in ctxs.values():
        c.close()


def test_zero_cell_request_and_shutdown_with_queue():
    from paper_0907_3768_gb300 import Server

    ctxs, reqs = _mix()
    ctx, J, n = reqs[0]
    srv = Server(hbm_budget_bytes=8 << 30, max_inflight=2)
    t0, _ = ctx.submit(srv, J[:0], n[:0])
    assert srv.poll(t0)[0] == "done"
    for ctx, J, n in reqs:
        ctx.submit(srv, J, n)
    srv.close()                          # finishes admitted requests, cancels the rest
    torch.cuda.synchronize()
    for c in ctxs.values():
        assert c.check() == 0
        c.close()


def test_submit_waits_for_the_producer_stream():
    """Inputs still being written on the producer's stream when submit is
    called: the server's first launch for the request waits for them on the
    device, so the result is bitwise that of a solve on finished inputs."""
    from paper_0907_3768_gb300 import Context, Server

    wl = _request_data(200, 96, 20000, snapshot=3)
    J_src, n_src = _padded(wl.J), torch.from_numpy(wl.n).cuda()
    with Context.from_workload(wl, precision="bf16x3") as ctx:
        ref = ctx.solve(J_src, n_src)
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            J = torch.empty_like(J_src)
            n = torch.empty_like(n_src)
            torch.cuda._sleep(100_000_000)  # a bounded device-side delay before the copies
            J.copy_(J_src)
            n.copy_(n_src)
        with Server(1 << 30, max_inflight=4) as srv:
            t, out = ctx.submit(srv, J, n, stream=side)  # no synchronisation before submit
            srv.wait(t, 60000.0)
        torch.cuda.synchronize()
        for k in ("T", "L", "resid", "flags"):
            assert torch.equal(out[k], ref[k]), k


TOL = {"fp32": (1e-5, 1e-4), "bf16x3": (1e-3, 5e-3), "fp16x3": (1e-3, 5e-3)}


def _grid_mix():
    """Every request shape of the serving stream: K in {100, 200, 350, 500} x G in
    {48, 96, 240} (K = 500 with the large grid and its 10 % near-opaque cells), the
    three precisions in turn, seeded cell counts."""
    from paper_0907_3768_gb300 import Context

    rng = np.random.default_rng(23)
    precs = ("bf16x3", "fp32", "fp16x3")
    out = []
    for i, (K, G) in enumerate([(K, G) for K in (100, 200, 350, 500) for G in (48, 96, 240)]):
        C = int(np.exp(rng.uniform(np.log(500), np.log(30000))))
        wl = _request_data(K, G, C, snapshot=7 + i)
        ctx = Context.from_workload(wl, precision=precs[i % 3])
        out.append((wl, ctx, precs[i % 3]))
    return out


def _check_against_oracle(wl, prec, out, ncells=64):
    """T, L, the residual and the flags of sampled cells against the FP64 oracle."""
    import oracle
    from metrics import assert_flags_match, l_err, t_err

    C = wl.J.shape[0]
    cells = np.unique(np.linspace(0, C - 1, min(ncells, C)).astype(np.int64))
    ref = oracle.run(wl.lam, wl.w, wl.C_abs, wl.J[cells], wl.n[cells], wl.T_min, wl.T_max)
    T = out["T"].cpu().numpy()[cells]
    L = out["L"].cpu().numpy()[cells, :wl.K]
    tT, tL = TOL[prec]
    assert t_err(T, ref["T"], ref["flags"]).max() <= tT, f"{prec} K={wl.K} G={wl.G}"
    assert l_err(L, ref["L"]).max() <= tL, f"{prec} K={wl.K} G={wl.G}"
    assert_flags_match(out["flags"].cpu().numpy()[cells], {"flags": ref["flags"], "A": ref["A"]}, wl)
    ok = (ref["flags"] == 0).all(axis=1)
    assert np.abs(out["resid"].cpu().numpy()[cells][ok]).max(initial=0.0) <= (2e-5 if prec == "fp32" else 2e-4)


@pytest.mark.parametrize("policy", ["default", "small rounds"])
def test_serving_matches_the_oracle(policy):
    """Every request of the mix and of the full grid of serving shapes, served
    together, against the FP64 oracle on sampled cells: T and L within the
    precision's tolerance, flags as the oracle's, residuals small.  The small
    policy forces multi-part batched rounds and requests chunked over several
    rounds at these sizes."""
    from paper_0907_3768_gb300 import Server

    grid = _grid_mix()
    _, mix = _mix()
    with Server(hbm_budget_bytes=8 << 30, max_inflight=32) as srv:
        if policy != "default":
            srv.set_policy(small_terms=2e7, batch_terms=1e8, chunk_terms=3e8, age_ms=5.0)
        inputs = [(_padded(wl.J), torch.from_numpy(wl.n).cuda()) for wl, _, _ in grid]  # alive until served
        subs = [(wl, prec, ctx.submit(srv, J, n)) for (wl, ctx, prec), (J, n) in zip(grid, inputs)]
        tix = [ctx.submit(srv, J, n) for ctx, J, n in mix]
        for _, _, (t, _) in subs:
            srv.wait(t, 120000.0)
        for t, _ in tix:
            srv.wait(t, 120000.0)
        st = srv.stats()
    assert st["failed"] == 0 and st["completed"] == len(subs) + len(tix)
    for wl, prec, (_, out) in subs:
        _check_against_oracle(wl, prec, out)
    for _, ctx, _ in grid:
        assert ctx.check() == 0
        ctx.close()


def test_served_mix_matches_the_oracle():
    """The alone-vs-mix requests (four grids, three grain sets, both GEMM
    orientations, three precisions) served together, against the oracle."""
    from paper_0907_3768_gb300 import Server

    rng = np.random.default_rng(11)
    shapes = [(100, 48, "bf16x3"), (350, 96, "fp32"), (500, 240, "fp16x3"), (200, 96, "bf16x3"),
              (100, 240, "bf16x3"), (200, 48, "fp16x3")]
    ctxs, reqs = _mix()
    wls = []
    for i in range(10):  # the same draws as _mix
        K, G, prec = shapes[i % len(shapes)]
        C = int(np.exp(rng.uniform(np.log(300), np.log(40000))))
        wls.append((_request_data(K, G, C, snapshot=i % 5), prec))
    with Server(hbm_budget_bytes=8 << 30, max_inflight=6) as srv:
        tickets = [ctx.submit(srv, J, n) for ctx, J, n in reqs]
        for t, _ in tickets:
            srv.wait(t, 60000.0)
    for (wl, prec), (_, out) in zip(wls, tickets):
        _check_against_oracle(wl, prec, out)
    for c in ctxs.values():
        c.close()
