"""Serving: the continuous-batching server gives each request the same result
alone and in the mix, admits by HBM footprint, and reports timestamps."""
import numpy as np
import pytest

import workload
from tests.gpu_common import ctx_fixture, dev, nominal

pytestmark = pytest.mark.gpu


def _mg():
    import paper_1511_08200_gb300 as mg
    return mg


def _requests(seed=7):
    rng = np.random.Generator(np.random.PCG64(seed))
    alpha, s, h = nominal()
    reqs = []
    for t in range(10):
        n = int(rng.choice([32, 48, 64, 96]))
        sigma = float(rng.uniform(0.5, 2.0))
        tol = 1e-6 if rng.uniform() < 0.5 else 1e-8
        reqs.append((t, n, workload.lognormal_delta(n, sigma, 500 + t), tol))
    return reqs, alpha, s, h


def test_server_same_alone_and_in_mix():
    import torch
    mg = _mg()
    ctx = ctx_fixture()
    reqs, alpha, s, h = _requests()
    srv = mg.Server(0, slots=4)
    deltas, phis, params = {}, {}, {}
    for tag, n, d, tol in reqs:
        deltas[tag] = dev(d)
        phis[tag] = torch.full_like(deltas[tag], float("nan"))
        params[tag] = mg.default_params(alpha=alpha, s=s, h=h, tol=tol, precision="mixed")
        srv.submit(deltas[tag], params[tag], phis[tag], tag=tag)
    got = {}
    while len(got) < len(reqs):
        for c in srv.poll(wait_ms=2000):
            got[c.tag] = c
    srv.close()
    for tag, n, d, tol in reqs:
        c = got[tag]
        assert c.status == 0, c
        assert c.t_submit <= c.t_admit <= c.t_done
        assert c.info.rel_residual <= tol
        alone, _, ia = ctx.solve_fifth_force(deltas[tag], params[tag])
        assert torch.equal(alone, phis[tag])
        assert ia.cell_updates == c.info.cell_updates
    ctx.close()


def test_server_fp64_and_mixed_same_alone_and_in_mix():
    """FP64 requests (host-driven on the workers' contexts) interleaved with mixed ones
    (captured graphs): every result is bit-identical to the same solve alone."""
    import torch
    mg = _mg()
    ctx = ctx_fixture()
    reqs, alpha, s, h = _requests(seed=8)
    srv = mg.Server(0, slots=4)
    deltas, phis, params = {}, {}, {}
    for tag, n, d, tol in reqs:
        prec = "fp64" if tag % 2 == 0 else "mixed"
        deltas[tag] = dev(d)
        phis[tag] = torch.full_like(deltas[tag], float("nan"))
        params[tag] = mg.default_params(alpha=alpha, s=s, h=h, tol=tol, precision=prec)
        srv.submit(deltas[tag], params[tag], phis[tag], tag=tag)
    got = {}
    while len(got) < len(reqs):
        for c in srv.poll(wait_ms=2000):
            got[c.tag] = c
    srv.close()
    for tag, n, d, tol in reqs:
        c = got[tag]
        assert c.status == 0, c
        assert c.info.rel_residual <= tol
        alone, _, ia = ctx.solve_fifth_force(deltas[tag], params[tag])
        assert torch.equal(alone, phis[tag]), tag
        assert ia.cycles == c.info.cycles
    ctx.close()


def test_server_respects_hbm_budget():
    """With a budget below two 96^3 hierarchies, requests still all complete, one
    at a time, and the held bytes never exceed the budget at the end."""
    import torch
    mg = _mg()
    alpha, s, h = nominal()
    one = mg.graph_workspace_bytes(96)     # a served mixed solve holds its cached graph
    budget = int(1.5 * one)
    srv = mg.Server(0, slots=3, hbm_budget_bytes=budget)
    d = dev(workload.lognormal_delta(96, 1.0, 3))
    p = mg.default_params(alpha=alpha, s=s, h=h, tol=1e-6, precision="mixed")
    phis = [torch.zeros_like(d) for _ in range(4)]
    for t in range(4):
        srv.submit(d, p, phis[t], tag=t)
    done = []
    while len(done) < 4:
        done += srv.poll(wait_ms=2000)
    assert all(c.status == 0 for c in done)
    assert srv.bytes_held() <= budget
    # the admissions did not overlap: each starts after an earlier one finished
    ivs = sorted((c.t_admit, c.t_done) for c in done)
    for a, b in zip(ivs, ivs[1:]):
        assert b[0] >= a[1] - 1e-3
    with pytest.raises(mg.MG5Error):
        srv.submit(dev(np.zeros((256,) * 3)), p, torch.zeros((256,) * 3, dtype=torch.float64,
                                                               device="cuda"), tag=99)
    srv.close()
    # a budget below one request: it completes as out of memory instead of waiting
    tiny = mg.Server(0, slots=2, hbm_budget_bytes=one // 2)
    with pytest.raises(mg.MG5Error):
        tiny.submit(d, p, torch.zeros_like(d), tag=1)
    tiny.close()
    for x in phis[1:]:
        assert torch.equal(x, phis[0])


def test_server_shares_captured_graphs_between_workers():
    """Requests of one key, one after another, reuse a single pooled graph whichever
    worker takes them: the server holds exactly one entry's bytes."""
    import torch
    mg = _mg()
    alpha, s, h = nominal()
    srv = mg.Server(0, slots=3)
    d = dev(workload.lognormal_delta(48, 1.0, 11))
    p = mg.default_params(alpha=alpha, s=s, h=h, tol=1e-8, precision="mixed")
    outs = []
    for t in range(6):
        phi = torch.zeros_like(d)
        srv.submit(d, p, phi, tag=t)
        got = []
        while not got:
            got = srv.poll(wait_ms=2000)
        assert got[0].status == 0 and got[0].tag == t
        outs.append(phi)
    assert srv.bytes_held() == mg.graph_workspace_bytes(48)
    srv.close()
    for x in outs[1:]:
        assert torch.equal(x, outs[0])


def test_bench_serving_stream_matches_oracle():
    """The first requests of the serving stream bench.py offers (same generator: sides 16 k from
    32 to 256, sigma ~ U(0.5, 2), each request its own field, tol 1e-6 or 1e-8, mixed
    precision), all submitted to a server of 8 slots at once: every one converges, and those of
    side <= 128 match the FP64 oracle within the bar their tolerance implies (phi within
    ~1.5 x tol of the discrete solution: 1e-5 for 1e-6, 1e-6 for 1e-8)."""
    import torch
    import bench
    import oracle
    from tests.gpu_common import host, rel_l2
    mg = _mg()
    beta, alpha, s = mg.ndgp_coefficients(1.0, 0.3, 1.0)
    h = bench.L_BOX / 512
    count = 24
    gaps, sizes, sigmas, tols = bench.serving_stream(count)
    fields = {i: bench.serving_field(i, sizes, sigmas, torch.device("cuda")) for i in range(count)}
    srv = mg.Server(0, slots=8)
    phis = {}
    for i in range(count):
        d = fields[i]
        p = mg.default_params(alpha=alpha, s=s, h=h, tol=float(tols[i]), precision="mixed")
        phis[i] = torch.full_like(d, float("nan"))
        srv.submit(d, p, phis[i], tag=i)
    got = {}
    while len(got) < count:
        for c in srv.poll(wait_ms=5000):
            got[c.tag] = c
    srv.close()
    checked = 0
    for i in range(count):
        c = got[i]
        assert c.status in (0, 1), c
        assert c.info.rel_residual <= tols[i]
        n = int(sizes[i])
        if n > 128:
            continue
        d = host(fields[i])
        ref, rinfo = oracle.solve(d, alpha, s, h, tol=1e-12)
        assert rinfo.status == 0
        bar = 1e-5 if tols[i] > 1e-7 else 1e-6
        assert rel_l2(host(phis[i]), ref) <= bar, (i, n, tols[i])
        checked += 1
    assert checked >= 8
