"""The search server: continuous batching gives every job the result it gets
alone, and every served table equals the oracle's within the cost-table bar;
admission respects slots and the HBM budget; failures and timeouts are
reported per job (needs a GB300)."""
import numpy as np
import pytest

import oracle
from paper_2604_26799_gb300 import mgs, synth
from tests.test_gpu_cost import assert_table_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BITS = [2, 3, 4, 6, 8, 10, 12, 14, 16]
G = 2048


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_26799_gb300 import build
    build.build()
    c = mgs.mgs_create(0)
    yield c
    mgs.mgs_destroy(c)


def make_jobs(sizes, seed0=40):
    jobs = []
    for i, n in enumerate(sizes):
        attrs, imp = synth.make_scene(n, seed=seed0 + i)
        keep = synth.keep_counts(n, list(synth.tenths()))
        grid = mgs.Grid(keep, BITS, G)
        budget = 0.35 * n * 59 * 8 / 8   # about 8 bits per value, in bytes
        jobs.append((attrs, imp, grid, budget))
    return jobs


def direct(ctx, job):
    """The one-call path: table on the device, solve on the host."""
    attrs, imp, grid, budget = job
    n, C = attrs.shape
    scene = mgs.mgs_scene_create(ctx, attrs, imp)
    try:
        L = mgs.mgs_table_layout_for(n, C, grid)
        tab = np.zeros(L.total_bytes, dtype=np.uint8)
        mgs.mgs_build_cost_table(ctx, scene, grid, tab)
    finally:
        mgs.mgs_scene_destroy(scene)
    return mgs.mgs_solve_budget(tab, L, grid, budget, mgs.solve_opts())


def serve(ctx, jobs, tables=None, **opts):
    srv = mgs.mgs_server_create(ctx, **opts)
    tables = tables or [None] * len(jobs)
    try:
        ids = [mgs.mgs_server_submit(srv, a, i, g, b, mgs.solve_opts(), table_out=t)
               for (a, i, g, b), t in zip(jobs, tables)]
        res = [mgs.mgs_server_wait(srv, j, timeout_ms=120000, max_choice=1 << 20) for j in ids]
        stats = mgs.mgs_server_stats(srv)
    finally:
        mgs.mgs_server_destroy(srv)
    return res, stats


def same(r, d):
    assert r["status"] == 0, r.get("error")
    assert r["r_index"] == d["r_index"]
    assert r["est_bytes"] == d["est_bytes"] and r["objective"] == d["objective"]
    assert np.array_equal(r["choice"], d["choice"])


def test_results_equal_alone_and_in_the_mix(ctx):
    jobs = make_jobs([30_000, 7_000, 55_000, 12_345, 41_000])
    ref = [direct(ctx, j) for j in jobs]
    # alone, one job per server
    for j, d in zip(jobs, ref):
        (r,), _ = serve(ctx, [j], max_jobs=1, slice_items=0)
        same(r, d)
    # all together, small slices so every launch mixes several jobs; each job's
    # table is copied out and checked against the oracle itself
    tables = []
    for attrs, imp, grid, budget in jobs:
        L = mgs.mgs_table_layout_for(attrs.shape[0], attrs.shape[1], grid)
        tables.append(np.zeros(L.total_bytes, dtype=np.uint8))
    res, stats = serve(ctx, jobs, tables=tables, max_jobs=8, slice_items=500)
    for r, d in zip(res, ref):
        same(r, d)
    assert stats["launches"] > len(jobs)   # the work was split across shared launches
    for (attrs, imp, grid, budget), t in zip(jobs, tables):
        L = mgs.mgs_table_layout_for(attrs.shape[0], attrs.shape[1], grid)
        ref_t = oracle.cost_table(attrs, imp, grid.keep, BITS, G)
        assert_table_close(mgs.table_views(t, L), ref_t, G, f"served n={attrs.shape[0]}")


def test_admission_by_memory_budget(ctx):
    jobs = make_jobs([20_000, 20_000, 20_000], seed0=60)
    ref = [direct(ctx, j) for j in jobs]
    # a budget below two jobs' footprint: one job in flight at a time, all still served
    res, _ = serve(ctx, jobs, max_jobs=8, hbm_budget_bytes=1, slice_items=0)
    for r, d in zip(res, ref):
        same(r, d)
    order = sorted(range(3), key=lambda i: res[i]["t_admit"])
    for a, b in zip(order, order[1:]):
        assert res[b]["t_admit"] >= res[a]["t_done"] - 1e-6


def test_failed_job_does_not_disturb_others(ctx):
    jobs = make_jobs([9_000, 9_000], seed0=70)
    bad_attrs = jobs[1][0].copy()
    bad_attrs[5, 9] = np.nan
    jobs[1] = (bad_attrs,) + jobs[1][1:]
    ref0 = direct(ctx, jobs[0])
    res, _ = serve(ctx, jobs, max_jobs=4, slice_items=200)
    same(res[0], ref0)
    assert res[1]["status"] == -2


def test_wait_timeout_is_reported(ctx):
    jobs = make_jobs([200_000], seed0=80)
    srv = mgs.mgs_server_create(ctx, max_jobs=2, slice_items=0)
    try:
        a, i, g, b = jobs[0]
        jid = mgs.mgs_server_submit(srv, a, i, g, b, mgs.solve_opts())
        try:
            mgs.mgs_server_wait(srv, jid, timeout_ms=0)
        except mgs.MgsError as e:
            assert e.status == -7
        r = mgs.mgs_server_wait(srv, jid, timeout_ms=120000)
        assert r["status"] == 0
    finally:
        mgs.mgs_server_destroy(srv)
