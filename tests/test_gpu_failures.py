"""Failure detection without any GPU fault (needs a GB300).

* A failed device allocation, injected on the host with
  mgs_debug_fail_allocation, at every allocation that creating a scene makes
  in turn: each attempt returns an error, releases what it held, and the next
  call builds the same table as before; a failed allocation while a table is
  built; a served job whose scene cannot be made resident fails alone, and
  the job queued behind it gets the result it gets on its own.
* The bounded waits of the tensor-core SH assignment: with a limit of a few
  clock cycles every wait gives up before its copy lands, each CTA drains its
  own copy and frees its tensor memory, and the call returns MGS_ERR_TIMEOUT;
  the next call, at the default limit, is exact again.
"""
import numpy as np
import pytest

from paper_2604_26799_gb300 import mgs, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

OOM, CUDA, TIMEOUT = -4, -5, -7


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_26799_gb300 import build
    build.build()
    c = mgs.mgs_create(0)
    yield c
    mgs.mgs_debug_fail_allocation(0)
    mgs.mgs_destroy(c)   # fails with BUSY if a failed call leaked a scene


def table_of(ctx, attrs, imp, grid, host=True):
    dev = torch.device("cuda:0")
    scene = mgs.mgs_scene_create(ctx, attrs if host else torch.from_numpy(attrs).to(dev),
                                 imp if host else torch.from_numpy(imp).to(dev))
    try:
        L = mgs.mgs_table_layout_for(attrs.shape[0], attrs.shape[1], grid)
        tab = torch.zeros(L.total_bytes, dtype=torch.uint8, device=dev)
        mgs.mgs_build_cost_table(ctx, scene, grid, tab)
        torch.cuda.synchronize()
    finally:
        mgs.mgs_scene_destroy(scene)
    return tab.cpu().numpy()


def test_scene_creation_fails_cleanly_at_every_allocation(ctx):
    attrs, imp = synth.make_scene(30_000, seed=90)
    grid = mgs.Grid(synth.keep_counts(30_000, [(1, 2), (1, 1)]), [2, 8, 16], 4096)
    ref = table_of(ctx, attrs, imp, grid)
    a0 = mgs.mgs_debug_allocations()
    sc = mgs.mgs_scene_create(ctx, attrs, imp)   # host inputs: staging + scene + sort scratch
    mgs.mgs_scene_destroy(sc)
    torch.cuda.synchronize()
    n_alloc = mgs.mgs_debug_allocations() - a0
    assert n_alloc >= 8
    for k in range(1, n_alloc + 1):
        mgs.mgs_debug_fail_allocation(k)
        with pytest.raises(mgs.MgsError) as e:
            mgs.mgs_scene_create(ctx, attrs, imp)
        assert e.value.status in (OOM, CUDA), (k, e.value)
        mgs.mgs_debug_fail_allocation(0)
    assert np.array_equal(table_of(ctx, attrs, imp, grid), ref)


def test_table_build_fails_cleanly(ctx):
    attrs, imp = synth.make_scene(20_000, seed=91)
    grid = mgs.Grid(synth.keep_counts(20_000, [(1, 3), (1, 1)]), [4, 12], 2048)
    ref = table_of(ctx, attrs, imp, grid)
    dev = torch.device("cuda:0")
    scene = mgs.mgs_scene_create(ctx, attrs, imp)
    try:
        L = mgs.mgs_table_layout_for(20_000, attrs.shape[1], grid)
        tab = torch.zeros(L.total_bytes, dtype=torch.uint8, device=dev)
        for k in (1, 2):   # the kept lists, then the launch scratch
            mgs.mgs_debug_fail_allocation(k)
            with pytest.raises(mgs.MgsError) as e:
                mgs.mgs_build_cost_table(ctx, scene, grid, tab)
            assert e.value.status in (OOM, CUDA)
            mgs.mgs_debug_fail_allocation(0)
        mgs.mgs_build_cost_table(ctx, scene, grid, tab)
        torch.cuda.synchronize()
        assert np.array_equal(tab.cpu().numpy(), ref)
    finally:
        mgs.mgs_scene_destroy(scene)


def test_served_job_failure_is_isolated(ctx):
    bits = [2, 4, 8, 12, 16]
    jobs = []
    for i, n in enumerate((9_000, 12_000, 7_000)):
        attrs, imp = synth.make_scene(n, seed=92 + i)
        grid = mgs.Grid(synth.keep_counts(n, list(synth.tenths())), bits, 2048)
        jobs.append((attrs, imp, grid, 0.3 * n * 59))
    direct = []
    for attrs, imp, grid, budget in jobs:
        L = mgs.mgs_table_layout_for(attrs.shape[0], attrs.shape[1], grid)
        direct.append(mgs.mgs_solve_budget(table_of(ctx, attrs, imp, grid), L, grid, budget, mgs.solve_opts()))
    srv = mgs.mgs_server_create(ctx, max_jobs=1, slice_items=0)
    try:
        a, i, g, b = jobs[0]
        j0 = mgs.mgs_server_submit(srv, a, i, g, b, mgs.solve_opts())
        r0 = mgs.mgs_server_wait(srv, j0, timeout_ms=120000, max_choice=1 << 20)
        # one job in flight at a time: the next allocation is job 1's first ingest allocation
        mgs.mgs_debug_fail_allocation(1)
        ids = [mgs.mgs_server_submit(srv, a, i, g, b, mgs.solve_opts()) for a, i, g, b in jobs[1:]]
        r1, r2 = [mgs.mgs_server_wait(srv, j, timeout_ms=120000, max_choice=1 << 20) for j in ids]
    finally:
        mgs.mgs_debug_fail_allocation(0)
        mgs.mgs_server_destroy(srv)
    assert r1["status"] in (OOM, CUDA)
    for r, d in ((r0, direct[0]), (r2, direct[2])):
        assert r["status"] == 0, r.get("error")
        assert r["r_index"] == d["r_index"] and r["objective"] == d["objective"]
        assert np.array_equal(r["choice"], d["choice"])


def test_tensor_wait_limit_times_out_and_recovers(ctx):
    dev = torch.device("cuda:0")
    attrs, _ = synth.make_scene(20_000, seed=93)
    x = torch.from_numpy(np.ascontiguousarray(attrs[:, 6:51])).to(dev)
    cb = x[::40].contiguous()
    mgs.mgs_vq_set_tensor_cores(ctx, False)
    ref, _ = mgs.mgs_vq_assign(ctx, x, cb)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    mgs.mgs_vq_set_tensor_cores(ctx, True)
    try:
        mgs.mgs_vq_set_wait_limit(ctx, 16)
        with pytest.raises(mgs.MgsError) as e:
            mgs.mgs_vq_assign(ctx, x, cb)
        assert e.value.status == TIMEOUT
    finally:
        mgs.mgs_vq_set_wait_limit(ctx, 0)
    idx, _ = mgs.mgs_vq_assign(ctx, x, cb)
    torch.cuda.synchronize()
    assert np.array_equal(idx.cpu().numpy(), ref)
    with pytest.raises(mgs.MgsError) as e:
        mgs.mgs_vq_set_wait_limit(ctx, -1)
    assert e.value.status == -1
