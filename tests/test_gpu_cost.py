"""Parity of the CUDA cost table with the CPU oracle (needs a GB300).

Bar: group sizes, min/max, the largest error and every code bit-exact;
SSE and L1 within a relative 1e-5 of the FP64 oracle; the entropy bound within
1e-5 relative plus 2^-20 bits (the L(h) table is in 2^-22-bit units).
"""
import numpy as np
import pytest

import oracle
from paper_2604_26799_gb300 import mgs, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_26799_gb300 import build
    build.build()
    c = mgs.mgs_create(0)
    yield c
    mgs.mgs_destroy(c)


def run_table(ctx, attrs, imp, keep, bits, G, plain=False, config=None, host=False):
    dev = torch.device("cuda:0")
    grid = mgs.Grid(keep, bits, G)
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(attrs).to(dev), torch.from_numpy(imp).to(dev))
    try:
        if config is not None:
            mgs.mgs_set_tile_config(ctx, G, len(bits), config)
        L = mgs.mgs_table_layout_for(attrs.shape[0], attrs.shape[1], grid)
        if host:
            buf = np.zeros(L.total_bytes, dtype=np.uint8)
            mgs.mgs_build_cost_table(ctx, scene, grid, buf)
            out = buf
        else:
            buf = torch.zeros(L.total_bytes, dtype=torch.uint8, device=dev)
            (mgs.mgs_build_cost_table_plain if plain else mgs.mgs_build_cost_table)(ctx, scene, grid, buf)
            torch.cuda.synchronize()
            out = buf.cpu().numpy()
    finally:
        if config is not None:
            mgs.mgs_set_tile_config(ctx, G, len(bits), -1)
        mgs.mgs_scene_destroy(scene)
    return mgs.table_views(out, L), L


def assert_table_close(got, ref, G, where=""):
    assert np.array_equal(got["cnt"], ref["cnt"]), where
    assert np.array_equal(got["vmin"], ref["vmin"]), where
    assert np.array_equal(got["vmax"], ref["vmax"]), where
    bad = got["linf"] != ref["linf"]
    assert not bad.any(), f"{where} linf differs at {np.argwhere(bad)[:5]}"
    for key in ("sse", "l1"):
        g, r = got[key], ref[key]
        tol = 1e-5 * np.abs(r)
        bad = np.abs(g - r) > tol
        assert not bad.any(), f"{where} {key}: {np.argwhere(bad)[:5]} {g[bad][:5]} vs {r[bad][:5]}"
    # entropy bound (Sec. III-F): the kernel sums L(h) = h log2 h from a table
    # rounded to 2^-22 bits, one term for L(n) and one per non-empty bin, and a
    # group of n elements has at most n non-empty bins: |error| <= (n + 1) 2^-23
    # bits, plus the FP64 rounding of the oracle's own sum
    g, r = got["hbits"], ref["hbits"]
    bound = (ref["cnt"].astype(np.float64)[:, None] + 1.0) * 2.0 ** -23 + 1e-12 * np.abs(r) + 1e-9
    bad = np.abs(g - r) > bound
    assert not bad.any(), f"{where} hbits: {np.argwhere(bad)[:5]} {g[bad][:5]} vs {r[bad][:5]}"


SMALL_BITS = [1, 2, 3, 4, 6, 7, 8, 10, 12, 13, 14, 16]


@pytest.mark.parametrize("G", [4096, 1000, 64, 1])
def test_table_matches_oracle(ctx, G):
    n = 20_000
    attrs, imp = synth.make_scene(n, seed=11)
    keep = np.array([1, 2000, 7777, 20_000], dtype=np.int64)
    got, _ = run_table(ctx, attrs, imp, keep, SMALL_BITS, G)
    ref = oracle.cost_table(attrs, imp, keep, SMALL_BITS, G)
    assert_table_close(got, ref, G, f"G={G}")


def test_single_scene_workload_matches_oracle(ctx):
    """The single-scene workload in full: N = 100,000 Gaussians, r = 1/2,
    b = {4, 6, 8, 10, 12, 16}, G = 4096 (12 full groups and one of 848 per
    channel), every entry of the table against the oracle."""
    w = synth.SMALL
    attrs, imp = synth.make_scene(w.n, seed=w.seed)
    keep = w.keep()
    assert list(keep) == [50_000]
    got, L = run_table(ctx, attrs, imp, keep, list(w.bits), w.group_size)
    assert int(L.n_items) == 59 * 13
    ref = oracle.cost_table(attrs, imp, keep, list(w.bits), w.group_size)
    assert_table_close(got, ref, w.group_size, "single scene")
    assert sorted(set(got["cnt"].tolist())) == [848, 4096]


def test_every_tile_shape_matches_oracle(ctx):
    n = 9_000
    attrs, imp = synth.make_scene(n, seed=12)
    keep = np.array([3000, 9000], dtype=np.int64)
    bits = [2, 5, 9, 12, 15, 16]
    ref = {}
    for cfg in range(mgs.mgs_tile_config_count()):
        name = mgs.mgs_tile_config_name(cfg)
        cap = int(name.split("_")[0][1:]) * int(name.split("_")[1][1:])
        G = min(cap, 16384)
        if G not in ref:
            ref[G] = oracle.cost_table(attrs, imp, keep, bits, G)
        got, _ = run_table(ctx, attrs, imp, keep, bits, G, config=cfg)
        assert_table_close(got, ref[G], G, name)


def edge_scene(n=6000, seed=3):
    rng = np.random.default_rng(seed)
    attrs = np.zeros((n, 12), dtype=np.float32)
    attrs[:, :3] = rng.uniform(0, 1, (n, 3))
    attrs[:, 3] = 1.5                                            # constant channel
    attrs[:, 4] = rng.uniform(0, 1e-36, n)                       # S subnormal at high b
    attrs[:, 5] = rng.uniform(0, 1e-44, n)                       # S underflows to 0
    attrs[:, 6] = rng.uniform(0, 1, n)
    attrs[::7, 6] = np.float32(1e-41)                            # subnormal c / R
    attrs[:, 7] = 1000.0 + rng.standard_normal(n) * 1e-3         # large offset
    attrs[:, 8] = np.round(rng.standard_normal(n) * 3)           # many exact ties
    attrs[:, 9] = -rng.exponential(1.0, n)                       # negative only
    attrs[:, 10] = rng.standard_normal(n) * 1e30                 # huge magnitude
    attrs[:, 11] = rng.laplace(0, 0.05, n)
    imp = rng.permutation(n).astype(np.float32)                  # distinct
    imp[:50] = 7.0                                               # ties in importance
    return attrs, imp


@pytest.mark.parametrize("G", [512, 4096])
def test_edge_channels_match_oracle(ctx, G):
    attrs, imp = edge_scene()
    keep = np.array([1, 2, 999, 6000], dtype=np.int64)
    bits = list(range(1, 17))
    got, _ = run_table(ctx, attrs, imp, keep, bits, G)
    ref = oracle.cost_table(attrs, imp, keep, bits, G)
    assert_table_close(got, ref, G, "edge")


def test_plain_loop_equals_fused(ctx):
    attrs, imp = synth.make_scene(15_000, seed=5)
    keep = np.array([5000, 15_000], dtype=np.int64)
    bits = [2, 8, 13, 16]
    a, _ = run_table(ctx, attrs, imp, keep, bits, 4096)
    b, _ = run_table(ctx, attrs, imp, keep, bits, 4096, plain=True)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_host_table_equals_device_table(ctx):
    attrs, imp = synth.make_scene(8000, seed=6)
    keep = np.array([4000, 8000], dtype=np.int64)
    a, _ = run_table(ctx, attrs, imp, keep, [4, 8], 1024)
    b, _ = run_table(ctx, attrs, imp, keep, [4, 8], 1024, host=True)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_scene_from_host_memory_and_morton(ctx):
    n = 300_000
    attrs, imp = synth.make_scene(n, seed=8)
    scene = mgs.mgs_scene_create(ctx, attrs, imp)   # host pointers
    try:
        codes = torch.empty(n, dtype=torch.int64, device="cuda")
        order = torch.empty(n, dtype=torch.int32, device="cuda")
        mgs.mgs_scene_morton(scene, codes, order)
        torch.cuda.synchronize()
    finally:
        mgs.mgs_scene_destroy(scene)
    ref_codes, ref_order = oracle.morton(attrs)
    assert np.array_equal(codes.cpu().numpy().view(np.uint64), ref_codes)
    assert np.array_equal(order.cpu().numpy().astype(np.int64), ref_order)


def test_quantize_groups_matches_oracle(ctx):
    n, G, keep = 12_000, 1000, 7_500
    attrs, imp = synth.make_scene(n, seed=9)
    attrs[:, 20] = 2.0
    ng = oracle.n_groups(keep, G)
    rng = np.random.default_rng(1)
    qbits = rng.integers(1, 17, size=(attrs.shape[1], ng)).astype(np.uint8)
    dev = torch.device("cuda:0")
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(attrs).to(dev), torch.from_numpy(imp).to(dev))
    try:
        codes = torch.empty((attrs.shape[1], keep), dtype=torch.int16, device=dev)
        mm = torch.empty((attrs.shape[1], ng, 2), dtype=torch.float32, device=dev)
        mgs.mgs_quantize_groups(ctx, scene, keep, G, torch.from_numpy(qbits).to(dev), codes, mm)
        torch.cuda.synchronize()
    finally:
        mgs.mgs_scene_destroy(scene)
    rc, rmm = oracle.quantize(attrs, imp, keep, G, qbits)
    assert np.array_equal(codes.cpu().numpy().view(np.uint16), rc)
    assert np.array_equal(mm.cpu().numpy(), rmm)


def test_batched_plan_and_graph_equal_single(ctx):
    dev = torch.device("cuda:0")
    bits = [2, 4, 8, 12, 14, 16]
    G = 2048
    sizes = [3000, 17_000, 9000]
    scenes, tables, singles, grids, inputs = [], [], [], [], []
    try:
        for i, n in enumerate(sizes):
            attrs, imp = synth.make_scene(n, seed=20 + i)
            inputs.append((attrs, imp))
            sc = mgs.mgs_scene_create(ctx, torch.from_numpy(attrs).to(dev), torch.from_numpy(imp).to(dev))
            scenes.append(sc)
            grid = mgs.Grid(synth.keep_counts(n, [(1, 3), (2, 3), (3, 3)]), bits, G)   # per-scene sizes
            grids.append(grid)
            L = mgs.mgs_table_layout_for(n, attrs.shape[1], grid)
            tables.append(torch.zeros(L.total_bytes, dtype=torch.uint8, device=dev))
            one = torch.zeros(L.total_bytes, dtype=torch.uint8, device=dev)
            mgs.mgs_build_cost_table(ctx, sc, grid, one)
            singles.append(one)
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            plan = mgs.mgs_plan_create(ctx, scenes, grids, tables, use_graph=True, stream=st)
            try:
                for rep in range(3):
                    for t in tables:
                        t.zero_()
                    mgs.mgs_plan_launch(plan, st)
                work, launches, cfg = mgs.mgs_plan_info(plan)
                assert launches == 1 and work > 0
            finally:
                st.synchronize()
                mgs.mgs_plan_destroy(plan)
        torch.cuda.synchronize()
        # every batched, graph-replayed table against the oracle itself
        for (attrs, imp), grid, t in zip(inputs, grids, tables):
            L = mgs.mgs_table_layout_for(attrs.shape[0], attrs.shape[1], grid)
            got = mgs.table_views(t.cpu().numpy(), L)
            ref = oracle.cost_table(attrs, imp, grid.keep, bits, G)
            assert_table_close(got, ref, G, f"batched n={attrs.shape[0]}")
        for t, o in zip(tables, singles):
            assert torch.equal(t, o)
        # the one-shot batched call gives the same tables
        for t in tables:
            t.zero_()
        mgs.mgs_build_cost_tables_batched(ctx, scenes, grids, tables)
        torch.cuda.synchronize()
        for t, o in zip(tables, singles):
            assert torch.equal(t, o)
        # grids that disagree in bit-widths cannot share a launch
        bad = [grids[0], mgs.Grid(grids[1].keep, [2, 4, 8], G), grids[2]]
        with pytest.raises(mgs.MgsError) as e:
            mgs.mgs_build_cost_tables_batched(ctx, scenes, bad, tables)
        assert e.value.status == -1
    finally:
        for sc in scenes:
            mgs.mgs_scene_destroy(sc)


def test_nonfinite_and_range_rejected(ctx):
    attrs, imp = synth.make_scene(1000, seed=1)
    bad = attrs.copy()
    bad[10, 7] = np.nan
    with pytest.raises(mgs.MgsError) as e:
        mgs.mgs_scene_create(ctx, bad, imp)
    assert e.value.status == -2
    bad = attrs.copy()
    bad[0, 5], bad[1, 5] = -3e38, 3e38
    with pytest.raises(mgs.MgsError) as e:
        mgs.mgs_scene_create(ctx, bad, imp)
    assert e.value.status == -3
    imp2 = imp.copy()
    imp2[3] = np.inf
    with pytest.raises(mgs.MgsError) as e:
        mgs.mgs_scene_create(ctx, attrs, imp2)
    assert e.value.status == -2


def test_autotune_picks_a_valid_shape(ctx):
    attrs, imp = synth.make_scene(30_000, seed=2)
    grid = mgs.Grid([15_000, 30_000], [4, 8, 16], 4096)
    dev = torch.device("cuda:0")
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(attrs).to(dev), torch.from_numpy(imp).to(dev))
    try:
        chosen, ms = mgs.mgs_autotune(ctx, scene, grid)
        assert 0 <= chosen < mgs.mgs_tile_config_count()
        assert ms[chosen] > 0 and ms[chosen] == ms[ms > 0].min()
    finally:
        mgs.mgs_set_tile_config(ctx, 4096, 3, -1)
        mgs.mgs_scene_destroy(scene)
