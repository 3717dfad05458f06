"""Parity at the full workload sizes, in the launch configuration bench.py
times (a persistent plan over the whole grid): sampled (ratio, channel, group)
items against the oracle computed one by one, invariants over every item, and
bit-exact Morton codes (needs a GB300)."""
import numpy as np
import pytest

import oracle
from paper_2604_26799_gb300 import mgs, synth
from tests.test_gpu_cost import assert_table_close

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


def plan_table(ctx, attrs, imp, w: synth.Workload, want_morton=False):
    dev = torch.device("cuda:0")
    grid = mgs.Grid(w.keep(), list(w.bits), w.group_size)
    st = torch.cuda.Stream()
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(attrs).to(dev), torch.from_numpy(imp).to(dev), stream=st)
    morton = None
    try:
        L = mgs.mgs_table_layout_for(w.n, attrs.shape[1], grid)
        tab = torch.empty(L.total_bytes, dtype=torch.uint8, device=dev)
        with torch.cuda.stream(st):
            plan = mgs.mgs_plan_create(ctx, [scene], grid, [tab], stream=st)
            mgs.mgs_plan_launch(plan, st)
            st.synchronize()
            mgs.mgs_plan_destroy(plan)
        if want_morton:
            codes = torch.empty(w.n, dtype=torch.int64, device=dev)
            order = torch.empty(w.n, dtype=torch.int32, device=dev)
            mgs.mgs_scene_morton(scene, codes, order)
            torch.cuda.synchronize()
            morton = (codes.cpu().numpy().view(np.uint64), order.cpu().numpy().astype(np.int64))
        host = tab.cpu().numpy()
    finally:
        mgs.mgs_scene_destroy(scene)
    return mgs.table_views(host, L), L, morton


def check_sampled(attrs, imp, w, got, L, n_samples, seed):
    rank = oracle.rank(imp)
    _, order = oracle.morton(attrs)
    C = attrs.shape[1]
    rng = np.random.default_rng(seed)
    keep = w.keep()
    for r in range(len(keep)):
        kept = oracle.kept(rank, order, int(keep[r]))
        ng = int(L.n_groups[r])
        gs = set(rng.integers(0, ng, size=n_samples).tolist()) | {ng - 1}   # include the ragged tail
        for g in sorted(gs):
            for c in sorted(set(rng.integers(0, C, size=3).tolist())):
                vals = attrs[order[kept[g * w.group_size:(g + 1) * w.group_size]], c]
                ref = oracle.group_cost(vals, list(w.bits))
                item = int(L.item_begin[r] + c * ng + g)
                one = {k: got[k][item:item + 1] for k in ("sse", "l1", "linf", "hbits", "cnt", "vmin", "vmax")}
                refd = dict(sse=ref["sse"][None], l1=ref["l1"][None], linf=ref["linf"][None],
                            hbits=ref["hbits"][None], cnt=np.array([vals.shape[0]], dtype=np.int32),
                            vmin=np.array([ref["vmin"]], dtype=np.float32),
                            vmax=np.array([ref["vmax"]], dtype=np.float32))
                assert_table_close(one, refd, w.group_size, f"r={r} c={c} g={g}")


def check_invariants(got, L, w, C):
    keep = w.keep()
    bits = np.asarray(w.bits, dtype=np.float64)
    for r in range(len(keep)):
        ng = int(L.n_groups[r])
        cnt = got["cnt"][int(L.item_begin[r]):int(L.item_begin[r + 1])].reshape(C, ng)
        assert np.all(cnt.sum(axis=1) == keep[r])
        assert np.all(cnt[:, :-1] == w.group_size)
    n = got["cnt"].astype(np.float64)[:, None]
    assert np.all(got["hbits"] >= -1e-6) and np.all(got["hbits"] <= n * np.minimum(bits[None, :], np.log2(np.maximum(n, 1))) + 1e-3)
    assert np.all(got["sse"] >= 0) and np.all(got["l1"] >= 0)
    S = (got["vmax"].astype(np.float64) - got["vmin"].astype(np.float64))[:, None] / 2.0 ** bits[None, :]
    mag = np.maximum(np.abs(got["vmin"]), np.abs(got["vmax"])).astype(np.float64)[:, None]
    assert np.all(got["linf"] <= 1.5 * S * (1 + 1e-6) + 4e-7 * mag)
    assert np.all(got["sse"] <= n * got["linf"].astype(np.float64) ** 2 * (1 + 1e-9) + 1e-300)


def test_scene_scale_sampled_parity(ctx):
    w = synth.SCENE
    attrs, imp = synth.make_scene(w.n, seed=w.seed)
    got, L, _ = plan_table(ctx, attrs, imp, w)
    check_invariants(got, L, w, attrs.shape[1])
    check_sampled(attrs, imp, w, got, L, n_samples=3, seed=1)


def test_large_grid_morton_and_sampled_parity(ctx):
    w = synth.LARGE
    attrs, imp = synth.make_scene(w.n, seed=w.seed)
    got, L, (codes, order) = plan_table(ctx, attrs, imp, w, want_morton=True)
    ref_codes, ref_order = oracle.morton(attrs)
    assert np.array_equal(codes, ref_codes)       # 21-bit-per-axis codes, bit-exact
    assert np.array_equal(order, ref_order)
    check_invariants(got, L, w, attrs.shape[1])
    check_sampled(attrs, imp, w, got, L, n_samples=1, seed=2)
