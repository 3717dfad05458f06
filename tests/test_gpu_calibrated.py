"""Alg. 1 with real compression (the S_Delta calibration loop of Eq.
(eq:size_estim)) on the GPU, against a step-by-step restatement of the loop:
the oracle's block coder gives every actual size S_a and the host solver (the
same answers as the device solver, bit for bit) solves each one-ratio ILP.
Every ratio's status, round count, S_a, S_Delta and Omega, and the chosen
widths, must agree; converged ratios meet the tolerance; the tau pick is the
smallest Omega among them (needs a GB300)."""
import ctypes

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


def ratio_view(lay, r):
    """The one-ratio view of a cost table: same buffer, offsets at ratio r's items."""
    v = mgs.mgs_table_layout()
    ctypes.memmove(ctypes.addressof(v), ctypes.addressof(lay), ctypes.sizeof(lay))
    ib = int(lay.item_begin[r])
    items = int(lay.item_begin[r + 1]) - ib
    e = ib * lay.n_bits
    v.n_ratios, v.n_items = 1, items
    v.item_begin[0], v.item_begin[1] = 0, items
    v.n_groups[0] = lay.n_groups[r]
    v.off_sse += 8 * e
    v.off_l1 += 8 * e
    v.off_hbits += 8 * e
    v.off_linf += 4 * e
    v.off_count += 4 * ib
    v.off_vmin += 4 * ib
    v.off_vmax += 4 * ib
    return v


def restated(attrs, imp, keep, bits, G, host_tab, lay, S_T, tol, max_rounds, init_bits, opts):
    """Alg. 1 step by step: compress at init_bits; skip if 2 S_a < S_T; then
    S_Delta = S_a - estimate(Q) without S_Delta, solve, compress, until
    |S_a - S_T| / S_T < tol."""
    C = attrs.shape[1]
    v = mgs.table_views(host_tab, lay)
    rec = []
    for r, K in enumerate(keep):
        ng = oracle.n_groups(int(K), G)
        m = C * ng
        ib = int(lay.item_begin[r])
        q = np.full((C, ng), init_bits, np.uint8)
        S_a = len(oracle.encode_config(attrs, imp, int(K), G, q)[0]) + opts.const_bytes
        rounds = 1
        est0 = opts.meta_bytes_per_group * m + opts.const_bytes    # summed in item order
        if opts.rate_model == mgs.MGS_RATE_FIXED:
            for x in v["cnt"][ib:ib + m].tolist():
                est0 += float(x) * init_bits / 8.0
        else:
            k0 = list(bits).index(init_bits)
            for x in v["hbits"][ib:ib + m, k0].tolist():
                est0 += x / 8.0
        if 2 * S_a < S_T:
            rec.append(dict(status=1, rounds=rounds, actual=S_a, delta=0.0, obj=0.0, bits=None))
            continue
        status, delta, obj, fb = 2, 0.0, 0.0, None
        vl = ratio_view(lay, r)
        vg = mgs.Grid(np.array([K], np.int64), list(bits), G)
        for _ in range(max_rounds):
            d = S_a - est0
            so = mgs.solve_opts(rate_model=opts.rate_model, norm=opts.norm, const_bytes=opts.const_bytes,
                                meta_bytes_per_group=opts.meta_bytes_per_group, delta_bytes=d)
            sol = mgs.mgs_solve_budgets(host_tab, vl, vg, [S_T], so)[0]
            if sol["r_index"] < 0:
                status = -1
                break
            fb = np.asarray(bits, np.uint8)[sol["choice"]].reshape(C, ng)
            est0 = sol["est_bytes"] - d
            delta, obj = d, sol["objective"]
            S_a = len(oracle.encode_config(attrs, imp, int(K), G, fb)[0]) + opts.const_bytes
            rounds += 1
            if abs(S_a - S_T) / S_T < tol:
                status = 0
                break
        rec.append(dict(status=status, rounds=rounds, actual=S_a, delta=delta, obj=obj, bits=fb))
    return rec


def setup(ctx, n, keep, bits, G, seed):
    attrs, imp = synth.make_scene(n, seed=seed)
    dev = torch.device("cuda:0")
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(attrs).to(dev), torch.from_numpy(imp).to(dev))
    grid = mgs.Grid(keep, bits, G)
    lay = mgs.mgs_table_layout_for(n, attrs.shape[1], grid)
    tab = torch.empty(lay.total_bytes, dtype=torch.uint8, device=dev)
    mgs.mgs_build_cost_table(ctx, scene, grid, tab)
    torch.cuda.synchronize()
    return attrs, imp, scene, grid, lay, tab


@pytest.mark.parametrize("rate_model", [1, 0])
def test_calibrated_search_matches_restatement(ctx, rate_model):
    n, G = 40_000, 1024
    keep = synth.keep_counts(n, [(1, 5), (2, 5), (3, 5), (4, 5), (1, 1)])
    bits = [2, 3, 4, 6, 8, 10, 12, 16]
    attrs, imp, scene, grid, lay, tab = setup(ctx, n, keep, bits, G, seed=17)
    try:
        C = attrs.shape[1]
        full8 = mgs.mgs_encode_config(ctx, scene, int(keep[-1]), G,
                                      np.full((C, oracle.n_groups(int(keep[-1]), G)), 8, np.uint8))
        S_T = 0.55 * full8
        opts = mgs.solve_opts(rate_model=rate_model, const_bytes=1000.0)
        got = mgs.mgs_search_calibrated(ctx, scene, grid, tab, lay, S_T, tolerance=0.05, max_rounds=8,
                                        init_bits=8, opts=opts)
        ref = restated(attrs, imp, keep, bits, G, tab.cpu().numpy(), lay, S_T, 0.05, 8, 8, opts)
    finally:
        mgs.mgs_scene_destroy(scene)
    for r, e in enumerate(ref):
        assert got["ratio_status"][r] == e["status"], (r, got["ratio_status"], [x["status"] for x in ref])
        assert got["ratio_rounds"][r] == e["rounds"], r
        assert got["ratio_actual"][r] == e["actual"], r
        assert got["ratio_delta"][r] == e["delta"], r
        assert got["ratio_objective"][r] == e["obj"], r
        if e["status"] == 0:
            assert abs(e["actual"] - S_T) / S_T < 0.05
    conv = [r for r, e in enumerate(ref) if e["status"] == 0]
    assert conv, [x["status"] for x in ref]
    best = min(conv, key=lambda r: (ref[r]["obj"], -r))
    assert got["r_index"] == best
    assert np.array_equal(got["bits"], ref[best]["bits"])
    assert got["actual_bytes"] == ref[best]["actual"]
    assert ref[0]["status"] == 1          # a fifth of the scene at 8 bits is under half the budget


def test_calibrated_search_errors(ctx):
    n, G = 8000, 512
    keep = synth.keep_counts(n, [(1, 2), (1, 1)])
    attrs, imp, scene, grid, lay, tab = setup(ctx, n, keep, [2, 4, 6], G, seed=5)
    try:
        with pytest.raises(mgs.MgsError) as e:       # entropy estimate needs init_bits in the grid
            mgs.mgs_search_calibrated(ctx, scene, grid, tab, lay, 1e5, init_bits=8,
                                      opts=mgs.solve_opts(rate_model=mgs.MGS_RATE_ENTROPY))
        assert e.value.status == -1
        with pytest.raises(mgs.MgsError):             # host table
            mgs.mgs_search_calibrated(ctx, scene, grid, tab.cpu().numpy(), lay, 1e5)
        res = mgs.mgs_search_calibrated(ctx, scene, grid, tab, lay, 10.0)   # nothing fits
        assert res["r_index"] == -1 and (res["ratio_status"] == -1).all()
    finally:
        mgs.mgs_scene_destroy(scene)
