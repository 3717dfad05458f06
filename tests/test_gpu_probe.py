"""Bit-exact codes and histograms out of the fused cost kernel (Sec. III-D
quantiser, Sec. III-F entropy bound), against the CPU oracle.

mgs_build_cost_table_probe runs the same fused kernel as mgs_build_cost_table
and also writes every code and every histogram bin it counted.  For every
(ratio, channel, group, bit-width) the codes must equal the oracle's codes of
that group and the histogram must equal their bin counts, at each group size
with a probe kernel (1024, 2048, 4096, 16384), on synthetic channels and on
edge channels (constant, subnormal ranges, huge values, large offsets, exact
ties that overflow the 8-bit counters of the large bit-widths and force their
exact recount).  With the histograms pinned, the entropy bound is checked
against the FP64 oracle within the rounding of the L(h) table alone:
(non-empty bins + 1) * 2^-23 bits.  Needs a GB300."""
import numpy as np
import pytest

import oracle
from paper_2604_26799_gb300 import mgs, synth
from tests.test_gpu_cost import assert_table_close, edge_scene

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


def probe(ctx, attrs, imp, keep, bits, G):
    dev = torch.device("cuda:0")
    n, C = attrs.shape
    grid = mgs.Grid(keep, bits, G)
    L = mgs.mgs_table_layout_for(n, C, grid)
    bins = sum(1 << b for b in bits)
    ncodes = sum(C * len(bits) * int(k) for k in keep)
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(attrs).to(dev), torch.from_numpy(imp).to(dev))
    try:
        tab = torch.zeros(L.total_bytes, dtype=torch.uint8, device=dev)
        hist = torch.full((int(L.n_items) * bins,), -1, dtype=torch.int32, device=dev)
        codes = torch.full((ncodes,), -1, dtype=torch.int16, device=dev)
        mgs.mgs_build_cost_table_probe(ctx, scene, grid, tab, hist, codes)
        torch.cuda.synchronize()
        # the probe kernel gives the production kernel's table bit for bit
        plain = torch.zeros_like(tab)
        mgs.mgs_build_cost_table(ctx, scene, grid, plain)
        torch.cuda.synchronize()
        assert torch.equal(tab, plain)
    finally:
        mgs.mgs_scene_destroy(scene)
    return (mgs.table_views(tab.cpu().numpy(), L), L, hist.cpu().numpy().view(np.uint32).reshape(int(L.n_items), bins),
            codes.cpu().numpy().view(np.uint16))


def check_probe(attrs, imp, keep, bits, G, got, L, hist, codes):
    n, C = attrs.shape
    nb = len(bits)
    rank = oracle.rank(imp)
    _, order = oracle.morton(attrs)
    hoff = np.concatenate([[0], np.cumsum([1 << b for b in bits])])
    coff = 0
    for r, K in enumerate(keep):
        K = int(K)
        idx = order[oracle.kept(rank, order, K)]   # Gaussians of the kept set, Morton order
        assert idx.shape[0] == K
        ng = int(L.n_groups[r])
        block = codes[coff:coff + C * nb * K].reshape(C, nb, K)
        for c in range(C):
            col = attrs[idx, c]
            for g in range(ng):
                vals = col[g * G:(g + 1) * G]
                ref = oracle.group_cost(vals, bits, want_codes=True)
                item = int(L.item_begin[r]) + c * ng + g
                where = f"r={r} c={c} g={g}"
                assert np.array_equal(block[c, :, g * G:g * G + vals.shape[0]], ref["codes"]), where
                for k, b in enumerate(bits):
                    h = hist[item, hoff[k]:hoff[k + 1]]
                    want = np.bincount(ref["codes"][k], minlength=1 << b)
                    bad = np.flatnonzero(h != want)
                    assert bad.size == 0, f"{where} b={b}: bins {bad[:8]} got {h[bad[:8]]} want {want[bad[:8]]}"
                    # entropy: only the rounding of the 2^-22-bit L(h) table remains
                    bound = (np.count_nonzero(want) + 1) * 2.0 ** -23 + 1e-12 * abs(ref["hbits"][k]) + 1e-9
                    assert abs(got["hbits"][item, k] - ref["hbits"][k]) <= bound, (where, b)
        coff += C * nb * K
    assert coff == codes.shape[0]


@pytest.mark.parametrize("G,bits", [
    (4096, [2, 3, 4, 5, 6, 8, 10, 12, 14, 16]),
    (4096, [1, 7, 9, 11, 13, 15]),
    (2048, list(range(1, 17))),
    (1024, [1, 2, 6, 8, 12, 13, 16]),
    (16384, [2, 4, 8, 12, 16]),
])
def test_probe_codes_and_histograms_synthetic(ctx, G, bits):
    n = 40_000 if G == 16384 else 12_000
    attrs, imp = synth.make_scene(n, seed=77)
    attrs = np.ascontiguousarray(attrs[:, [0, 1, 2, 3, 10, 30, 51, 52, 55]])
    keep = np.array([1, 1500, n // 2 + 7, n], dtype=np.int64)
    got, L, hist, codes = probe(ctx, attrs, imp, keep, bits, G)
    check_probe(attrs, imp, keep, bits, G, got, L, hist, codes)
    ref = oracle.cost_table(attrs, imp, keep, bits, G)
    assert_table_close(got, ref, G, f"G={G}")


EDGE_BITS = [1, 2, 4, 6, 8, 10, 11, 12, 13, 14, 15, 16]
WORKLOAD_BITS = [2, 3, 4, 5, 6, 8, 10, 12, 14, 16]


# the workload's ten bit-widths at G = 4096 give every large option its own
# table (12, 14 and 16 bits as byte counters, counted with no barrier between
# them); the twelve edge bit-widths take region B one option at a time
@pytest.mark.parametrize("G,bits", [(1024, EDGE_BITS), (4096, EDGE_BITS), (4096, WORKLOAD_BITS)])
def test_probe_codes_and_histograms_edge(ctx, G, bits):
    attrs, imp = edge_scene()
    keep = np.array([1, 2, 999, 6000], dtype=np.int64)
    got, L, hist, codes = probe(ctx, attrs, imp, keep, bits, G)
    check_probe(attrs, imp, keep, bits, G, got, L, hist, codes)
    if G < 4096:
        return
    # the exact-ties channel overflows 8-bit counters at the byte-counted
    # bit-widths in a group of 4096: their counts come from the exact recount
    r = 3
    item = int(L.item_begin[r]) + 8 * int(L.n_groups[r])
    hoff = np.concatenate([[0], np.cumsum([1 << b for b in bits])])
    for b in (12, 16) if bits is WORKLOAD_BITS else (16,):
        k = bits.index(b)
        assert hist[item, hoff[k]:hoff[k + 1]].max() > 255, b


def test_probe_rejects_small_or_host_buffers(ctx):
    attrs, imp = synth.make_scene(3000, seed=5)
    dev = torch.device("cuda:0")
    grid = mgs.Grid(np.array([3000], dtype=np.int64), [4, 8], 1024)
    L = mgs.mgs_table_layout_for(3000, 59, grid)
    scene = mgs.mgs_scene_create(ctx, attrs, imp)
    try:
        tab = torch.zeros(L.total_bytes, dtype=torch.uint8, device=dev)
        need = int(L.n_items) * (16 + 256)
        with pytest.raises(mgs.MgsError) as e:
            mgs.mgs_build_cost_table_probe(ctx, scene, grid, tab,
                                           torch.zeros(need - 1, dtype=torch.int32, device=dev), None)
        assert e.value.status == -1
        with pytest.raises(mgs.MgsError) as e:
            mgs.mgs_build_cost_table_probe(ctx, scene, grid, tab, np.zeros(need, dtype=np.uint32), None)
        assert e.value.status == -1
        with pytest.raises(mgs.MgsError) as e:
            mgs.mgs_build_cost_table_probe(ctx, scene, grid, tab, None,
                                           torch.zeros(59 * 2 * 3000 - 1, dtype=torch.int16, device=dev))
        assert e.value.status == -1
    finally:
        mgs.mgs_scene_destroy(scene)
