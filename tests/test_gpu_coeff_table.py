"""Cost tables of coefficient arrays (the RAHT ACs of Sec. III-D are the
quantised signal) against the oracle's group cost on the same arrays: groups
are consecutive runs of the array in its own order, ratios take prefixes;
validation errors (needs a GB300)."""
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


def oracle_table(coeffs, keep, bits, G):
    """Items [r][c][g] of consecutive groups of the first keep[r] rows."""
    m, C = coeffs.shape
    out = {k: [] for k in ("sse", "l1", "linf", "hbits", "cnt", "vmin", "vmax")}
    for K in keep:
        for c in range(C):
            for g0 in range(0, int(K), G):
                vals = coeffs[g0:min(g0 + G, int(K)), c]
                r = oracle.group_cost(vals, bits)
                for k in ("sse", "l1", "linf", "hbits"):
                    out[k].append(r[k])
                out["cnt"].append(len(vals))
                out["vmin"].append(r["vmin"])
                out["vmax"].append(r["vmax"])
    return dict(sse=np.array(out["sse"]), l1=np.array(out["l1"]), linf=np.array(out["linf"], np.float32),
                hbits=np.array(out["hbits"]), cnt=np.array(out["cnt"], np.int32),
                vmin=np.array(out["vmin"], np.float32), vmax=np.array(out["vmax"], np.float32))


def gpu_table(ctx, coeffs_d, keep, bits, G):
    m, C = coeffs_d.shape
    grid = mgs.Grid(np.asarray(keep, np.int64), bits, G)
    L = mgs.mgs_table_layout_for(m, C, grid)
    tab = torch.empty(L.total_bytes, dtype=torch.uint8, device=coeffs_d.device)
    mgs.mgs_build_cost_table_coeffs(ctx, coeffs_d, grid, tab)
    torch.cuda.synchronize()
    return mgs.table_views(tab.cpu().numpy(), L)


@pytest.mark.parametrize("G", [4096, 1000, 64])
def test_random_coefficients_with_prefixes(ctx, G):
    rng = np.random.default_rng(G)
    m, C = 23_457, 11
    coeffs = (rng.laplace(0, 0.1, (m, C)) * rng.uniform(0.01, 10, C)).astype(np.float32)
    coeffs[:, 3] = 1.5                                   # a constant channel: degenerate groups
    keep = [m // 3, m]
    bits = [1, 2, 4, 8, 12, 16]
    got = gpu_table(ctx, torch.from_numpy(coeffs).cuda(), keep, bits, G)
    assert_table_close(got, oracle_table(coeffs, keep, bits, G), G)


def test_raht_ac_table(ctx):
    """The AC coefficients of a scene's RAHT, tabulated as they come out of mgs_raht."""
    n = 40_000
    attrs, imp = synth.make_scene(n, seed=21)
    dev = torch.device("cuda:0")
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(attrs).to(dev), torch.from_numpy(imp).to(dev))
    try:
        _, ac, V = mgs.mgs_raht(ctx, scene, [3, 4, 5, 51, 52, 53, 54], 16, keep=n // 2)
        ac = ac.contiguous()
        bits = [2, 4, 6, 8, 10, 12, 14, 16]
        got = gpu_table(ctx, ac, [V - 1], bits, 1024)
    finally:
        mgs.mgs_scene_destroy(scene)
    assert_table_close(got, oracle_table(ac.cpu().numpy(), [V - 1], bits, 1024), 1024)


def test_coefficient_validation(ctx):
    c = torch.zeros((100, 3), dtype=torch.float32, device="cuda")
    c[7, 1] = float("nan")
    with pytest.raises(mgs.MgsError) as e:
        gpu_table(ctx, c, [100], [4], 16)
    assert e.value.status == -2
    c[7, 1] = 3e38
    c[8, 1] = -3e38
    with pytest.raises(mgs.MgsError) as e:
        gpu_table(ctx, c, [100], [4], 16)
    assert e.value.status == -3
