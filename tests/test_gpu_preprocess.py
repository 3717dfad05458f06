"""Preprocessing (Sec. III-A view-independent importance, Sec. III-D Euler
replacement) on the GPU against the oracle: copied channels bit-exact, V_q
(an exact order statistic of the device's FP32 volumes) and I_g within FP32
rounding of the FP64 oracle, Euler angles (FP32 where well-conditioned,
FP64 near gimbal lock) directly and through the decoder's rotation matrix;
edge cases; and the cost table of the preprocessed
58-channel scene (needs a GB300)."""
import math

import numpy as np
import pytest

import oracle
from paper_2604_26799_gb300 import mgs, synth
from tests import pins
from tests.test_gpu_cost import assert_table_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# angles: FP32 where |sin(theta)| <= 0.95 (a few ulp of pi, conditioning <= 3.2),
# FP64 rounded once near gimbal lock
ANGLE_TOL = 2e-6
MATRIX_TOL = 3e-6
IMP_RTOL = 2e-5


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_26799_gb300 import build
    build.build()
    c = mgs.mgs_create(0)
    yield c
    mgs.mgs_destroy(c)


def run(ctx, attrs, imp, beta):
    dev = torch.device("cuda:0")
    out, ig, vq = mgs.mgs_preprocess(ctx, torch.from_numpy(attrs).to(dev), torch.from_numpy(imp).to(dev), beta)
    torch.cuda.synchronize()
    return out.cpu().numpy(), ig.cpu().numpy(), vq


def wrap(d):
    return (d + math.pi) % (2 * math.pi) - math.pi


def compare(attrs, out, ig, vq, ref, sample=None):
    r_out, r_ig, r_vq = ref
    rows = np.arange(attrs.shape[0]) if sample is None else sample
    assert np.array_equal(out[rows, :55], attrs[rows, :55])
    assert abs(vq - r_vq) <= 2e-6 * r_vq
    assert np.allclose(ig[rows], r_ig[rows], rtol=IMP_RTOL, atol=0)
    e_gpu = out[rows, 55:58].astype(np.float64)
    e_ref = r_out[rows, 55:58].astype(np.float64)
    for k in range(0, len(rows), max(1, len(rows) // 2000)):
        assert np.allclose(pins.euler_matrix(e_gpu[k]), pins.euler_matrix(e_ref[k]), atol=MATRIX_TOL), rows[k]
    # well-conditioned rows in FP32, the others in FP64 rounded once: the angles
    # agree everywhere, gimbal lock included
    diff = np.abs(wrap(e_gpu - e_ref))
    bad = np.argwhere(diff > ANGLE_TOL)
    assert bad.size == 0, [(rows[i], c, e_gpu[i], e_ref[i]) for i, c in bad[:5]]


def special_scene(n=20_000, seed=31):
    attrs, imp = synth.make_scene(n, seed=seed)
    q = attrs[:, 55:59]
    q[0] = [0, 0, 0, 0]                                   # zero quaternion -> zero angles
    h = math.pi / 4
    q[1] = [math.cos(h), 0, math.sin(h), 0]               # theta = pi/2 (gimbal lock)
    q[2] = [math.cos(h), 0, -math.sin(h), 0]              # theta = -pi/2
    q[3] = [0.5, 0.5, 0.5, 0.5]
    q[4] = [-3.0, 0.0, 0.0, 0.0]                          # unnormalised, sign-flipped identity
    attrs[5:50, 52:55] = attrs[5, 52:55]                  # a run of equal volumes
    return attrs, imp


@pytest.mark.parametrize("beta", [0.0, 0.5, 1.0, 3.0])
def test_preprocess_matches_oracle(ctx, beta):
    attrs, imp = special_scene()
    out, ig, vq = run(ctx, attrs, imp, beta)
    ref = oracle.preprocess(attrs, imp, beta)
    compare(attrs, out, ig, vq, ref)
    assert np.array_equal(out[0, 55:58], np.zeros(3, np.float32))
    assert np.allclose(out[4, 55:58], 0.0, atol=1e-7)
    if beta == 0.0:
        assert np.array_equal(ig, imp)


def test_preprocess_full_size(ctx):
    w = synth.SCENE
    attrs, imp = synth.make_scene(w.n, seed=w.seed)
    out, ig, vq = run(ctx, attrs, imp, 1.0)
    ref = oracle.preprocess(attrs, imp, 1.0)
    rows = np.random.default_rng(2).choice(w.n, 200_000, replace=False)
    compare(attrs, out, ig, vq, ref, sample=np.sort(rows))
    assert np.allclose(ig, ref[1], rtol=IMP_RTOL, atol=0)


def test_preprocess_edges(ctx):
    attrs, imp = synth.make_scene(3, seed=5)
    out, ig, vq = run(ctx, attrs[:1].copy(), imp[:1].copy(), 2.0)   # n = 1: V_q is that volume
    assert ig[0] == imp[0]
    two = attrs[:2].copy()
    two[:, 52:55] = [[-4.0, -4.0, -4.0], [-3.0, -4.0, -4.0]]
    out, ig, vq = run(ctx, two, imp[:2].copy(), 1.0)                 # rank floor(0.9) = 0: the smaller
    ref = oracle.preprocess(two, imp[:2], 1.0)
    assert abs(vq - ref[2]) <= 2e-6 * ref[2] and ig[0] == imp[0] and ig[1] == imp[1]
    same = np.repeat(attrs[:1], 64, axis=0)
    out, ig, vq = run(ctx, same, np.ones(64, np.float32), 5.0)       # equal volumes: V_norm = 1 exactly
    assert np.all(ig == 1.0)
    dev = torch.device("cuda:0")
    bad = attrs.copy()
    bad[1, 57] = np.nan
    with pytest.raises(mgs.MgsError) as e:
        mgs.mgs_preprocess(ctx, torch.from_numpy(bad).to(dev), torch.from_numpy(imp).to(dev), 1.0)
    assert e.value.status == -2
    with pytest.raises(mgs.MgsError) as e:
        mgs.mgs_preprocess(ctx, torch.from_numpy(attrs).to(dev), torch.from_numpy(imp).to(dev), -1.0)
    assert e.value.status == -1


def test_cost_table_of_preprocessed_scene(ctx):
    """Preprocess, then build the 58-channel cost table; the oracle's table of the
    device's preprocessed arrays is matched with the usual parity bar."""
    n, G = 30_000, 1024
    attrs, imp = synth.make_scene(n, seed=12)
    dev = torch.device("cuda:0")
    out_d, ig_d, _ = mgs.mgs_preprocess(ctx, torch.from_numpy(attrs).to(dev), torch.from_numpy(imp).to(dev), 1.0)
    keep = synth.keep_counts(n, [(1, 4), (3, 4), (1, 1)])
    bits = [2, 4, 8, 12, 16]
    grid = mgs.Grid(keep, bits, G)
    scene = mgs.mgs_scene_create(ctx, out_d, ig_d)
    try:
        L = mgs.mgs_table_layout_for(n, 58, grid)
        tab = torch.empty(L.total_bytes, dtype=torch.uint8, device=dev)
        mgs.mgs_build_cost_table(ctx, scene, grid, tab)
        torch.cuda.synchronize()
        got = mgs.table_views(tab.cpu().numpy(), L)
    finally:
        mgs.mgs_scene_destroy(scene)
    ref = oracle.cost_table(out_d.cpu().numpy(), ig_d.cpu().numpy(), keep, bits, G)
    assert_table_close(got, ref, G)
