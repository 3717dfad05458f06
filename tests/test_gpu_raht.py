"""RAHT (Sec. III-D) on the GPU against the FP64 oracle: the voxel count is
exact; the DC and every AC agree within the FP32 rounding of a chain of
orthonormal merges -- a few ulp per level of the size sqrt(w) * |x| of the
node a coefficient comes from (w the merge weight, |x| the largest magnitude
of a Gaussian under that node, both reported by the oracle per coefficient);
edge cases; full-size parity (needs a GB300)."""
import math

import numpy as np
import pytest

import oracle
from paper_2604_26799_gb300 import mgs, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CHANNELS = [3, 4, 5, 51, 52, 53, 54, 55, 56, 57]   # SH DC, opacity, log-scales, rotation


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_26799_gb300 import build
    build.build()
    c = mgs.mgs_create(0)
    yield c
    mgs.mgs_destroy(c)


def gpu_raht(ctx, attrs, channels, depth, imp=None, keep=0):
    dev = torch.device("cuda:0")
    imp = np.ones(attrs.shape[0], np.float32) if imp is None else imp
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(attrs).to(dev), torch.from_numpy(imp).to(dev))
    try:
        dc, ac, V = mgs.mgs_raht(ctx, scene, channels, depth, keep=keep)
        torch.cuda.synchronize()
        return dc, ac.cpu().numpy(), V
    finally:
        mgs.mgs_scene_destroy(scene)


def close(gpu, attrs, channels, depth, imp=None, keep=0):
    dc, ac, V = gpu
    rdc, rac, rV, rw, rr = oracle.raht(attrs, channels, depth, weights=True, importance=imp, keep=keep,
                                        ranges=True)
    assert V == rV and ac.shape == rac.shape
    S = np.abs(attrs[:, channels]).max(axis=0).astype(np.float64)      # |x| bound per channel
    tol = 3 * depth * 2.5e-7 + 1e-6                                     # ulp-scale per level
    assert np.all(np.abs(dc - rdc) <= tol * math.sqrt(V) * S + 1e-30)
    # each AC against the magnitude under its own node, not the channel's
    bound = tol * np.sqrt(rw.astype(np.float64))[:, None] * rr
    bad = np.argwhere(np.abs(ac.astype(np.float64) - rac) > bound)
    assert bad.size == 0, [(int(i), int(c), float(ac[i, c]), float(rac[i, c]), float(bound[i, c])) for i, c in bad[:5]]


@pytest.mark.parametrize("depth", [1, 4, 8, 12, 16, 21])
def test_raht_matches_oracle(ctx, depth):
    attrs, _ = synth.make_scene(20_000, seed=40 + depth)
    close(gpu_raht(ctx, attrs, CHANNELS, depth), attrs, CHANNELS, depth)


def test_raht_duplicates_and_edges(ctx):
    attrs, _ = synth.make_scene(4000, seed=7)
    dup = np.concatenate([attrs, attrs[:1000]], axis=0)        # 1000 voxels hold two Gaussians
    dup[4000:, 51] += 0.25
    close(gpu_raht(ctx, dup, CHANNELS, 14), dup, CHANNELS, 14)
    one = attrs[:1].copy()                                      # a single Gaussian: only a DC
    dc, ac, V = gpu_raht(ctx, one, [51], 10)
    assert V == 1 and ac.shape[0] == 0 and dc[0] == one[0, 51]
    flat = np.repeat(attrs[:1], 50, axis=0)                     # one voxel, 50 identical Gaussians
    flat[:, 51] = np.arange(50, dtype=np.float32)
    dc, ac, V = gpu_raht(ctx, flat, [51], 21)
    assert V == 1 and dc[0] == np.float32(np.arange(50).mean())
    with pytest.raises(mgs.MgsError):
        gpu_raht(ctx, attrs, [59], 10)
    with pytest.raises(mgs.MgsError):
        gpu_raht(ctx, attrs, [3], 22)


def test_raht_full_size(ctx):
    w = synth.SCENE
    attrs, _ = synth.make_scene(w.n, seed=w.seed)
    gpu = gpu_raht(ctx, attrs, CHANNELS, 16)
    close(gpu, attrs, CHANNELS, 16)
    dc, ac, V = gpu
    assert V > 1_000_000 and np.all(np.isfinite(ac))


@pytest.mark.parametrize("frac", [(1, 10), (1, 2), (9, 10)])
def test_raht_kept_set_matches_oracle(ctx, frac):
    attrs, imp = synth.make_scene(30_000, seed=17)
    keep = int(synth.keep_counts(30_000, [frac])[0])
    close(gpu_raht(ctx, attrs, CHANNELS, 14, imp=imp, keep=keep), attrs, CHANNELS, 14, imp=imp, keep=keep)
