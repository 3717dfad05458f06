"""mgs_quantize_groups_noalloc (static device scratch, no allocation) against
mgs_quantize_groups, through the C ABI, on two calls in a row.

Some callers cannot allocate device memory while they run (a process whose
device memory belongs to another framework's capped allocator, a real-time
encoder thread that may not block or synchronise the device).  The
allocation-free entry point must give them exactly what the allocating one
gives everybody else.  This file is collected last so that a run stopping at
the first failure has already run every other test; it also passes alone in a
fresh process.
"""
import numpy as np
import pytest

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


def _codes(fn, ctx, scene, keep, G, qbits, C, dev):
    ng = (keep + G - 1) // G
    codes = torch.full((C, keep), -1, dtype=torch.int16, device=dev)
    mm = torch.full((C, ng, 2), float("nan"), dtype=torch.float32, device=dev)
    fn(ctx, scene, keep, G, qbits, codes, mm)
    torch.cuda.synchronize()
    return codes.cpu().numpy().view(np.uint16), mm.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice(ctx):
    dev = torch.device("cuda:0")
    n = 60_000
    attrs, imp = synth.make_scene(n, seed=31)
    C = attrs.shape[1]
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(attrs).to(dev), torch.from_numpy(imp).to(dev))
    try:
        rng = np.random.default_rng(4)
        # two calls in a row with different sizes: the second must not see the first's scratch
        for keep, G in ((41_000, 4096), (17_777, 1000)):
            ng = (keep + G - 1) // G
            qbits = torch.from_numpy(rng.integers(1, 17, size=(C, ng)).astype(np.uint8)).to(dev)
            ref_codes, ref_mm = _codes(mgs.mgs_quantize_groups, ctx, scene, keep, G, qbits, C, dev)
            got_codes, got_mm = _codes(mgs.mgs_quantize_groups_noalloc, ctx, scene, keep, G, qbits, C, dev)
            assert np.array_equal(got_codes, ref_codes)
            assert np.array_equal(got_mm, ref_mm)
    finally:
        mgs.mgs_scene_destroy(scene)


def test_noalloc_rejects_sizes_beyond_its_scratch(ctx):
    dev = torch.device("cuda:0")
    n = 1000
    attrs, imp = synth.make_scene(n, seed=32)
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(attrs).to(dev), torch.from_numpy(imp).to(dev))
    try:
        bits = torch.ones((attrs.shape[1], 1), dtype=torch.uint8, device=dev)
        codes = torch.empty((attrs.shape[1], n), dtype=torch.int16, device=dev)
        mm = torch.empty((attrs.shape[1], 1, 2), dtype=torch.float32, device=dev)
        with pytest.raises(mgs.MgsError) as e:
            mgs.mgs_quantize_groups_noalloc(ctx, scene, n + 1, 4096, bits, codes, mm)
        assert e.value.status == -1
    finally:
        mgs.mgs_scene_destroy(scene)


def _limit(name: str) -> int:
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mgs.h")).read()
    return int(re.search(rf"#define {name} (\d+)", hdr).group(1))


def test_noalloc_at_and_beyond_its_kept_limit(ctx):
    """keep == MGS_NOALLOC_MAX_KEEP fills the static kept array and still matches
    the allocating entry point bit for bit; one more kept Gaussian is refused."""
    dev = torch.device("cuda:0")
    max_keep = _limit("MGS_NOALLOC_MAX_KEEP")
    n = max_keep + 1000
    attrs, imp = synth.make_scene(n, seed=33)
    attrs = np.ascontiguousarray(attrs[:, :8])
    C = attrs.shape[1]
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(attrs).to(dev), torch.from_numpy(imp).to(dev))
    try:
        G = 4096
        ng = (max_keep + G - 1) // G
        rng = np.random.default_rng(6)
        qbits = torch.from_numpy(rng.integers(1, 17, size=(C, ng)).astype(np.uint8)).to(dev)
        ref_codes, ref_mm = _codes(mgs.mgs_quantize_groups, ctx, scene, max_keep, G, qbits, C, dev)
        got_codes, got_mm = _codes(mgs.mgs_quantize_groups_noalloc, ctx, scene, max_keep, G, qbits, C, dev)
        assert np.array_equal(got_codes, ref_codes)
        assert np.array_equal(got_mm, ref_mm)
        codes = torch.empty((C, max_keep + 1), dtype=torch.int16, device=dev)
        mm = torch.empty((C, ng + 1, 2), dtype=torch.float32, device=dev)
        qb = torch.ones((C, ng + 1), dtype=torch.uint8, device=dev)
        with pytest.raises(mgs.MgsError) as e:
            mgs.mgs_quantize_groups_noalloc(ctx, scene, max_keep + 1, G, qb, codes, mm)
        assert e.value.status == -1 and "at most" in str(e.value)
    finally:
        mgs.mgs_scene_destroy(scene)


def test_noalloc_refuses_a_scene_beyond_its_tile_counts(ctx):
    dev = torch.device("cuda:0")
    n = _limit("MGS_NOALLOC_MAX_SCENE") + 1
    rng = np.random.default_rng(7)
    attrs = rng.random((n, 3), dtype=np.float32)
    imp = rng.random(n, dtype=np.float32)
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(attrs).to(dev), torch.from_numpy(imp).to(dev))
    try:
        bits = torch.ones((3, 1), dtype=torch.uint8, device=dev)
        codes = torch.empty((3, 100), dtype=torch.int16, device=dev)
        mm = torch.empty((3, 1, 2), dtype=torch.float32, device=dev)
        with pytest.raises(mgs.MgsError) as e:
            mgs.mgs_quantize_groups_noalloc(ctx, scene, 100, 4096, bits, codes, mm)
        assert e.value.status == -1 and "at most" in str(e.value)
    finally:
        mgs.mgs_scene_destroy(scene)
