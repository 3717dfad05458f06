"""The block coder on the GPU (Alg. 1's actual size S_a; Sec. III-G entropy
coding) against the oracle: the stream and every block size are byte-identical
for chosen configurations across group sizes (one rANS lane up to 32, ragged
last groups), every width 1..16, constant channels (R = 0), and at scene scale;
blocks of the GPU stream decode by the independent reader; argument errors
(needs a GB300)."""
import numpy as np
import pytest

import oracle
from paper_2604_26799_gb300 import mgs, synth
from tests import pins

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


def gpu_encode(ctx, attrs, imp, keep, G, q_bits, host_bits=False):
    dev = torch.device("cuda:0")
    C = attrs.shape[1]
    ng = oracle.n_groups(keep, G)
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(attrs).to(dev), torch.from_numpy(imp).to(dev))
    try:
        out = torch.empty(mgs.mgs_encode_bound(keep, G, C), dtype=torch.uint8, device=dev)
        sizes = torch.zeros((C, ng), dtype=torch.int32, device=dev)
        bits = q_bits if host_bits else torch.from_numpy(q_bits).to(dev)
        total = mgs.mgs_encode_config(ctx, scene, keep, G, bits, out, sizes)
        torch.cuda.synchronize()
    finally:
        mgs.mgs_scene_destroy(scene)
    return out[:total].cpu().numpy().tobytes(), sizes.cpu().numpy()


def assert_same(got, ref):
    s_gpu, sz_gpu = got
    s_ref, sz_ref = ref
    assert np.array_equal(sz_gpu, sz_ref.astype(np.int32)), np.argwhere(sz_gpu != sz_ref)[:5]
    assert len(s_gpu) == len(s_ref)
    if s_gpu != s_ref:
        a = np.frombuffer(s_gpu, np.uint8)
        b = np.frombuffer(s_ref, np.uint8)
        first = int(np.argmax(a != b))
        raise AssertionError(f"streams differ first at byte {first}")


@pytest.mark.parametrize("G,n,keep_frac", [(100, 3000, 0.7), (512, 5000, 1.0), (1000, 20000, 0.55),
                                           (4096, 30000, 1.0), (16384, 40000, 0.9)])
def test_encode_matches_oracle(ctx, G, n, keep_frac):
    attrs, imp = synth.make_scene(n, seed=G)
    attrs[:, 7] = 1.25                       # constant channel: R = 0 in every group
    keep = int(n * keep_frac)
    ng = oracle.n_groups(keep, G)
    rng = np.random.default_rng(G)
    q_bits = rng.integers(1, 17, size=(attrs.shape[1], ng)).astype(np.uint8)
    got = gpu_encode(ctx, attrs, imp, keep, G, q_bits)
    ref = oracle.encode_config(attrs, imp, keep, G, q_bits)
    assert_same(got, ref)
    assert (got[1][7] == 9).all()


@pytest.mark.parametrize("b", [1, 2, 5, 8, 12, 13, 16])
def test_encode_every_width(ctx, b):
    """One width everywhere: raw and rANS blocks, one and several histogram windows."""
    n, G = 20_000, 4096
    attrs, imp = synth.make_scene(n, seed=40 + b)
    keep = 17_000
    q_bits = np.full((attrs.shape[1], oracle.n_groups(keep, G)), b, dtype=np.uint8)
    got = gpu_encode(ctx, attrs, imp, keep, G, q_bits)
    ref = oracle.encode_config(attrs, imp, keep, G, q_bits)
    assert_same(got, ref)
    modes = set()
    stream, sizes = got
    at = 0
    for c in range(attrs.shape[1]):
        for g in range(sizes.shape[1]):
            if sizes[c, g] > 9:
                modes.add(stream[at + 9])
            at += int(sizes[c, g])
    if b <= 8:
        assert 1 in modes


def test_encode_stream_decodes(ctx):
    n, G, keep = 6000, 1024, 5000
    attrs, imp = synth.make_scene(n, seed=3)
    ng = oracle.n_groups(keep, G)
    q_bits = np.random.default_rng(3).integers(1, 17, size=(attrs.shape[1], ng)).astype(np.uint8)
    stream, sizes = gpu_encode(ctx, attrs, imp, keep, G, q_bits, host_bits=True)
    codes, _ = oracle.quantize(attrs, imp, keep, G, q_bits)
    flat = sizes.reshape(-1)
    offs = np.concatenate([[0], np.cumsum(flat)])
    for c in (0, 5, 30, 58):
        for g in range(ng):
            i = c * ng + g
            blk = stream[offs[i]:offs[i + 1]]
            ln = min(G, keep - g * G)
            got, b, _, _, used, _ = pins.read_block_py(blk, ln)
            assert used == len(blk) and b == q_bits[c, g]
            assert np.array_equal(np.asarray(got, np.uint16), codes[c, g * G:g * G + ln])


def test_encode_scene_scale(ctx):
    """Scene scale (5.27 M Gaussians, 59 channels, G = 4096, half kept) with
    widths drawn around 8 bits: every block size and byte equal to the oracle's."""
    w = synth.SCENE
    attrs, imp = synth.make_scene(w.n, seed=w.seed)
    keep, G = w.n // 2, 4096
    ng = oracle.n_groups(keep, G)
    rng = np.random.default_rng(9)
    q_bits = np.clip(np.rint(rng.normal(8, 3, size=(attrs.shape[1], ng))), 1, 16).astype(np.uint8)
    got = gpu_encode(ctx, attrs, imp, keep, G, q_bits)
    ref = oracle.encode_config(attrs, imp, keep, G, q_bits)
    assert_same(got, ref)


def test_encode_errors(ctx):
    n, G, keep = 3000, 512, 2000
    attrs, imp = synth.make_scene(n, seed=4)
    dev = torch.device("cuda:0")
    C = attrs.shape[1]
    ng = oracle.n_groups(keep, G)
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(attrs).to(dev), torch.from_numpy(imp).to(dev))
    try:
        bits = np.full((C, ng), 6, dtype=np.uint8)
        total = mgs.mgs_encode_config(ctx, scene, keep, G, bits)          # measure only
        small = torch.empty(total - 1, dtype=torch.uint8, device=dev)
        with pytest.raises(mgs.MgsError) as e:
            mgs.mgs_encode_config(ctx, scene, keep, G, bits, small)
        assert e.value.status == -1
        full = torch.empty(total, dtype=torch.uint8, device=dev)
        assert mgs.mgs_encode_config(ctx, scene, keep, G, bits, full) == total
        bad = bits.copy()
        bad[3, 1] = 17
        with pytest.raises(mgs.MgsError) as e:
            mgs.mgs_encode_config(ctx, scene, keep, G, bad)
        assert e.value.status == -1
        bad[3, 1] = 0
        with pytest.raises(mgs.MgsError):
            mgs.mgs_encode_config(ctx, scene, keep, G, bad)
        with pytest.raises(mgs.MgsError):
            mgs.mgs_encode_config(ctx, scene, n + 1, G, bits)
    finally:
        mgs.mgs_scene_destroy(scene)
    ref, _ = oracle.encode_config(attrs, imp, keep, G, np.full((C, ng), 6, np.uint8))
    assert total == len(ref)
