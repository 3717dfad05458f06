"""Vector quantisation of the 1+D SH coefficients (Sec. III-D) on the GPU
against the oracle: assignments and scores bit-exact for D from 3 to 64,
ragged vector counts and codebook tiles, K = 1; mini-batch k-means codebooks,
counts and every batch's assignment bit-exact over several batches; at scene
scale (5.27 M x 45, K = 4096) one full mini-batch and sampled final
assignments; retention of top-ranked vectors; argument errors (needs a
GB300)."""
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


@pytest.fixture(params=["tensor", "cuda"])
def path(ctx, request):
    """Both score paths: tcgen05 with exact re-scores, and the CUDA cores."""
    mgs.mgs_vq_set_tensor_cores(ctx, request.param == "tensor")
    mgs.mgs_vq_stats(ctx)
    yield request.param
    mgs.mgs_vq_set_tensor_cores(ctx, True)


def sh_rows(n, seed, D=45):
    attrs, _ = synth.make_scene(n, seed=seed)
    x = np.ascontiguousarray(attrs[:, 6:51])
    if D <= 45:
        return np.ascontiguousarray(x[:, :D])
    return np.ascontiguousarray(np.concatenate([x, attrs[:, :D - 45]], axis=1))


@pytest.mark.parametrize("n,D,K", [(20_000, 45, 1000), (777, 3, 70), (5000, 16, 64), (3001, 64, 129),
                                   (1, 45, 7), (300, 45, 1), (2500, 33, 300)])
def test_assign_matches_oracle(ctx, path, n, D, K):
    x = sh_rows(n, seed=n + D, D=D)
    rows = synth.vq_init_rows(n, min(K, n), seed=K)
    cb = x[rows] if K <= n else x[np.arange(K) % n]
    cb = np.ascontiguousarray(cb[:K]) + np.float32(1e-3) * np.arange(K, dtype=np.float32)[:, None]
    dev = torch.device("cuda:0")
    xd, cbd = torch.from_numpy(x).to(dev), torch.from_numpy(np.ascontiguousarray(cb, np.float32)).to(dev)
    score = torch.empty(n, dtype=torch.float32, device=dev)
    idx, _ = mgs.mgs_vq_assign(ctx, xd, cbd, score_out=score)
    torch.cuda.synchronize()
    ref_i, ref_s = oracle.vq_assign(x, cb)
    assert np.array_equal(idx.cpu().numpy(), ref_i)
    assert np.array_equal(score.cpu().numpy().view(np.uint32), ref_s.view(np.uint32))


def test_assign_ties_to_lower_index(ctx, path):
    x = sh_rows(500, seed=3)
    cb = np.repeat(x[:8], 3, axis=0)              # every entry three times
    dev = torch.device("cuda:0")
    idx, _ = mgs.mgs_vq_assign(ctx, torch.from_numpy(x).to(dev), torch.from_numpy(cb).to(dev))
    got = idx.cpu().numpy()
    assert np.array_equal(got, oracle.vq_assign(x, cb)[0])
    assert np.all(got % 3 == 0)


@pytest.mark.parametrize("n,K,batch,iters", [(30_000, 256, 4096, 6), (4000, 70, 999, 4), (2000, 5, 1, 3)])
def test_train_matches_oracle(ctx, path, n, K, batch, iters):
    x = sh_rows(n, seed=K)
    cb0 = x[synth.vq_init_rows(n, K, seed=n)]
    bt = synth.vq_batches(n, iters, batch, seed=K + batch)
    dev = torch.device("cuda:0")
    cbd = torch.from_numpy(cb0.copy()).to(dev)
    cnt = torch.zeros(K, dtype=torch.int64, device=dev)
    asg = torch.empty((iters, batch), dtype=torch.int32, device=dev)
    mgs.mgs_vq_train(ctx, torch.from_numpy(x).to(dev), cbd, cnt, torch.from_numpy(bt).to(dev), assign_out=asg)
    torch.cuda.synchronize()
    ref_cb, ref_cnt, ref_a = oracle.vq_train(x, cb0, bt)
    assert np.array_equal(asg.cpu().numpy(), ref_a)
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    assert np.array_equal(cbd.cpu().numpy().view(np.uint32), ref_cb.view(np.uint32))


def test_vq_scene_scale(ctx, path):
    """5.27 M x 45, K = 4096: one mini-batch of 65536 (the bench's batch) equal to
    the oracle's, then the final assignment of every vector, checked on a sample."""
    w = synth.SCENE
    attrs, _ = synth.make_scene(w.n, seed=w.seed)
    x = np.ascontiguousarray(attrs[:, 6:51])
    del attrs
    K = synth.VQ_K
    cb0 = x[synth.vq_init_rows(w.n, K, seed=1)]
    bt = synth.vq_batches(w.n, 1, synth.VQ_BATCH, seed=2)
    dev = torch.device("cuda:0")
    xd = torch.from_numpy(x).to(dev)
    cbd = torch.from_numpy(cb0.copy()).to(dev)
    cnt = torch.zeros(K, dtype=torch.int64, device=dev)
    mgs.mgs_vq_train(ctx, xd, cbd, cnt, torch.from_numpy(bt).to(dev))
    idx, _ = mgs.mgs_vq_assign(ctx, xd, cbd)
    torch.cuda.synchronize()
    ref_cb, ref_cnt, _ = oracle.vq_train(x, cb0, bt)
    assert np.array_equal(cnt.cpu().numpy(), ref_cnt)
    assert np.array_equal(cbd.cpu().numpy().view(np.uint32), ref_cb.view(np.uint32))
    rows = np.sort(np.random.default_rng(4).choice(w.n, 3000, replace=False))
    got = idx.cpu().numpy()[rows]
    assert np.array_equal(got, oracle.vq_assign(x[rows], ref_cb)[0])


def test_retain_and_errors(ctx):
    dev = torch.device("cuda:0")
    idx = torch.arange(100, dtype=torch.int32, device=dev) % 7
    rows = torch.tensor([5, 50, 99, 0], dtype=torch.int32, device=dev)
    mgs.mgs_vq_retain(ctx, rows, 7, idx)
    got = idx.cpu().numpy()
    assert list(got[[5, 50, 99, 0]]) == [7, 8, 9, 10]
    assert got[1] == 1 and got[98] == 98 % 7
    x = torch.from_numpy(sh_rows(100, seed=1)).to(dev)
    cb = x[:4].clone()
    with pytest.raises(mgs.MgsError):                                  # a batch row outside x
        mgs.mgs_vq_train(ctx, x, cb, torch.zeros(4, dtype=torch.int64, device=dev),
                         torch.tensor([[0, 100]], dtype=torch.int32, device=dev))
    with pytest.raises(mgs.MgsError):                                  # host memory
        mgs.mgs_vq_assign(ctx, x.cpu(), cb)
    wide = torch.zeros((10, 65), dtype=torch.float32, device=dev)
    with pytest.raises(mgs.MgsError):                                  # D > 64
        mgs.mgs_vq_assign(ctx, wide, wide[:2].clone())


def test_tensor_path_rescores_few(ctx):
    """The tensor path re-scores every vector's winner and few others: the TF32
    bound is tight enough that the candidates stay a small multiple of n."""
    n, K = 20_000, 1024
    x = sh_rows(n, seed=8)
    cb = np.ascontiguousarray(x[synth.vq_init_rows(n, K, seed=9)])
    dev = torch.device("cuda:0")
    mgs.mgs_vq_set_tensor_cores(ctx, True)
    mgs.mgs_vq_stats(ctx)
    idx, _ = mgs.mgs_vq_assign(ctx, torch.from_numpy(x).to(dev), torch.from_numpy(cb).to(dev))
    scores, rescored = mgs.mgs_vq_stats(ctx)
    assert scores == n * K
    assert n <= rescored <= 8 * n, rescored
    assert np.array_equal(idx.cpu().numpy(), oracle.vq_assign(x, cb)[0])


def test_tensor_path_near_ties(ctx):
    """Entries a few ulp apart and vectors on their midpoints: the approximate
    scores cannot separate them, the exact re-scores do."""
    rng = np.random.default_rng(12)
    base = rng.laplace(0, 0.05, size=(64, 45)).astype(np.float32)
    cb = np.concatenate([base, np.nextafter(base, np.float32(1)), base * np.float32(1 + 2 ** -20)])
    x = np.concatenate([base, (base + np.nextafter(base, np.float32(1))) / 2,
                        rng.laplace(0, 0.05, size=(500, 45)).astype(np.float32)]).astype(np.float32)
    dev = torch.device("cuda:0")
    mgs.mgs_vq_set_tensor_cores(ctx, True)
    idx, _ = mgs.mgs_vq_assign(ctx, torch.from_numpy(np.ascontiguousarray(x)).to(dev),
                               torch.from_numpy(np.ascontiguousarray(cb)).to(dev))
    assert np.array_equal(idx.cpu().numpy(), oracle.vq_assign(x, cb)[0])
