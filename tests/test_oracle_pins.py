"""The CPU oracle against what the paper and the mathematics fix (no GPU)."""
import numpy as np
import pytest

import oracle
from oracle import mckp
from tests import pins


@pytest.mark.parametrize("b", list(range(1, 17)))
def test_grid_closed_form_same_b(oracle_lib, b):
    pins.check_grid(oracle_lib, b, b)


@pytest.mark.parametrize("b_data,b_q", [(10, 1), (10, 3), (10, 7), (8, 12), (6, 16), (12, 5)])
def test_grid_closed_form_other_b(oracle_lib, b_data, b_q):
    pins.check_grid(oracle_lib, b_data, b_q)


@pytest.mark.parametrize("j,off", [(4, 11), (4, 5), (6, 37), (8, 200), (3, 0), (10, 999)])
def test_dyadic_offset_grid_exact(oracle_lib, j, off):
    for b in range(1, 17):
        pins.check_dyadic(oracle_lib, j, off, b)


@pytest.mark.parametrize("value,n", [(0.0, 1), (3.25, 7), (-1e-3, 4096), (1e30, 33)])
def test_constant_group(oracle_lib, value, n):
    pins.check_constant(oracle_lib, value, n, list(range(1, 17)))


@pytest.mark.parametrize("seed", range(6))
def test_invariants_random(oracle_lib, seed):
    rng = np.random.default_rng(100 + seed)
    dists = [
        lambda n: rng.standard_normal(n) * 2.0,
        lambda n: rng.laplace(0.0, 0.05, n),
        lambda n: rng.uniform(-4.0, -3.9, n),
        lambda n: np.round(rng.standard_normal(n) * 4) / 4,   # many ties
        lambda n: rng.standard_normal(n) * 1e-20,               # tiny scale, normal floats
        lambda n: rng.standard_normal(n) + 1000.0,              # large offset, small range
    ]
    for n in (1, 2, 3, 17, 1000):
        vals = dists[seed](n).astype(np.float32)
        pins.check_invariants(oracle_lib, vals, list(range(1, 17)))


def test_uniform_noise_textbook(oracle_lib):
    pins.check_uniform_noise(oracle_lib)


@pytest.mark.parametrize("m,M", [(-0.375, 0.625), (1.0, 1.0000002), (-7.1, 3.3), (0.0, 1e-3)])
def test_two_point(oracle_lib, m, M):
    pins.check_two_point(oracle_lib, m, M, list(range(1, 17)))


def test_morton_lattice(oracle_lib):
    pins.check_morton_lattice(oracle_lib)


def test_rank_matches_lexsort(oracle_lib):
    pins.check_rank(oracle_lib)


def test_subnormal_scale_degenerate(oracle_lib):
    # range 2^-140: 2^-140 / 2^16 underflows to 0 -> degenerate rule; at b=1 S is subnormal, not 0
    vals = np.array([0.0, 2.0 ** -140, 0.0], dtype=np.float32)
    out = oracle.group_cost(vals, [1, 16], want_codes=True)
    assert np.all(out["codes"][1] == 0) and out["sse"][1] == 0.0 and out["hbits"][1] == 0.0
    assert out["codes"][0][1] == 1 and out["codes"][0][0] == 0


def test_nonfinite_rejected(oracle_lib):
    with pytest.raises(oracle.OracleError) as e:
        oracle.group_cost(np.array([1.0, np.nan], dtype=np.float32), [4])
    assert e.value.code == oracle.ERR_NONFINITE
    with pytest.raises(oracle.OracleError) as e:
        oracle.group_cost(np.array([-3e38, 3e38], dtype=np.float32), [4])
    assert e.value.code == oracle.ERR_RANGE


def _tiny_scene(n=300, seed=7, C=5):
    rng = np.random.default_rng(seed)
    attrs = rng.standard_normal((n, C)).astype(np.float32)
    attrs[:, :3] = rng.uniform(0, 1, (n, 3)).astype(np.float32)
    imp = np.exp(rng.standard_normal(n)).astype(np.float32)
    return attrs, imp


def test_kept_sets_nested_and_sized(oracle_lib):
    attrs, imp = _tiny_scene()
    rk = oracle.rank(imp)
    _, order = oracle.morton(attrs)
    prev = set()
    for K in (0, 1, 30, 150, 299, 300):
        kp = oracle.kept(rk, order, K)
        assert kp.shape[0] == K
        assert np.all(np.diff(kp) > 0)  # Morton order
        s = set(kp.tolist())
        assert prev <= s
        prev = s
        # exactly the K most important Gaussians (library sort)
        top = set(np.argsort(-imp.astype(np.float64), kind="stable")[:K].tolist())
        assert {int(order[p]) for p in kp} == top


def test_cost_table_items_match_group_cost(oracle_lib):
    attrs, imp = _tiny_scene()
    keep = np.array([30, 150, 300], dtype=np.int64)
    bits = [1, 3, 8, 16]
    G = 64
    t = oracle.cost_table(attrs, imp, keep, bits, G)
    rk = oracle.rank(imp)
    _, order = oracle.morton(attrs)
    item = 0
    C = attrs.shape[1]
    for K in keep:
        kp = oracle.kept(rk, order, K)
        ng = oracle.n_groups(K, G)
        for c in range(C):
            total = 0
            for g in range(ng):
                vals = attrs[order[kp[g * G:(g + 1) * G]], c]
                ref = oracle.group_cost(vals, bits)
                assert t["cnt"][item] == vals.shape[0]
                assert (t["cnt"][item] == G) or g == ng - 1
                total += t["cnt"][item]
                for key in ("sse", "l1", "linf", "hbits"):
                    assert np.array_equal(t[key][item], ref[key])
                assert t["vmin"][item] == ref["vmin"] and t["vmax"][item] == ref["vmax"]
                item += 1
            assert total == K
    assert item == t["cnt"].shape[0]


def test_threaded_table_equals_serial(oracle_lib):
    """The CPU baseline's threaded driver gives the serial table entry for entry."""
    attrs, imp = _tiny_scene()
    keep = np.array([30, 150, 300], dtype=np.int64)
    bits = [1, 3, 8, 16]
    a = oracle.cost_table(attrs, imp, keep, bits, 16)
    for threads in (2, 7):
        b = oracle.cost_table(attrs, imp, keep, bits, 16, threads=threads)
        for key in a:
            assert np.array_equal(a[key], b[key]), (threads, key)


def test_mckp_dp_equals_bruteforce():
    rng = np.random.default_rng(11)
    for trial in range(25):
        n_items, n_b = rng.integers(1, 6), rng.integers(1, 4)
        bits = np.sort(rng.choice(np.arange(1, 9), size=n_b, replace=False))
        cnt = rng.integers(1, 40, size=n_items)
        dist = rng.uniform(0, 10, size=(n_items, n_b))
        w = cnt[:, None] * bits[None, :]
        rates = w.astype(np.float64)
        lo = rates.min(axis=1).sum() / 8 + 9 * n_items
        hi = rates.max(axis=1).sum() / 8 + 9 * n_items
        budget = float(rng.uniform(lo - 5, hi + 5))
        bf = mckp.solve_bruteforce(dist, rates, budget)
        dp = mckp.solve_dp_integer(dist, w, budget)
        if bf is None:
            assert dp is None
            continue
        assert dp is not None
        assert abs(bf[0] - dp[0]) <= 1e-9 * max(1.0, bf[0])
        assert mckp.assignment_bytes(rates, dp[1], 0.0) <= budget


def test_choose_tau_rule():
    mk = lambda f, o, top: dict(feasible=f, objective=o, bytes_min=0.0, bytes_top=top)
    # r0 skipped (top size below budget), r1 and r2 candidates; r1 lower distortion wins
    assert mckp.choose_tau([mk(True, 1.0, 50), mk(True, 2.0, 200), mk(True, 3.0, 300)], 100) == 1
    # ties go to the larger ratio
    assert mckp.choose_tau([mk(True, 2.0, 200), mk(True, 2.0, 300)], 100) == 1
    # everything skipped -> largest feasible ratio
    assert mckp.choose_tau([mk(True, 1.0, 10), mk(True, 2.0, 20), mk(False, 0, 0)], 100) == 1
    assert mckp.choose_tau([mk(False, 0, 0)], 100) is None


def test_euler_axes():
    pins.check_euler_axes(oracle.lib())


def test_euler_roundtrip_against_quaternion_matrix():
    pins.check_euler_roundtrip(oracle.lib())


def test_preprocess_quantile_and_importance():
    pins.check_preprocess(oracle.lib())


def test_raht_worked_example():
    pins.check_raht_example(oracle.lib())


def test_raht_ranges():
    pins.check_raht_ranges(oracle.lib())


def test_raht_orthonormal():
    pins.check_raht_orthonormal(oracle.lib())


def test_raht_constant_and_dedup():
    pins.check_raht_constant_and_dedup(oracle.lib())


def test_raht_kept_set():
    pins.check_raht_keep(oracle.lib())


def test_coder_roundtrip_independent_reader():
    pins.check_coder_roundtrip(oracle.lib())


def test_coder_size_against_entropy_bound():
    pins.check_coder_entropy(oracle.lib())


def test_coder_frequency_normalisation():
    pins.check_coder_normalisation(oracle.lib())


def test_encode_config_concatenates_blocks():
    """A whole configuration: blocks in (channel, group) order, each readable
    on its own and equal to the block of that group's quantised codes."""
    from paper_2604_26799_gb300 import synth
    attrs, imp = synth.make_scene(3000, seed=21)
    attrs = attrs[:, :6].copy()
    keep, G = 2100, 512
    ng = oracle.n_groups(keep, G)
    rng = np.random.default_rng(5)
    q_bits = rng.integers(1, 17, size=(6, ng)).astype(np.uint8)
    stream, sizes = oracle.encode_config(attrs, imp, keep, G, q_bits)
    codes, minmax = oracle.quantize(attrs, imp, keep, G, q_bits)
    at = 0
    for c in range(6):
        for g in range(ng):
            n = min(G, keep - g * G)
            blk = stream[at:at + int(sizes[c, g])]
            got, b, mn, mx, used, _ = pins.read_block_py(blk, n)
            assert used == len(blk) and b == q_bits[c, g]
            assert np.array_equal(np.asarray(got, np.uint16), codes[c, g * G:g * G + n])
            assert np.float32(mn) == minmax[c, g, 0] and np.float32(mx) == minmax[c, g, 1]
            at += len(blk)
    assert at == len(stream) == int(sizes.sum())


def test_vq_assignment():
    pins.check_vq_assign(oracle.lib())


def test_vq_minibatch_update():
    pins.check_vq_update(oracle.lib())
