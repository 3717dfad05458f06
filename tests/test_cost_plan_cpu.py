"""The cost kernel's shared-memory histogram plan (host logic, no device): for
every tile configuration and many bit-width lists, the tables of region A are
laid out back to back in mode order with the sizes their modes need, the large
options either share region B in windows that cover their tables or each have
their own table in it, the 16-bit-pair recount windows cover the pair tables,
the plan fits the shared memory of the configuration's CTAs, and the finishing
units cover every bin of every small option exactly once."""
import numpy as np
import pytest

from paper_2604_26799_gb300 import mgs

LANE, DIRECT, PAIR, BYTE = 0, 1, 2, 3


def bit_lists():
    rng = np.random.default_rng(5)
    fixed = [[2, 3, 4, 5, 6, 8, 10, 12, 14, 16], list(range(1, 17)), [4, 6, 8, 10, 12, 16], [2, 4, 8, 12, 16],
             [1, 2, 4, 6, 8, 10, 11, 12, 13, 14, 15, 16], [2, 5, 9, 12, 15, 16], [14, 16], [16], [1], [8, 10]]
    rand = [sorted(rng.choice(np.arange(1, 17), size=int(rng.integers(1, 17)), replace=False).tolist())
            for _ in range(40)]
    return fixed + rand


def up4(w):
    return (w + 3) & ~3


@pytest.mark.parametrize("config", range(mgs.mgs_tile_config_count()))
def test_plan_invariants(config):
    name = mgs.mgs_tile_config_name(config)
    nw = int(name.split("_")[0][1:]) // 32
    for bits in bit_lists():
        p = mgs.mgs_debug_cost_plan(config, bits)
        mode, off, words = p["mode"], p["off"], p["words"]
        n = len(bits)
        assert np.all(np.diff(mode) >= 0), (name, bits)
        for k, b in enumerate(bits):
            assert mode[k] != LANE or b <= 6
            assert mode[k] != DIRECT or b <= 10
            assert mode[k] != PAIR or b <= 12
            assert mode[k] != BYTE or b >= 11
        ns = p["n_small"]
        assert ns == int(np.sum(mode != BYTE))
        assert p["n_lane"] == int(np.sum(mode == LANE)) and p["n_direct"] == int(np.sum(mode == DIRECT))
        # region A: back to back, sized for the mode
        a = 0
        for k in range(ns):
            b = bits[k]
            need = up4({LANE: 32 << b, DIRECT: 1 << b, PAIR: 1 << (b - 1)}[int(mode[k])])
            assert off[k] == a and words[k] == need, (name, bits, k)
            a += need
        assert p["a_words"] == a
        # region B
        bw = p["b_words"]
        if p["concurrent"]:
            o = 0
            for k in range(ns, n):
                need = up4(max(4, 1 << (bits[k] - 2)))
                assert off[k] == o and words[k] == need and p["windows"][k] == 1
                o += need
            assert bw == o
            assert p["smem"] <= p["budget"]
        else:
            for k in range(ns, n):
                need = max(4, 1 << (bits[k] - 2))
                assert words[k] == min(need, bw) and p["windows"][k] * bw >= need
                assert (p["windows"][k] - 1) * bw < need
        for k in range(ns, n):
            assert p["rwindows"][k] * bw >= 1 << (bits[k] - 1)
        assert p["smem"] <= 227 * 1024
        # finishing units: every bin of every small option exactly once
        units = p["units"]
        assert len(units) >= ns and len(units) <= 16
        if ns <= nw:
            assert len(units) <= nw
        for k in range(ns):
            iv = sorted((int(lo), int(hi)) for kk, lo, hi in units if kk == k)
            assert iv and iv[0][0] == 0 and iv[-1][1] == 1 << bits[k], (name, bits, k, iv)
            assert all(iv[j][1] == iv[j + 1][0] for j in range(len(iv) - 1)), (name, bits, k, iv)


def test_plan_rejects_bad_arguments():
    with pytest.raises(mgs.MgsError):
        mgs.mgs_debug_cost_plan(-1, [4, 8])
    with pytest.raises(mgs.MgsError):
        mgs.mgs_debug_cost_plan(mgs.mgs_tile_config_count(), [4, 8])
    with pytest.raises(mgs.MgsError):
        mgs.mgs_debug_cost_plan(0, list(range(1, 18)))
