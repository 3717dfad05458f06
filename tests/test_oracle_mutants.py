"""Plant plausible mistakes in a copy of the oracle and check that the pins
catch each one (the mistake is planted on the CPU, in a temporary copy)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "scale_2b_minus_1": ("float S = R / twob;", "float S = R / (twob - 1.0f);"),
    "zero_point_floor": ("float Z = rintf(zr);", "float Z = floorf(zr);"),
    "zero_point_sign": ("float x = y + Z;", "float x = y - Z;"),
    "dequant_drops_Z": ("float qz = (float)q - Z;", "float qz = (float)q;"),
    "error_sign": ("float e = chat - c;", "float e = chat + c;"),
    "code_truncates": ("int q = (int)rintf(xc);", "int q = (int)xc;"),
    "range_transposed": ("float R = M - m;", "float R = m - M;"),
    "sse_not_squared": ("s2 += (double)e * (double)e;", "s2 += fabs((double)e);"),
    "entropy_drops_n": ("double p = (double)hist[s] / (double)n;", "double p = (double)hist[s];"),
    "morton_y_bit": ("code |= (uint64_t)((y >> k) & 1u) << (3 * k + 1);",
                     "code |= (uint64_t)((y >> k) & 1u) << (3 * k + 2);"),
    "morton_scale": ("double s = floor((double)t * 2097152.0);",
                     "double s = floor((double)t * 2097151.0);"),
    "rank_ascending": ("if (x->key > y->key) return -1; /* larger importance first */",
                       "if (x->key > y->key) return 1;"),
    "rank_tiebreak": ("if (x->idx < y->idx) return -1; /* ties: smaller index first */",
                      "if (x->idx < y->idx) return 1;"),
    "euler_roll_sign": ("e[0] = atan2(2.0 * (w * x + y * z),", "e[0] = atan2(2.0 * (w * x - y * z),"),
    "euler_pitch_offset": ("e[1] = -ORACLE_PI / 2.0 + 2.0 * atan2(sqrt(a), sqrt(b));",
                           "e[1] = 2.0 * atan2(sqrt(a), sqrt(b));"),
    "euler_yaw_args": ("e[2] = atan2(2.0 * (w * z + x * y), 1.0 - 2.0 * (y * y + z * z));",
                       "e[2] = atan2(1.0 - 2.0 * (y * y + z * z), 2.0 * (w * z + x * y));"),
    "euler_not_normalised": ("double w = q_in[0] / nrm, x = q_in[1] / nrm, y = q_in[2] / nrm, z = q_in[3] / nrm;",
                             "double w = q_in[0], x = q_in[1], y = q_in[2], z = q_in[3];"),
    "quantile_index": ("double vq = sorted[(9 * (n - 1)) / 10];", "double vq = sorted[(9 * n) / 10];"),
    "volume_not_clipped": ("double vn = vq > 0.0 ? fmin(vol[i] / vq, 1.0) : 1.0;",
                           "double vn = vq > 0.0 ? vol[i] / vq : 1.0;"),
    "raht_ac_sign": ("double ac = t1 * x2 - t2 * x1;", "double ac = t1 * x1 - t2 * x2;"),
    "raht_weights_not_rooted": ("double t1 = sqrt(w1) / sw, t2 = sqrt(w2) / sw;",
                                "double t1 = w1 / sw, t2 = w2 / sw;"),
    "raht_mean_not_divided": ("x[m * n_c + k] = q - p > 1 ? sum / (double)(q - p) : sum;",
                              "x[m * n_c + k] = sum;"),
    "raht_weight_not_summed": ("w[out] = w[i] + w[i + 1];", "w[out] = w[i];"),
    "rans_cum_dropped": ("x[lane] = (uint32_t)((x[lane] / f[s]) * M + x[lane] % f[s] + cum[s]);",
                         "x[lane] = (uint32_t)((x[lane] / f[s]) * M + x[lane] % f[s]);"),
    "rans_lane_reversed": ("int lane = (int)(i % lanes);", "int lane = (int)((n - 1 - i) % lanes);"),
    "rans_renorm_threshold": ("uint64_t xmax = ((uint64_t)(ORACLE_RANS_L >> k) << 8) * f[s];",
                              "uint64_t xmax = ((uint64_t)(ORACLE_RANS_L >> k) << 7) * f[s];"),
    "gamma_lsb_first": ("for (int j = N; j >= 0; j--) put_bit(w, (unsigned)((x >> j) & 1u));",
                        "for (int j = 0; j <= N; j++) put_bit(w, (unsigned)((x >> j) & 1u));"),
    "raw_bit_order": ("for (int j = 0; j < b; j++) put_bit(&rw, (codes[i] >> j) & 1u);",
                      "for (int j = 0; j < b; j++) put_bit(&rw, (codes[i] >> (b - 1 - j)) & 1u);"),
    "shortfall_to_last_tie": ("if (hist[s] > hist[top]) top = s;", "if (hist[s] >= hist[top]) top = s;"),
    "mode_choice_inverted": ("if (rans_payload < raw_payload) {", "if (rans_payload > raw_payload) {"),
    "frequency_not_scaled": ("f[s] = (uint32_t)(((uint64_t)hist[s] * M) / (uint64_t)n);",
                             "f[s] = hist[s];"),
    "vq_score_sign": ("float score = fmaf(-2.0f, dot, cc[k]);", "float score = fmaf(2.0f, dot, cc[k]);"),
    "vq_norm_dropped": ("float score = fmaf(-2.0f, dot, cc[k]);", "float score = -2.0f * dot;"),
    "vq_tie_to_higher": ("if (k == 0 || score < best_s) {", "if (k == 0 || score <= best_s) {"),
    "vq_count_ignored": ("double v = (double)counts[k];", "double v = 0.0;"),
    "vq_mean_over_batch_only": ("cb[(int64_t)k * D + d] = (float)(num / (v + (double)m[k]));",
                                "cb[(int64_t)k * D + d] = (float)(num / (double)m[k]);"),
    "vq_batch_row_shift": ("memcpy(xb + (int64_t)j * D, x + (int64_t)rows[j] * D, sizeof(float) * D);",
                           "memcpy(xb + (int64_t)j * D, x + (int64_t)rows[j] * D + 1, sizeof(float) * (D - 1));"),
    "raht_keep_ignored": ("        K = oracle_kept(rank, order, n, keep, pos);",
                          "        for (int64_t t = 0; t < n; t++) pos[t] = t;"),
    "raht_range_min": ("double r = r1 > r2 ? r1 : r2;", "double r = r1 < r2 ? r1 : r2;"),
    "raht_range_not_carried": ("                    xr[out * n_c + k] = r;", "                    xr[out * n_c + k] = r1;"),
}

RUNNER = r"""
import sys, numpy as np
sys.path.insert(0, {root!r})
import oracle
from tests import pins
L = oracle.load({so!r})
checks = [
    lambda: [pins.check_grid(L, b, b) for b in (1, 4, 9, 16)],
    lambda: [pins.check_grid(L, 10, b) for b in (3, 12)],
    lambda: [pins.check_dyadic(L, 4, 11, b) for b in range(1, 17)],
    lambda: [pins.check_dyadic(L, 6, 37, b) for b in range(1, 17)],
    lambda: pins.check_constant(L, 3.25, 9, list(range(1, 17))),
    lambda: [pins.check_invariants(L, v, list(range(1, 17))) for v in (
        np.random.default_rng(0).standard_normal(500).astype(np.float32) * 2 + 1,
        np.random.default_rng(1).uniform(-4, -3.9, 300).astype(np.float32))],
    lambda: pins.check_uniform_noise(L),
    lambda: pins.check_two_point(L, -7.1, 3.3, list(range(1, 17))),
    lambda: pins.check_morton_lattice(L),
    lambda: pins.check_rank(L),
    lambda: pins.check_euler_axes(L),
    lambda: pins.check_euler_roundtrip(L),
    lambda: pins.check_preprocess(L),
    lambda: pins.check_raht_example(L),
    lambda: pins.check_raht_orthonormal(L),
    lambda: pins.check_raht_constant_and_dedup(L),
    lambda: pins.check_raht_keep(L),
    lambda: pins.check_raht_ranges(L),
    lambda: pins.check_coder_roundtrip(L),
    lambda: pins.check_coder_entropy(L),
    lambda: pins.check_coder_normalisation(L),
    lambda: pins.check_vq_assign(L),
    lambda: pins.check_vq_update(L),
]
failed = 0
for c in checks:
    try:
        c()
    except Exception:
        failed += 1
print("FAILED_CHECKS", failed)
sys.exit(0 if failed else 7)
"""


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found: {old}"
    mut = tmp_path / "oracle_mut.c"
    mut.write_text(src.replace(old, new))
    so = tmp_path / "liboracle_mut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                    "-fno-fast-math", "-o", str(so), str(mut), "-lm"], check=True)
    code = RUNNER.format(root=ROOT, so=str(so))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    # exit 0 = at least one pin failed on the mutant (what we want); 7 = mutant survived
    assert r.returncode != 7, f"mutant {name} survived every pin:\n{r.stdout}\n{r.stderr}"
    assert r.returncode == 0 or r.returncode < 0, r.stderr
