"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a private copy of the oracle's C source (never
in the committed file), builds it on the CPU, and checks that at least one pin
of ``test_oracle_pins`` fails against the mutated build.
"""
import os
import subprocess

import pytest

import oracle as orc
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(orc.__file__), "mbp_oracle.c")


def _tree_pin():
    for u in (1, 2, 3):
        for trial in range(4):
            pins.test_tree_codes_reach_exact_map(u, trial)


def _parity_pin():
    for d in (2, 3, 4):
        for z in (0, 1):
            pins.test_check_node_is_parity_posterior(d, z)


def _frames_pin():
    pins.test_small_code_converged_frames_are_the_unique_solution()


def _syndrome_pin():
    pins.test_syndrome_against_dense_gf2_and_linearity()


def _llr_pin():
    for e in (0.02, 0.1):
        pins.test_bsc_llr_is_channel_likelihood_ratio(e)


def _minsum_pin():
    import test_oracle_variants as var
    for u in (1, 2):
        for trial in range(3):
            var.test_minsum_tree_codes_reach_max_log_posteriors(u, trial)
    for d in (3, 4):
        var.test_minsum_bracketed_by_sum_product(d)


def _clip_pin():
    for u in (1, 2, 3):
        for trial in range(3):
            pins.test_clip_star_centre_is_map_of_clipped_leaves(u, trial)
            pins.test_clip_chain_closed_form(u, trial)
    for u in (1, 2):
        for trial in range(3):
            pins.test_clip_star_leaves_take_the_clipped_centre_extrinsic(u, trial)
            pins.test_clip_far_away_star_posteriors_exact(u, trial)


MUTATIONS = {
    # variable-to-check message forgets the channel prior
    "v2c_drops_prior": ("            double s = LP[i];\n            for (int64_t b",
                        "            double s = 0.0;\n            for (int64_t b", _tree_pin),
    # variable-to-check message keeps its own check's message (not extrinsic)
    "v2c_not_extrinsic": ("if (C->col_edge[b] != a) s += c2v[C->col_edge[b]];", "s += c2v[C->col_edge[b]];", _tree_pin),
    # syndrome sign of eq. (6) ignored
    "c2v_ignores_syndrome": ("double s = z ? -1.0 : 1.0;\n  for (int k = 0; k < d; ++k) {\n    double ext;",
                             "double s = 1.0;\n  for (int k = 0; k < d; ++k) {\n    double ext;", _tree_pin),
    # wrong sign of the correction term of the boxplus
    "boxplus_sign": ("- log1p(exp(-fabs(a - b)))", "+ log1p(exp(-fabs(a - b)))", _parity_pin),
    # prefix combination shifted by one edge
    "prefix_off_by_one": ("orc_boxplus(pre[k - 1], v2c[k - 1])", "orc_boxplus(pre[k - 1], v2c[k])", _parity_pin),
    # posterior of eq. (2) forgets the channel prior
    "posterior_drops_prior": ("          double s = LP[i];\n          for (int64_t a",
                              "          double s = 0.0;\n          for (int64_t a", _tree_pin),
    # hard decision with the wrong orientation
    "hard_decision_flipped": ("set_bit(xhat, i, LV[i] < 0.0);", "set_bit(xhat, i, LV[i] > 0.0);", _frames_pin),
    # syndrome of eq. (1) reads the wrong bit of x
    "syndrome_wrong_bit": ("p ^= bit_of(x, C->edge_col[k]);", "p ^= bit_of(x, C->edge_col[k] + 1);", _syndrome_pin),
    # min-sum rule takes its own edge into the minimum (not extrinsic)
    "minsum_not_extrinsic": ("      if (r == k) continue;\n      s *= sgn(v2c[r]);", "      s *= sgn(v2c[r]);",
                             _minsum_pin),
    # min-sum rule ignores the syndrome bit
    "minsum_ignores_syndrome": ("    double s = z ? -1.0 : 1.0, mn = INFINITY;", "    double s = 1.0, mn = INFINITY;",
                                _minsum_pin),
    # variable-to-check messages not clipped before eq. (6)
    "v2c_no_clip": ("v2c[a] = clip(s, L);", "v2c[a] = s;", _clip_pin),
    # variable-to-check clip at half the bound
    "v2c_clip_half": ("v2c[a] = clip(s, L);", "v2c[a] = clip(s, 0.5 * L);", _clip_pin),
    # variable-to-check clip at a fixed 20 instead of the L_max given
    "v2c_clip_fixed": ("v2c[a] = clip(s, L);", "v2c[a] = clip(s, 20.0);", _clip_pin),
    # check-to-variable messages of the decoder not clipped after eq. (6) (a degree-1 check then sends inf)
    "decode_c2v_no_clip": ("else if (orc_check_node(d, vin, zj, L, vout)) return -2;",
                           "else if (orc_check_node(d, vin, zj, INFINITY, vout)) return -2;", _clip_pin),
    # eq. (5) with P^0 and P^1 swapped
    "llr_orientation": ("L_P[i] = log(p0 / p1);", "L_P[i] = log(p1 / p0);", _llr_pin),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, tmp_path):
    old, new, pin = MUTATIONS[name]
    src = open(SRC).read()
    assert old in src, f"mutation anchor for {name} not found"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    so = tmp_path / "mutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-shared", "-fPIC",
                           "-o", str(so), str(mutated), "-lm", "-lpthread"])
    with orc.library_override(str(so)):
        with pytest.raises((AssertionError, RuntimeError, ValueError, ZeroDivisionError, FloatingPointError)):
            pin()
