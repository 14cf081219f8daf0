"""The oracles' pins catch plausible mistakes.  Each case plants one mistake in a copy of
oracle/oracle.c (compiled on the CPU) or oracle/prop_oracle.py (a dropped term, a wrong sign,
index or tie rule, a transposed operand, a missing rounding point) and runs that oracle's pins
against it in a child process: some pin must fail.  The unchanged oracles pass through the
same harness."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    # maximum scoring subsequence: the restart at 0 dropped
    "kadane_no_restart": ("    if (ending_here < 0) ending_here = 0;\n", ""),
    # substitution score: N against N scored as a match
    "n_matches_n": ("x[n++] = (a < 4 && a == b) ? sm : sx;", "x[n++] = (a == b) ? sm : sx;"),
    # reverse complement: complemented but not reversed
    "revcomp_not_reversed": ("uint8_t c = q[m - 1 - k];", "uint8_t c = q[k];"),
    # reverse complement: reversed but not complemented
    "revcomp_not_complemented": ("out[k] = (uint8_t)(c < 4 ? 3 - c : 4);", "out[k] = c;"),
    # base codes: G and T confused
    "g_coded_as_t": ("case 'G': case 'g': return 2;", "case 'G': case 'g': return 3;"),
    # fragment of a diagonal off by one
    "fragment_index_off_by_one": ("int64_t f = d / F;", "int64_t f = (d + 1) / F;"),
    # genome padded with A instead of N
    "padding_with_a": ("for (int64_t i = G; i < glen; ++i) g[i] = 4;", "for (int64_t i = G; i < glen; ++i) g[i] = 0;"),
    # best diagonal of a fragment: ties to the later (strand, d)
    "diagonal_ties_to_last": ("if (K > S[f]) {", "if (K >= S[f]) {"),
    # best fragment: ties to the highest index
    "best_ties_to_last": ("if (S[f] > S[b1]) b1 = f;", "if (S[f] >= S[b1]) b1 = f;"),
    # second fragment: ties to the highest index
    "second_ties_to_last": ("if (b2 < 0 || S[f] > S[b2]) b2 = f;", "if (b2 < 0 || S[f] >= S[b2]) b2 = f;"),
    # ratio test: strict instead of "at least 0.9"
    "ratio_strict": ("(int64_t)10 * out->second_score >= (int64_t)9 * out->best_score",
                     "(int64_t)10 * out->second_score > (int64_t)9 * out->best_score"),
    # affine gaps: open and extend transposed in the read-gap recurrence
    "gap_open_extend_swapped": ("e = max2(AT(H, i, j - 1) + gap_open, AT(E, i, j - 1) + gap_extend);",
                                "e = max2(AT(H, i, j - 1) + gap_extend, AT(E, i, j - 1) + gap_open);"),
    # band one diagonal narrower on one side
    "band_asymmetric": ("return t >= -W && t <= W;", "return t >= -W && t < W;"),
    # base qualities: the mismatch score not divided among the three other bases
    "pssm_mismatch_not_divided": ("*mm = round_half_away((double)scale * mismatch * x / 3.0);",
                                  "*mm = round_half_away((double)scale * mismatch * x);"),
    # base qualities: the error probability 10^(-Q/10) read as 10^(-Q)
    "pssm_phred_scale": ("double x = 1.0 - pow(10.0, -Q / 10.0);", "double x = 1.0 - pow(10.0, -Q / 1.0);"),
    # MaxSSmap_fast: the odd read positions sampled instead of the even ones
    "fast_step_odd_positions": ("for (int32_t k = 0; k < m; k += step) {", "for (int32_t k = step - 1; k < m; k += step) {"),
    # lowercase bases rejected
    "lowercase_a_invalid": ("case 'A': case 'a': return 0;", "case 'A': return 0;"),
    # strand tie rule reversed (reverse complement before the read)
    "strand_ties_reversed": ("for (int32_t sg = 0; sg < 2; ++sg) {", "for (int32_t sg = 1; sg >= 0; --sg) {"),
    # base qualities: phase two's gap costs left unscaled (scores in 1/scale units, gaps not)
    "pssm_gap_unscaled": ("W, gap_open * scale, gap_extend * scale,", "W, gap_open, gap_extend,"),
    # neighbour rule: only the right neighbour excluded
    "neighbour_rule_one_side": ("if (exclude_neighbors && (f == b1 - 1 || f == b1 + 1)) continue;",
                                "if (exclude_neighbors && (f == b1 + 1)) continue;"),
}


def _run_pins(src: str, tmp_path):
    """Compile src as the oracle and run the pins against it; returns the child's exit code
    (0: every pin passed, 1: a pin failed, negative: the planted mistake crashed the oracle)."""
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no gcc")
    mdir = tmp_path / "oracle"
    mdir.mkdir()
    (mdir / "oracle.c").write_text(src)
    shutil.copy(os.path.join(ROOT, "oracle", "oracle.h"), mdir / "oracle.h")
    so = mdir / "liboracle_variant.so"
    subprocess.check_call([cc, "-O2", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(mdir / "oracle.c"), "-lm"])
    env = dict(os.environ, MSS_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-x", "-q",
                        "-p", "no:cacheprovider", "-m", "not gpu"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def test_unchanged_oracle_passes_through_the_same_harness(tmp_path):
    rc, out = _run_pins(open(SRC).read(), tmp_path)
    assert rc == 0, out


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"{name}: the planted line must occur exactly once"
    rc, out = _run_pins(src.replace(old, new), tmp_path)
    assert rc == 1 or rc < 0, f"{name}: no pin failed\n{out}"


PROP_SRC = os.path.join(ROOT, "oracle", "prop_oracle.py")

PROP_MUTANTS = {
    # tap direction: convolution instead of correlation
    "tap_direction": ("    s = t - 3\n    lo, hi", "    s = 3 - t\n    lo, hi"),
    # ReLU dropped in layers 2-4
    "relu_dropped": ("        a = rnd(np.maximum(z, 0.0))\n", "        a = rnd(z)\n"),
    # bias dropped in layers 2-4
    "bias_dropped": ("        z = bs[l][None, :] + sum(", "        z = 0.0 + sum("),
    # squared norm instead of the norm
    "squared_norm": ("nrm = np.sqrt(np.sum(v * v)) + 1e-6", "nrm = np.sum(v * v) + 1e-6"),
    # epsilon of the normalisation dropped
    "norm_epsilon_dropped": ("nrm = np.sqrt(np.sum(v * v)) + 1e-6", "nrm = np.sqrt(np.sum(v * v)) + 1e-30"),
    # the last maximum kept instead of the first
    "argmax_last": ("arg = np.argmax(a, axis=0)          # first maximum",
                    "arg = a.shape[0] - 1 - np.argmax(a[::-1], axis=0)"),
    # BF16 weights of layers 2-4 not applied in the forward pass
    "weights_not_rounded": ("W = rnd(ws[l]) if rounding else ws[l]", "W = ws[l]"),
    # layer-1 output not rounded to BF16
    "layer1_not_rounded": ("    a = rnd(np.maximum(z, 0.0))\n    acts.append(a)\n    pres = [z]",
                           "    a = np.maximum(z, 0.0)\n    acts.append(a)\n    pres = [z]"),
    # T treated as N
    "t_as_n": ("ok = x < 4", "ok = x < 3"),
    # backward: the layer-1 ReLU mask dropped
    "backward_l1_mask_dropped": ("gz1 = g * (acts[1] > 0)", "gz1 = g"),
    # backward: the data gradient shifted the wrong way
    "backward_shift_direction": ("            s = t - 3\n            contrib", "            s = 3 - t\n            contrib"),
    # loss gradient not averaged over the batch
    "ce_not_averaged": ("    d /= B\n", ""),
    # mean pooling: the sum instead of the mean
    "mean_pool_not_divided": ("        v = a.sum(axis=0) / L\n", "        v = a.sum(axis=0)\n"),
    # mean pooling backward: the 1/L factor dropped
    "mean_pool_backward_not_divided": ("g[:, :] = dv[None, :] / L", "g[:, :] = dv[None, :]"),
    # mean pooling over the padded length (one more row than the sequence)
    "mean_pool_wrong_length": ("        v = a.sum(axis=0) / L\n", "        v = a.sum(axis=0) / (L + 1)\n"),
    # BF16 rounding: ties away from zero
    "bf16_ties_away": ("u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16", "u = (u + 0x8000) >> 16 << 16"),
}


def _run_prop_pins(src: str, tmp_path):
    path = tmp_path / "prop_oracle_variant.py"
    path.write_text(src)
    env = dict(os.environ, MSS_PROP_ORACLE=str(path))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_prop_oracle_pins.py"), "-x",
                        "-q", "-p", "no:cacheprovider", "-m", "not gpu"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def test_unchanged_prop_oracle_passes_through_the_same_harness(tmp_path):
    rc, out = _run_prop_pins(open(PROP_SRC).read(), tmp_path)
    assert rc == 0, out


@pytest.mark.parametrize("name", sorted(PROP_MUTANTS))
def test_prop_pins_catch_planted_mistake(name, tmp_path):
    old, new = PROP_MUTANTS[name]
    src = open(PROP_SRC).read()
    assert src.count(old) == 1, f"{name}: the planted line must occur exactly once"
    rc, out = _run_prop_pins(src.replace(old, new), tmp_path)
    assert rc == 1 or rc < 0, f"{name}: no pin failed\n{out}"
