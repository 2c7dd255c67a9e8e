"""Plant plausible mistakes in a copy of the oracle source and check that the
pins catch every one of them (a dropped term, a wrong sign, a wrong index, a
transposed operand, a wrong derivative, a wrong threshold).

The mistakes are planted in a temporary copy compiled on the CPU; the oracle
itself is never modified.
"""
import os
import shutil
import tempfile

import pytest

import oracle
from tests import test_oracle_pins as P

MUTANTS = {
    "sigmoid_sign": ("return 1.0 / (1.0 + exp(-x));", "return 1.0 / (1.0 + exp(x));"),
    "drop_b1": ("double z1 = b1[j];", "double z1 = 0.0;"),
    "drop_b2": ("double z2 = b2;", "double z2 = 0.0;"),
    "W1_transposed": ("z1 += x[k] * W1[(long)j * D + k];", "z1 += x[k] * W1[(long)k * H + j];"),
    "output_deriv_dropped": ("double d2 = dLdo[i] * o * (1.0 - o);", "double d2 = dLdo[i];"),
    "hidden_deriv_wrong": ("    return v * (1.0 - v);", "    return v;"),
    "tanh_deriv_wrong": ("return 1.0 - v * v;", "return 1.0 - v;"),
    "error_sign": ("double e = o[i] - y[i];", "double e = y[i] - o[i];"),
    "update_sign": ("W1[p] -= lr * gW1[p];", "W1[p] += lr * gW1[p];"),
    "bias_update_dropped": ("b1[j] -= lr * gb1[j];", "b1[j] -= 0.0 * gb1[j];"),
    "mean_scale_dropped": ("double c = loss_mean ? (n > 0 ? 1.0 / (double)n : 0.0) : 1.0;",
                           "double c = loss_mean ? 1.0 : 1.0;"),
    "gb1_uses_d2": ("gb1[j] += d1;", "gb1[j] += d2;"),
    "gW1_uses_h": ("gW1[(long)j * D + k] += d1 * x[k];", "gW1[(long)j * D + k] += d1 * h[j];"),
    "gW1_transposed": ("gW1[(long)j * D + k] += d1 * x[k];", "gW1[(long)k * H + j] += d1 * x[k];"),
    "gw2_uses_o": ("gw2[j] += d2 * h[j];", "gw2[j] += d2 * o;"),
    "hidden_delta_no_w2": ("double d1 = d2 * w2[j] * orc_hidden_act_deriv(act, h[j]);",
                           "double d1 = d2 * orc_hidden_act_deriv(act, h[j]);"),
    "gX_wrong_operand": ("gX[i * D + k] += d1 * W1[(long)j * D + k];", "gX[i * D + k] += d1 * x[k];"),
    "predict_strict": ("label[i] = o[i] >= 0.5 ? 1 : 0;", "label[i] = o[i] > 0.5 ? 1 : 0;"),
    "loss_hist_half_dropped": ("loss_hist[e] = 0.5 * sse", "loss_hist[e] = sse"),
    "minibatch_loss_last_batch_only": ("sse += orc_mse_gradients(", "sse = orc_mse_gradients("),
    "gnorm_missing_b2": ("    s += gb2 * gb2;\n", "\n"),
    "zscore_sample_deviation": ("sqrt(q / (double)n_fit)", "sqrt(q / (double)(n_fit - 1))"),
    "zscore_stats_over_all_rows": ("for (long i = 0; i < n_fit; ++i) s += X[i * D + j];",
                                   "for (long i = 0; i < n; ++i) s += X[i * D + j];"),
    "zscore_not_centred": ("(X[i * D + j] - m) / sd", "X[i * D + j] / sd"),
}

PINS = [
    P.test_sigmoid_closed_values,
    P.test_sigmoid_matches_scipy_expit,
    lambda: P.test_zero_weights_221_closed_form(True),
    P.test_ln3_forward_exact,
    P.test_ln3_gradients_closed_form,
    lambda: P.test_gradients_match_central_fd(0, True, 0),
    lambda: P.test_gradients_match_central_fd(2, True, 1),
    P.test_backward_upstream_matches_torch_autograd,
    P.test_update_is_plain_gd_step,
    P.test_one_epoch_equals_fd_gradient_step,
    P.test_loss_history_is_loss_before_each_update,
    P.test_minibatch_is_sequence_of_full_batch_steps,
    P.test_predict_threshold_and_tie,
    P.test_empty_input,
    P.test_zscore_statistics_match_numpy_population_moments,
    P.test_zscore_affine_invariance_constant_column_and_test_rows,
]


@pytest.fixture(scope="module")
def tmpdir_module():
    d = tempfile.mkdtemp(prefix="orc_mutants_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmpdir_module):
    src = open(oracle.SOURCE).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, "mutation site not found: " + name
    mutated = src.replace(old, new, 1)
    cpath = os.path.join(tmpdir_module, name + ".c")
    with open(cpath, "w") as f:
        f.write(mutated)
    so = oracle.compile_c(cpath, os.path.join(tmpdir_module, name + ".so"))
    caught = []
    with oracle.substituted_library(so):
        for pin in PINS:
            try:
                pin()
            except (AssertionError, ValueError, FloatingPointError):
                caught.append(getattr(pin, "__name__", "lambda"))
    assert caught, "no pin caught mutant " + name
