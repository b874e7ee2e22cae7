"""Pins for the oracle's selector functions (no GPU): BF16 rounding, the MLP loss and its
gradient, the FP32 inference emulation and decision rule, and the feature definition."""
import math

import numpy as np
import pytest

import oracle

P = oracle.SEL_PARAMS
O_W1, O_B1 = 0, 64 * 24
O_W2, O_B2 = O_B1 + 64, O_B1 + 64 + 64 * 64
O_W3, O_B3 = O_B2 + 64, O_B2 + 64 + 11 * 64


def test_bf16_rounding_closed_forms():
    assert oracle.bf16_round(1.0) == 1.0
    assert oracle.bf16_round(1.0 + 2 ** -8) == 1.0                 # tie -> even (mantissa ...0)
    assert oracle.bf16_round(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6   # tie -> even (rounds up)
    assert oracle.bf16_round(1.0 + 2 ** -8 + 2 ** -20) == 1.0 + 2 ** -7
    assert oracle.bf16_round(-3.0) == -3.0
    assert oracle.bf16_round(2.0 ** -130) == 2.0 ** -130           # subnormal float, 8 leading bits


def test_mlp_zero_network_closed_form():
    theta = np.zeros(P, np.float32)
    X = np.random.default_rng(0).normal(size=(5, 24)).astype(np.float32)
    y = np.array([0, 3, 10, 3, 7], np.int32)
    loss, g = oracle.mlp_loss_grad(theta, X, y)
    assert abs(loss - math.log(11)) < 1e-14
    # d loss / d b3 = mean(p - onehot) with p uniform
    exp_b3 = np.full(11, 1 / 11.0)
    for c in y:
        exp_b3[c] -= 1.0 / len(y)
    np.testing.assert_allclose(g[O_B3:O_B3 + 11], exp_b3, atol=1e-15)
    assert not g[:O_B3].any()  # zero weights and ReLU(0) = 0 block every other gradient


def _params(seed, scale=0.3):
    r = np.random.default_rng(seed)
    th = r.normal(0, scale, P).astype(np.float32)
    # weights exactly representable in BF16 so that +-1 BF16 ulp steps are exact perturbations
    for lo, hi in ((O_W1, O_B1), (O_W2, O_B2), (O_W3, O_B3)):
        th[lo:hi] = np.array([oracle.bf16_round(float(v)) for v in th[lo:hi]], np.float32)
    return th


@pytest.mark.parametrize("seed", [1, 2])
def test_mlp_gradient_finite_differences(seed):
    r = np.random.default_rng(100 + seed)
    th = _params(seed)
    X = r.normal(size=(6, 24)).astype(np.float32)
    y = r.integers(0, 11, 6).astype(np.int32)
    _, g = oracle.mlp_loss_grad(th, X, y)
    # biases: smooth central differences
    for idx in list(range(O_B1, O_B1 + 5)) + list(range(O_B2, O_B2 + 5)) + list(range(O_B3, O_B3 + 11)):
        h = 1e-3
        tp, tm = th.copy(), th.copy()
        tp[idx] += h
        tm[idx] -= h
        fd = (oracle.mlp_loss_grad(tp, X, y)[0] - oracle.mlp_loss_grad(tm, X, y)[0]) / (tp[idx] - tm[idx])
        assert abs(fd - g[idx]) <= 2e-3 * max(1.0, abs(g[idx])), idx
    # weights: +- one BF16 ulp (exact in the rounded forward pass); checks every layer's indexing
    for idx in (O_W1 + 3 * 24 + 5, O_W1 + 40 * 24 + 23, O_W2 + 7 * 64 + 50, O_W2 + 63 * 64 + 1,
                O_W3 + 2 * 64 + 9, O_W3 + 10 * 64 + 63):
        w = float(th[idx])
        ulp = 2.0 ** (math.frexp(w)[1] - 8) if w != 0 else 2.0 ** -20
        tp, tm = th.copy(), th.copy()
        tp[idx] = w + ulp
        tm[idx] = w - ulp
        assert oracle.bf16_round(float(tp[idx])) == tp[idx] and oracle.bf16_round(float(tm[idx])) == tm[idx]
        fd = (oracle.mlp_loss_grad(tp, X, y)[0] - oracle.mlp_loss_grad(tm, X, y)[0]) / (2 * ulp)
        assert abs(fd - g[idx]) <= 0.05 * abs(g[idx]) + 1e-4, (idx, fd, g[idx])


def test_mlp_select_closed_form_decision():
    # zero weights: the output probabilities are softmax(b3) -> decision from cumulative sums
    p = np.array([0.05, 0.10, 0.30, 0.40, 0.10, 0.05, 0, 0, 0, 0, 0], np.float64)
    b3 = np.log(np.maximum(p, 1e-30)).astype(np.float32)
    model = dict(mean=np.zeros(24, np.float32), inv_std=np.ones(24, np.float32),
                 W1=np.zeros(64 * 24, np.uint16), b1=np.zeros(64, np.float32),
                 W2=np.zeros(64 * 64, np.uint16), b2=np.zeros(64, np.float32),
                 W3=np.zeros(11 * 64, np.uint16), b3=b3, thr=0.8, s_lo=2, fallback=9)
    s, probs = oracle.mlp_select(model, np.zeros(24, np.float32), 12)
    np.testing.assert_allclose(probs, p, atol=1e-6)
    assert s == 2 + 3          # cumulative 0.05, 0.15, 0.45, 0.85 >= 0.8 at class 3
    model["thr"] = 0.99
    assert oracle.mlp_select(model, np.zeros(24, np.float32), 12)[0] == 2 + 5
    assert oracle.mlp_select(model, np.zeros(24, np.float32), 6)[0] == 6  # capped


def test_mlp_select_closed_form_through_all_layers():
    """A network whose decision depends on every layer: W1 = 0 with b1[0] = 1 gives h1 = e_0;
    W2[0][0] = 1 gives h2 = e_0 (ReLU keeps it); W3[4][0] = 5 gives z = 5 e_4, so
    p_4 = e^5 / (e^5 + 10) and the other classes 1 / (e^5 + 10): the cumulative sum first reaches
    0.9 at class 4 (s = 2 + 4).  The input (normalised by mean and inv_std) feeds a unit that
    ReLU cuts off (W1[1][0] = -1 with x_0 = 3) and that also enters h2_0: without the ReLU,
    h2_0 = 1 - 3 would vanish and the decision would fall to class 9."""
    bf = lambda v: np.array([v], np.float32).view(np.uint32)[0] >> 16   # exact BF16 bits of v
    W1 = np.zeros(64 * 24, np.uint16)
    W1[1 * 24 + 0] = bf(-1.0)
    b1 = np.zeros(64, np.float32)
    b1[0] = 1.0
    W2 = np.zeros(64 * 64, np.uint16)
    W2[0 * 64 + 0] = bf(1.0)
    W2[0 * 64 + 1] = bf(1.0)                        # h2_0 = h1_0 + h1_1 = 1 + relu(-3)
    W3 = np.zeros(11 * 64, np.uint16)
    W3[4 * 64 + 0] = bf(5.0)
    model = dict(mean=np.full(24, -1.0, np.float32), inv_std=np.full(24, 1.5, np.float32), W1=W1, b1=b1,
                 W2=W2, b2=np.zeros(64, np.float32), W3=W3, b3=np.zeros(11, np.float32),
                 thr=0.9, s_lo=2, fallback=13)
    feat = np.zeros(24, np.float32)
    feat[0] = 1.0                                   # x_0 = (1 - (-1)) * 1.5 = 3
    s, probs = oracle.mlp_select(model, feat, 12)
    want = np.full(11, 1.0 / (math.exp(5) + 10))
    want[4] = math.exp(5) / (math.exp(5) + 10)
    np.testing.assert_allclose(probs, want, rtol=1e-5)
    assert s == 2 + 4


def test_features_closed_forms():
    A = np.array([[1.0, 2.0 ** -5, 2.0 ** -40, 0.0],
                  [3.0, 3.0, 3.0, 3.0]])
    B = np.ones((4, 3))
    f = oracle.features(A, B, 1e-10)
    assert f[0] == 1.0 and f[1] == math.log2(3) and f[2] == 2.0
    # row 0: gaps 0, 5, 40, zero -> bins 0, 1, 9, 9 ; row 1: all gap 0 -> bin 0
    np.testing.assert_array_equal(f[3:13], np.array([5, 1, 0, 0, 0, 0, 0, 0, 0, 2], np.float32) / 8)
    np.testing.assert_array_equal(f[13:23], np.array([1, 0, 0, 0, 0, 0, 0, 0, 0, 0], np.float32))
    assert abs(f[23] + 10) < 1e-6
    g = oracle.features(np.asfortranarray(A.T), B, 1e-14, transa="T")
    np.testing.assert_array_equal(f[:23], g[:23])


def test_features_bin_edges():
    """Gaps on the bin edges: the row maximum 1.0 has frexp exponent 1; 2^-3, 2^-4, 2^-35 and
    2^-36 have gaps 3, 4, 35 and 36, so they fall in [0, 4), [4, 8), [32, 36) and the last bin."""
    A = np.array([[1.0, 2.0 ** -3, 2.0 ** -4, 2.0 ** -35, 2.0 ** -36]])
    f = oracle.features(A, np.ones((5, 1)), 1e-12)
    np.testing.assert_array_equal(f[3:13], np.array([2, 1, 0, 0, 0, 0, 0, 0, 1, 1], np.float32) / 5)


def test_selector_training_helpers_match_oracle_inference(tmp_path):
    """The training tool's NumPy forward pass and decision rule (used to choose the decision
    threshold on held-out GEMMs) agree with the oracle's FP32 emulation of the GPU inference."""
    from paper_2503_22875_gb300 import selector as S
    rng = np.random.default_rng(11)
    theta = S.init_params(3)
    X = rng.normal(size=(200, S.N_IN)).astype(np.float32)
    mean, std = X.mean(0), X.std(0) + 1e-3
    P = S.predict_probs(theta, mean, std, X)
    assert np.allclose(P.sum(1), 1, atol=1e-5)
    path = str(tmp_path / "m.ozgsel")
    S.write_model(path, theta, mean, std, 0.9, 13)
    model = S.read_model(path)
    agree = 0
    for x, p in zip(X, P):
        s_orc, probs = oracle.mlp_select(model, x, 13)
        assert np.allclose(probs, p, atol=2e-5)
        agree += int(S.decide(p[None], 0.9, 13)[0] == s_orc)
    assert agree >= 198  # ties at the threshold may round differently


def test_threshold_choice_minimises_expected_work():
    from paper_2503_22875_gb300 import selector as S
    # two classes of GEMMs: confident predictions make a low threshold cheap; the chosen
    # threshold must be the grid minimum of the stated cost
    probs = np.zeros((4, S.N_CLASSES), np.float32)
    probs[:, 5] = 0.92  # s = 7
    probs[:, 6] = 0.08  # s = 8
    s_min = np.array([7, 7, 7, 8])
    work = np.ones(4)
    best, table = S.choose_threshold(probs, s_min, work, 13)
    costs = {t: v["cost"] for t, v in table.items()}
    assert costs[best] == min(costs.values())
    # at thr <= 0.92 every GEMM runs at s = 7 and the one that needs 8 is rejected by the check
    # and re-runs at s + 2 = 9 (45 products); above, all run at s = 8
    assert table[0.9]["cost"] == 4 * 28 + 45 and table[0.95]["cost"] == 4 * 36
    # with a fallback of 8 the re-run stops at the fallback (36 products)
    _, table8 = S.choose_threshold(probs, s_min, work, 8)
    assert table8[0.9]["cost"] == 4 * 28 + 36
