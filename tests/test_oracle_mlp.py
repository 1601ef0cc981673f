"""Pins of the oracle's learned-guess reference (oracle/mlp_oracle.c): each
check ties it to something other than its own formulas -- identities of the
tanh-form GELU, finite differences, a network whose output is known in closed
form, the closed forms of the first Adam steps, library bfloat16 rounding and
the star pressures of Toro's Table 4.3."""
import math

import numpy as np
import pytest

from conftest import read_golden

NP = 4673
OFF_W1, OFF_B1, OFF_W2, OFF_B2, OFF_W3, OFF_B3 = 0, 384, 448, 4544, 4608, 4672


def test_layout(oracle_mod):
    assert oracle_mod.mlp_n_params() == NP == 64 * 6 + 64 + 64 * 64 + 64 + 64 + 1


@pytest.mark.parametrize("x", [0.0, 1e-3, 0.3, -0.7, 1.0, 2.5, -4.0, 7.0])
def test_gelu_odd_part_is_identity(oracle_mod, x):
    # x/2 (1 + tanh u) - (-x/2)(1 - tanh u) = x for any odd u(x)
    g = oracle_mod.gelu
    assert g(x) - g(-x) == pytest.approx(x, rel=1e-15, abs=1e-300)


def test_gelu_limits_and_slope(oracle_mod):
    assert oracle_mod.gelu(0.0) == 0.0
    assert oracle_mod.gelu(10.0) == 10.0     # tanh saturates to 1 in binary64
    assert oracle_mod.gelu(-10.0) == 0.0
    assert oracle_mod.gelu_grad(0.0) == 0.5
    # the erf form's value at 1 is 0.841345; the tanh form differs by < 2e-4
    assert abs(oracle_mod.gelu(1.0) - 0.5 * (1 + math.erf(1 / math.sqrt(2)))) < 2e-4


@pytest.mark.parametrize("x", [-3.0, -1.2, -0.4, 0.05, 0.6, 1.7, 3.3])
def test_gelu_grad_against_differences(oracle_mod, x):
    h = 1e-5
    fd = (oracle_mod.gelu(x + h) - oracle_mod.gelu(x - h)) / (2 * h)
    assert oracle_mod.gelu_grad(x) == pytest.approx(fd, abs=1e-9)


def mirrored_network(rng):
    """Units k and k+32 of each hidden layer see opposite pre-activations,
    and the next layer takes their difference, so gelu(a) - gelu(-a) = a
    makes the whole network the affine map  y = c.(V (W x + beta) + d) + b3."""
    W = rng.normal(size=(32, 6))
    beta = rng.normal(size=32)
    V = rng.normal(size=(32, 32)) * 0.3
    d = rng.normal(size=32)
    c = rng.normal(size=32)
    b3 = 0.25
    th = np.zeros(NP)
    W1 = np.vstack([W, -W])
    b1 = np.concatenate([beta, -beta])
    W2h = np.hstack([V, -V])                 # a2_o = sum_k V_ok (h1_k - h1_{k+32}) + d_o
    W2 = np.vstack([W2h, -W2h])
    b2 = np.concatenate([d, -d])
    w3 = np.concatenate([c, -c])
    th[OFF_W1:OFF_B1] = W1.ravel()
    th[OFF_B1:OFF_W2] = b1
    th[OFF_W2:OFF_B2] = W2.ravel()
    th[OFF_B2:OFF_W3] = b2
    th[OFF_W3:OFF_B3] = w3
    th[OFF_B3] = b3
    return th, (W, beta, V, d, c, b3)


def test_forward_mirrored_network_is_affine(oracle_mod):
    rng = np.random.default_rng(11)
    th, (W, beta, V, d, c, b3) = mirrored_network(rng)
    x = rng.normal(size=(50, 6))
    want = (V @ (W @ x.T + beta[:, None]) + d[:, None]).T @ c + b3
    got = oracle_mod.mlp_forward(th, x)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)
    # a transposed second layer would not reproduce it (V is not symmetric)
    th_t = th.copy()
    th_t[OFF_W2:OFF_B2] = th[OFF_W2:OFF_B2].reshape(64, 64).T.ravel()
    assert not np.allclose(oracle_mod.mlp_forward(th_t, x), want, rtol=1e-6)


def random_theta(rng, scale=0.4):
    th = rng.normal(size=NP) * scale
    th[OFF_W1:OFF_B1] /= math.sqrt(6)
    th[OFF_W2:OFF_B2] /= 8.0
    th[OFF_W3:OFF_B3] /= 8.0
    return th


def test_loss_grad_against_central_differences(oracle_mod):
    rng = np.random.default_rng(5)
    th = random_theta(rng)
    x = rng.normal(size=(4, 6)) + 1.0
    t = rng.normal(size=4)
    loss, g = oracle_mod.mlp_loss_grad(th, x, t)
    y = oracle_mod.mlp_forward(th, x)
    assert loss == pytest.approx(np.mean((y - t) ** 2), rel=1e-14)
    # every parameter of the small layers, a sample of the 64x64 one
    idx = list(range(OFF_W1, OFF_W2)) + list(range(OFF_B2, NP))
    idx += list(rng.choice(np.arange(OFF_W2, OFF_B2), 400, replace=False))
    h = 1e-6
    for k in idx:
        tp = th.copy()
        tm = th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (np.mean((oracle_mod.mlp_forward(tp, x) - t) ** 2)
              - np.mean((oracle_mod.mlp_forward(tm, x) - t) ** 2)) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-9), k


def test_adam_first_two_steps_closed_form(oracle_mod):
    rng = np.random.default_rng(2)
    n = 32
    th0 = rng.normal(size=n)
    g1 = rng.normal(size=n)
    g2 = rng.normal(size=n)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    th = th0.copy()
    m = np.zeros(n)
    v = np.zeros(n)
    oracle_mod.adam_step(th, m, v, g1, 1, lr, b1, b2, eps)
    # bias-corrected moments after one step are g and g^2
    th1 = th0 - lr * g1 / (np.abs(g1) + eps)
    assert np.allclose(th, th1, rtol=0, atol=1e-15)
    oracle_mod.adam_step(th, m, v, g2, 2, lr, b1, b2, eps)
    mh = (b1 * g1 + g2) / (1 + b1)
    vh = (b2 * g1 ** 2 + g2 ** 2) / (1 + b2)
    assert np.allclose(th, th1 - lr * mh / (np.sqrt(vh) + eps), rtol=0, atol=1e-14)


def test_bf16_rounding_against_library(oracle_mod):
    torch = pytest.importorskip("torch")
    # ties to even at 1 + 2^-8 (down) and at 1 + 2^-7 + 2^-8 (up)
    assert oracle_mod.bf16_round(1 + 2 ** -8) == 1.0
    assert oracle_mod.bf16_round(1 + 2 ** -7 + 2 ** -8) == 1 + 2 ** -6
    assert oracle_mod.bf16_round(1 + 3 * 2 ** -9) == 1 + 2 ** -7
    rng = np.random.default_rng(3)
    v = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-6, 6, size=2000),
                        np.float32(1) + np.arange(-300, 300) * np.float32(2 ** -16)]).astype(np.float32)
    lib = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    ours = np.array([oracle_mod.bf16_round(float(a)) for a in v])
    assert np.array_equal(lib, ours)


def test_forward_bf16_against_library_quantisation(oracle_mod):
    """The quantised forward pass against the same pass written with torch's
    bfloat16 casts: quantisation points and layer order must agree."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    th = random_theta(rng).astype(np.float32)
    x = (rng.normal(size=(40, 6)) * 0.5 + 1.0).astype(np.float32)
    q = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.float64)
    W1 = q(th[OFF_W1:OFF_B1].reshape(64, 6))
    W2 = q(th[OFF_W2:OFF_B2].reshape(64, 64))
    gelu = lambda a: 0.5 * a * (1 + torch.tanh(math.sqrt(2 / math.pi) * (a + 0.044715 * a ** 3)))
    a1 = q(x) @ W1.T + t(th[OFF_B1:OFF_W2])
    h1 = gelu(a1).to(torch.float32).to(torch.bfloat16).to(torch.float64)
    a2 = h1 @ W2.T + t(th[OFF_B2:OFF_W3])
    y = gelu(a2) @ t(th[OFF_W3:OFF_B3]) + float(th[OFF_B3])
    ours = oracle_mod.mlp_forward_bf16(th, x)
    assert np.allclose(ours, y.numpy(), rtol=1e-12, atol=1e-12)
    # and the quantisation matters at the level bfloat16 predicts
    full = oracle_mod.mlp_forward(th.astype(np.float64), x.astype(np.float64))
    assert 1e-5 < np.max(np.abs(full - ours)) < 0.05


def test_features_of_mirrored_states(oracle_mod):
    r, u, p, g = 1.3, 0.4, 2.0, 1.4
    x, pb, ptr = oracle_mod.mlp_features([[r, u, p, r, -u, p]], gamma=g)
    a = math.sqrt(g * p / r)
    assert np.allclose(x[0], [0, u / a, 0, 0, -u / a, 0], rtol=1e-15, atol=0)
    assert pb[0] == p
    # a common velocity drops out (the star pressure is Galilean invariant)
    x2, _, _ = oracle_mod.mlp_features([[r, u + 5.0, p, r, -u + 5.0, p]], gamma=g)
    assert np.allclose(x2, x, rtol=1e-14, atol=1e-15)
    # left/right deviations are opposite; Sod's are the relative jumps
    x3, _, _ = oracle_mod.mlp_features([[1.0, 0.0, 1.0, 0.125, 0.0, 0.1]])
    assert np.allclose(x3[0], [0.875 / 1.125, 0, 0.9 / 1.1, -0.875 / 1.125, 0, -0.9 / 1.1], rtol=1e-15)
    # identical states at rest: the two-rarefaction guess is exact
    _, _, ptr = oracle_mod.mlp_features([[r, 0.0, p, r, 0.0, p]], gamma=g)
    assert ptr[0] == pytest.approx(p, rel=1e-14)


def test_tr_guess_exact_for_two_rarefactions_and_sod_target(oracle_mod):
    rows = [[float(v) for v in ln.split()] for ln in read_golden("toro_table_4_3.txt")]
    # Toro test 2 (123 problem): two rarefactions, where the guess is the
    # exact star pressure (printed as 0.00189)
    t2 = rows[1]
    assert oracle_mod.tr_guess(t2[:6]) == pytest.approx(t2[6], abs=5e-6)
    # Sod (test 1): a shock on the right; the guess differs, the target is
    # log(p*/pbar) with p* from the table
    t1 = rows[0]
    x, pb, ptr = oracle_mod.mlp_features([t1[:6]])
    assert pb[0] == 0.55
    ps, _, _ = oracle_mod.riemann(t1[0:3], t1[3:6], tol=1e-14, maxit=100)
    assert math.log(ps / pb[0]) == pytest.approx(math.log(t1[6] / 0.55), abs=2e-5)
    assert ptr[0] > t1[6] * 1.005


def test_target_scaling(oracle_mod):
    rows = [[float(v) for v in ln.split()] for ln in read_golden("toro_table_4_3.txt")]
    # two rarefactions (Toro test 2): q <= 0 and the target is exactly 0
    t2 = rows[1]
    y, q = oracle_mod.mlp_target(t2[:6], 1, t2[6])
    assert q <= 0 and y == 0.0
    # s(q) = (q/(1+q))^3: q^3 for weak shocks, bounded by 1 for strong ones
    assert oracle_mod.shock_scale(1e-2) == pytest.approx(1e-6 / 1.01 ** 3, rel=1e-14)
    assert oracle_mod.shock_scale(1.0) == 0.125
    assert oracle_mod.shock_scale(1e6) == pytest.approx(1.0, rel=4e-6)
    assert oracle_mod.shock_scale(-0.5) == 0.0
    # Toro test 3 (q ~ 9e4): the target is log(p*/p_TR) itself, of order one
    t3 = rows[2]
    y3, q3 = oracle_mod.mlp_target(t3[:6], 1, t3[6])
    assert q3 > 1e4 and -1.0 < y3 < -0.3
    # a weak shock: log(p*/p_TR) shrinks like q^3, so the scaled target stays
    # of order one as the jump vanishes
    ys = []
    for eps in (0.2, 0.1, 0.05):
        pair = [1.0, 0.0, 1.0 + eps, 1.0, 0.0, 1.0]
        ps, _, _ = oracle_mod.riemann(pair[:3], pair[3:], tol=1e-15, maxit=100)
        y, q = oracle_mod.mlp_target(pair, 1, ps)
        assert q > 0
        ys.append(y)
    assert all(abs(v) < 1.0 for v in ys) and abs(ys[2] - ys[1]) < abs(ys[1] - ys[0])
    # target 0 is log(p*/pbar)
    t1 = rows[0]
    y0, _ = oracle_mod.mlp_target(t1[:6], 0, t1[6])
    assert y0 == pytest.approx(math.log(t1[6] / 0.55), rel=1e-14)
