"""Surrogate MLP: the FP64 oracle against finite differences and an independent
bfloat16 conversion (CPU), and the tensor-core kernels against the oracle (GPU)."""
import numpy as np
import pytest

from oracle.mlp import MLPOracle, bf16_round, ensemble_stats, gelu, gelu_grad


def test_oracle_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    m = MLPOracle([5, 7, 6, 3])
    p = m.init_params(rng)
    x = rng.normal(size=(4, 5))
    t = rng.normal(size=(4, 3))
    _, g = m.loss_and_grad(p, x, t)
    eps = 1e-6
    for i in rng.choice(m.n_params, 40, replace=False):
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        num = (m.loss_and_grad(pp, x, t)[0] - m.loss_and_grad(pm, x, t)[0]) / (2 * eps)
        assert abs(num - g[i]) <= 1e-6 * max(1.0, abs(num)), (i, num, g[i])


def test_gelu_derivative_and_values():
    z = np.linspace(-6, 6, 101)
    np.testing.assert_allclose(gelu_grad(z), (gelu(z + 1e-6) - gelu(z - 1e-6)) / 2e-6, rtol=1e-6, atol=1e-9)
    # GELU(z) -> z for large z, -> 0 for very negative z, GELU(0) = 0
    assert abs(gelu(np.array(8.0)) - 8.0) < 1e-12 and abs(gelu(np.array(-8.0))) < 1e-12 and gelu(np.array(0.0)) == 0


def test_bf16_round_matches_torch():
    import torch
    rng = np.random.default_rng(1)
    a = np.concatenate([rng.normal(size=2000) * 10 ** rng.uniform(-8, 8, 2000), [0.0, -0.0, 1.0, 3.0 / 7.0]])
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(bf16_round(a), ref)


def test_oracle_adam_first_step_is_sign_times_lr():
    """With zero moments the first Adam step moves every parameter by lr * sign(g)
    (up to eps): the bias corrections cancel the (1 - beta) factors."""
    p = np.zeros(5)
    g = np.array([1.0, -2.0, 0.5, -1e-3, 3.0])
    p1, _, _ = MLPOracle.adam(p, g, np.zeros(5), np.zeros(5), 1, lr=1e-3)
    np.testing.assert_allclose(p1, -1e-3 * np.sign(g), rtol=1e-4)



def test_ensemble_stats_closed_forms():
    """Two members a, b: mean (a + b)/2 and std |a - b|/2; identical members:
    std 0 and no fallback; the affine map applies before the statistics."""
    a = np.array([[1.0, 5.0, -2.0]])
    b = np.array([[3.0, 5.0, 2.0]])
    mean, std, spread, fb = ensemble_stats([a, b], n_spread=2, tol=0.5)
    np.testing.assert_array_equal(mean, [[2.0, 5.0, 0.0]])
    np.testing.assert_array_equal(std, [[1.0, 0.0, 2.0]])
    assert spread[0] == 1.0 and fb[0]  # the third output is outside n_spread
    mean, std, spread, fb = ensemble_stats([a, a, a], scale=[2.0, 1.0, 1.0], shift=[1.0, 0.0, 0.0], n_spread=3, tol=0.0)
    np.testing.assert_array_equal(mean, [[3.0, 5.0, -2.0]])
    assert np.all(std == 0) and spread[0] == 0 and not fb[0]
    # a row factor on the first output only, then an offset: std scales with |row|
    mean, std, _, _ = ensemble_stats([a, b], row=[3.0], n_row=1, offset=[10.0, 0.0, 0.0])
    np.testing.assert_array_equal(mean, [[16.0, 5.0, 0.0]])
    np.testing.assert_array_equal(std, [[3.0, 0.0, 2.0]])

# ---------------------------------------------------------------------------
# GPU: tensor-core kernels against the oracle with the same bf16 rounding
# ---------------------------------------------------------------------------
def _rel(a, b):
    return np.linalg.norm(np.asarray(a, float) - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.gpu
@pytest.mark.parametrize("dims,B", [([12, 128, 256, 128], 128), ([12, 512, 512, 512, 512, 512, 1024], 256)])
def test_mlp_forward_and_gradients_match_oracle(dims, B):
    import torch

    from paper_2009_10400_b300.mlp import MLP
    rng = np.random.default_rng(3)
    orc = MLPOracle(dims)
    p = orc.init_params(rng).astype(np.float32).astype(np.float64)
    x = rng.uniform(-1, 1, (B, dims[0]))
    t = rng.normal(size=(B, dims[-1])) * 0.1
    net = MLP(dims, max_batch=max(B, 256))
    net.set_params(p)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    td = torch.tensor(t, dtype=torch.float32, device="cuda")
    y = net.forward(xd)
    g, loss = net.gradients(xd, td)
    net.sync()
    x32 = x.astype(np.float32).astype(np.float64)
    t32 = t.astype(np.float32).astype(np.float64)
    y_ref, _, _ = orc.forward(p, x32, bf16=True)
    loss_ref, g_ref = orc.loss_and_grad(p, x32, t32, bf16=True)
    assert _rel(y.cpu().numpy(), y_ref) < 2e-3, _rel(y.cpu().numpy(), y_ref)
    assert abs(loss.item() - loss_ref) < 2e-3 * loss_ref
    g = g.cpu().numpy()
    for (a, b, c, N, K) in orc.offsets:  # per layer, weights and biases
        assert _rel(g[a:b], g_ref[a:b]) < 1e-2, ("W", N, K, _rel(g[a:b], g_ref[a:b]))
        assert _rel(g[b:c], g_ref[b:c]) < 1e-2, ("b", N, _rel(g[b:c], g_ref[b:c]))
    # and against the unrounded FP64 gradient, the bf16 training precision
    _, g64 = orc.loss_and_grad(p, x32, t32, bf16=False)
    assert _rel(g, g64) < 5e-2


@pytest.mark.gpu
def test_mlp_adam_step_and_training_reduces_loss():
    import torch

    from paper_2009_10400_b300.mlp import MLP
    rng = np.random.default_rng(4)
    dims = [12, 256, 256, 128]
    orc = MLPOracle(dims)
    p = orc.init_params(rng).astype(np.float32).astype(np.float64)
    B = 256
    x = rng.uniform(-1, 1, (B, 12))
    w_true = rng.normal(size=(12, 128)) / 4
    t = np.tanh(x @ w_true)
    net = MLP(dims, max_batch=B)
    net.set_params(p)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    td = torch.tensor(t, dtype=torch.float32, device="cuda")
    net.train_step(xd, td, 1e-3)
    net.sync()
    p1 = net.get_params().astype(np.float64)
    _, g_ref = orc.loss_and_grad(p, x.astype(np.float32).astype(np.float64), t.astype(np.float32).astype(np.float64),
                                 bf16=True)
    p1_ref, _, _ = MLPOracle.adam(p, g_ref, np.zeros_like(p), np.zeros_like(p), 1, 1e-3)
    moved = np.abs(p1_ref - p) > 5e-4  # parameters with a clear gradient sign
    assert np.mean(np.sign(p1 - p)[moved] == np.sign(p1_ref - p)[moved]) > 0.98
    losses = []
    for _ in range(300):
        losses.append(net.train_step(xd, td, 1e-3).item())
    net.sync()
    assert losses[-1] < 0.2 * losses[0], (losses[0], losses[-1])



@pytest.mark.gpu
def test_ensemble_kernel_matches_oracle():
    import torch

    from paper_2009_10400_b300.mlp import ensemble
    rng = np.random.default_rng(7)
    B, N, E = 300, 1000, 5
    ys = [rng.normal(size=(B, N)).astype(np.float32) for _ in range(E)]
    scale = rng.uniform(0.5, 3.0, N).astype(np.float32)
    shift = rng.uniform(-40, 40, N).astype(np.float32)
    d = [torch.tensor(y, device="cuda") for y in ys]
    X = rng.uniform(1e6, 1e7, (B, 12)).astype(np.float32)  # raw input rows; column 0 gives the row factor
    offset = np.where(np.arange(N) < 500, 37.0, 0.0).astype(np.float32)
    mean, std, spread, fb = ensemble(d, torch.tensor(scale, device="cuda"), torch.tensor(shift, device="cuda"),
                                     n_spread=700, tol=4.0, row_src=torch.tensor(X, device="cuda"), row_mult=2e-7,
                                     n_row_scaled=500, out_offset=torch.tensor(offset, device="cuda"))
    torch.cuda.synchronize()
    m_ref, s_ref, sp_ref, fb_ref = ensemble_stats(ys, scale, shift, n_spread=700, tol=4.0,
                                                  row=X[:, 0].astype(np.float64) * 2e-7, n_row=500, offset=offset)
    np.testing.assert_allclose(mean.cpu().numpy(), m_ref, rtol=1e-5, atol=2e-5 * np.abs(m_ref).max())
    np.testing.assert_allclose(std.cpu().numpy(), s_ref, rtol=1e-4, atol=1e-5)
    np.testing.assert_allclose(spread.cpu().numpy(), sp_ref, rtol=1e-4)
    clear = np.abs(sp_ref - 4.0) > 1e-3 * 4.0  # decisions away from the threshold are exact
    assert clear.sum() > B // 2
    np.testing.assert_array_equal(fb.cpu().numpy().astype(bool)[clear], fb_ref[clear])


@pytest.mark.gpu
def test_input_scaling_and_row_gather():
    """The input map inside the first kernel equals scaling the inputs on the
    host (same FP32 arithmetic: bitwise), and an Adam step on gathered rows of
    a device data set equals a step on the copied rows (bitwise)."""
    import torch

    from paper_2009_10400_b300.mlp import MLP
    rng = np.random.default_rng(8)
    dims = [12, 128, 256]
    p = MLPOracle(dims).init_params(rng).astype(np.float32)
    shift = rng.uniform(-1, 1, 12).astype(np.float32)
    scale = rng.uniform(0.1, 2.0, 12).astype(np.float32)
    x = rng.uniform(-3, 3, (512, 12)).astype(np.float32)
    t = rng.normal(size=(512, 256)).astype(np.float32)
    a, b = MLP(dims, max_batch=256), MLP(dims, max_batch=256)
    a.set_params(p)
    b.set_params(p)
    a.set_input_scaling(shift, scale)
    xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
    xs = torch.tensor((x - shift) * scale, device="cuda")
    ya = a.forward(xd[:256]).cpu().numpy()
    yb = b.forward(xs[:256]).cpu().numpy()
    np.testing.assert_array_equal(ya, yb)
    rows = rng.permutation(512)[:256].astype(np.int32)
    rd = torch.tensor(rows, device="cuda")
    for _ in range(3):
        la = a.train_step_rows(xd, td, rd, 1e-3).item()
        lb = b.train_step(xs[rd.long()].contiguous(), td[rd.long()].contiguous(), 1e-3).item()
        assert la == lb
    a.sync()
    b.sync()
    np.testing.assert_array_equal(a.get_params(), b.get_params())


@pytest.mark.gpu
@pytest.mark.parametrize("norm", [0, 1])
def test_surrogate_engine_transform_standardisation_and_training(norm):
    """The surrogate engine (tled_sur): temperatures learned as rise per unit
    source power and standardised (per output, or one scale per output group),
    checked through networks whose outputs are known -- all zero (answer: the
    column means mapped back) and all one (answer: mean + scale); then seeded
    training is reproducible and fits its data."""
    import torch

    from paper_2009_10400_b300.mlp import SurrogateEngine
    rng = np.random.default_rng(11)
    n, n_in, n_out, n_T = 512, 12, 256, 128
    dims = [n_in, 128, 128, n_out]
    X = rng.uniform(0.0, 1.0, (n, n_in))
    X[:, 0] = rng.uniform(1e6, 1e7, n)  # source power, W/m^3
    feat = X.copy()
    feat[:, 0] = (X[:, 0] - 5.5e6) / 4.5e6
    w1 = rng.normal(size=(n_in, n_out)) / 2  # a smooth function of the inputs, learnable
    base = np.tanh(feat @ w1) * np.linspace(0.1, 3.0, n_out) + np.linspace(-1, 1, n_out)
    Y = base.copy()
    Y[:, :n_T] = 37.0 + (X[:, :1] / 5e6) * (2.0 + np.abs(base[:, :n_T]))  # temperatures, linear in power
    eng = SurrogateEngine(dims, 3, n_T, max_batch=512, max_rows=1024, max_epochs=8)
    eng.set_inputs(np.zeros(n_in), np.concatenate([[1e7], np.ones(n_in - 1)]))
    eng.set_outputs(0, 5e6, 37.0, norm)
    xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    yd = torch.tensor(Y, dtype=torch.float32, device="cuda")
    hist = eng.train(xd, yd, epochs=8, batch=128, lr=2e-3, seed=3)
    assert hist.shape == (3, 8) and np.all(hist[:, -1] < 0.8 * hist[:, 0]), hist
    # the transform and its statistics, in FP64 here
    Z = Y.copy()
    Z[:, :n_T] = (Y[:, :n_T] - 37.0) / (X[:, :1] / 5e6)
    mu, sd = Z.mean(0), Z.std(0)
    if norm == 1:
        sd = np.concatenate([np.full(n_T, np.sqrt(np.mean(sd[:n_T] ** 2))),
                             np.full(n_out - n_T, np.sqrt(np.mean(sd[n_T:] ** 2)))])
    row = np.concatenate([X[:, :1] / 5e6 * np.ones((1, n_T)), np.ones((n, n_out - n_T))], 1)
    off = np.concatenate([np.full(n_T, 37.0), np.zeros(n_out - n_T)])
    n_par = sum(k * m + m for k, m in zip(dims[:-1], dims[1:]))
    mean = torch.empty(n, n_out, device="cuda")
    std = torch.empty(n, n_out, device="cuda")
    spread = torch.empty(n, device="cuda")
    fb = torch.empty(n, dtype=torch.uint8, device="cuda")
    for level in (0.0, 1.0):  # every member answers `level` (standardised) for every output
        p = np.zeros(n_par, np.float32)
        p[-n_out:] = level  # last layer bias
        for k in range(3):
            eng.set_member_params(k, p)
        eng.predict(xd, n_T, 0.5, mean, std, spread, fb)
        eng.sync()
        expect = (mu + level * sd) * row + off
        np.testing.assert_allclose(mean.cpu().numpy(), expect, rtol=2e-5, atol=2e-5 * np.abs(expect).max())
        # identical members: the spread is rounding of the ensemble mean only
        rnd = 1e-6 * np.abs(expect).max()
        assert float(std.abs().max()) <= rnd and float(spread.max()) <= rnd and int(fb.sum()) == 0
    # seeded training is reproducible (graph-replayed epochs, members side by side)
    eng.train(xd, yd, epochs=8, batch=128, lr=2e-3, seed=3)
    p_a = [eng.member_params(k) for k in range(3)]
    eng.train(xd, yd, epochs=8, batch=128, lr=2e-3, seed=3)
    for k in range(3):
        np.testing.assert_array_equal(eng.member_params(k), p_a[k])
    assert not np.array_equal(p_a[0], p_a[1])  # the members start and shuffle differently


@pytest.mark.gpu
def test_surrogate_engine_symmetry_augmentation():
    """Training-set augmentation: with the identity and a map that mirrors input 1
    (x' = 1 - x) and reverses the outputs, the engine trains on both copies of
    every row; networks answering zero then return the column means of the
    augmented, transformed targets (computed here in FP64)."""
    import torch

    from paper_2009_10400_b300.mlp import SurrogateEngine
    rng = np.random.default_rng(12)
    n, n_in, n_out, n_T = 256, 4, 128, 64
    dims = [n_in, 128, n_out]
    X = rng.uniform(0.0, 1.0, (n, n_in))
    X[:, 0] = rng.uniform(1e6, 1e7, n)
    Y = rng.normal(size=(n, n_out)) * 3.0
    Y[:, :n_T] += 37.0
    src = np.tile(np.arange(n_in), (2, 1))
    a, b = np.ones((2, n_in)), np.zeros((2, n_in))
    a[1, 1], b[1, 1] = -1.0, 1.0
    perm = np.stack([np.arange(n_out), np.arange(n_out)[::-1]])
    eng = SurrogateEngine(dims, 2, n_T, max_batch=256, max_rows=2 * n, max_epochs=2, max_sym=2)
    eng.set_symmetries(src, a, b, perm)
    eng.set_outputs(0, 5e6, 37.0, 0)
    xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    yd = torch.tensor(Y, dtype=torch.float32, device="cuda")
    eng.train(xd, yd, epochs=1, batch=128, lr=1e-3, seed=1)
    Xa = np.concatenate([X, X * a[1] + b[1]])
    Ya = np.concatenate([Y, Y[:, perm[1]]])
    Za = Ya.copy()
    Za[:, :n_T] = (Ya[:, :n_T] - 37.0) / (Xa[:, :1] / 5e6)
    mu = Za.mean(0)
    n_par = sum(k * m + m for k, m in zip(dims[:-1], dims[1:]))
    for k in range(2):
        eng.set_member_params(k, np.zeros(n_par, np.float32))
    mean = torch.empty(n, n_out, device="cuda")
    eng.predict(xd, n_T, 1.0, mean)
    eng.sync()
    row = np.concatenate([X[:, :1] / 5e6 * np.ones((1, n_T)), np.ones((n, n_out - n_T))], 1)
    expect = mu * row + np.concatenate([np.full(n_T, 37.0), np.zeros(n_out - n_T)])
    np.testing.assert_allclose(mean.cpu().numpy(), expect, rtol=2e-5, atol=2e-5 * np.abs(expect).max())
    # rows beyond max_rows after augmentation are refused
    big = torch.zeros(2 * n + 128, n_in, device="cuda")
    with pytest.raises(Exception):
        eng.train(big, torch.zeros(2 * n + 128, n_out, device="cuda"), epochs=1, batch=128, lr=1e-3, seed=1)
