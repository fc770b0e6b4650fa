"""Pins of the FP64 reference of the correction network."""
import numpy as np
import pytest

from oracle import mlp
from workloads.water import init_mlp_params


def test_bf16_round_matches_library():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = (rng.normal(size=2000) * 10.0 ** rng.uniform(-5, 5, size=2000)).astype(np.float32)
    x = np.concatenate([x, np.float32([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 0.0])])
    ref = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)


def test_parameter_layout_of_both_widths():
    assert mlp.n_params(48) == mlp.N_PARAMS == 7491
    assert mlp.n_params(32) == 6467
    assert mlp.width_of(np.zeros(7491)) == 48 and mlp.width_of(np.zeros(6467)) == 32
    with pytest.raises(ValueError):
        mlp.width_of(np.zeros(7490))
    # pack inverts unpack, the blocks in the documented order
    theta = np.arange(6467, dtype=np.float64)
    p = mlp.unpack(theta)
    assert p["W1"].shape == (64, 32) and p["W1"][1, 0] == 32 and p["b1"][0] == 2048
    assert p["W3"].shape == (3, 64) and p["b3"][2] == 6466
    assert np.array_equal(mlp.pack(p), theta)


@pytest.mark.parametrize("n_in", [48, 32])
def test_gradient_matches_central_differences(n_in):
    rng = np.random.default_rng(1)
    theta = init_mlp_params(3, n_in=n_in).astype(np.float64)
    theta[64 * n_in:64 * n_in + 64] = rng.normal(size=64) * 0.1  # nonzero b1
    X = rng.normal(size=(20, n_in))
    T = rng.normal(size=(20, 3))
    _, g = mlp.loss_and_grad(theta, X, T, bf16=False)
    h = 1e-6
    idx = rng.choice(mlp.n_params(n_in), size=120, replace=False)
    fd = np.empty(len(idx))
    for k, j in enumerate(idx):
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        fd[k] = (mlp.loss_and_grad(tp, X, T, bf16=False)[0] - mlp.loss_and_grad(tm, X, T, bf16=False)[0]) / (2 * h)
    assert np.max(np.abs(fd - g[idx])) <= 1e-6 * max(1.0, np.max(np.abs(g[idx])))


@pytest.mark.parametrize("n_in", [48, 32])
def test_zero_weights_give_bias_and_linear_regime(n_in):
    p = {name: np.zeros(shape) for name, shape in mlp.shapes(n_in)}
    p["b3"] = np.array([0.5, -1.0, 2.0])
    y, _ = mlp.forward(mlp.pack(p), np.ones((4, n_in)), bf16=False)
    assert np.allclose(y, p["b3"])
    # small weights: tanh is the identity to third order, so y = W3 W2 W1 x
    rng = np.random.default_rng(2)
    for name, shape in mlp.shapes(n_in):
        p[name] = rng.normal(size=shape) * (1e-5 if name.startswith("W") else 0.0)
    x = rng.normal(size=(5, n_in))
    y, _ = mlp.forward(mlp.pack(p), x, bf16=False)
    lin = x @ (p["W3"] @ p["W2"] @ p["W1"]).T
    assert np.max(np.abs(y - lin)) <= 1e-6 * np.max(np.abs(lin))


# ---------------------------------------------------------------- features
from oracle.pppm import bspline_M  # noqa: E402


def test_cardinal_bspline_integer_values():
    # the centred cardinal B-spline of order 5 at the integers: 115/192, 19/96, 1/384
    v = bspline_M(5, np.array([0.0, 1.0, -1.0, 2.0, -2.0, 2.5]))
    assert np.allclose(v, [115 / 192, 19 / 96, 19 / 96, 1 / 384, 1 / 384, 0.0], rtol=0, atol=1e-15)


@pytest.mark.parametrize("kind,width,zero_from", [("cell", 48, 36), ("stated", 32, 30)])
def test_features_constant_mesh_and_one_hot(kind, width, zero_from):
    rng = np.random.default_rng(4)
    box, mesh = np.array([9.0, 10.0, 11.0]), (8, 10, 12)
    phi = np.full(mesh, 2.5)
    pos = rng.uniform(-3.0, 14.0, size=(17, 3))
    types = rng.integers(0, 3, size=17).astype(np.int8)
    for p in (3, 4, 5):
        X = mlp.features(phi, pos, types, box, mesh, p, s_in=0.5, kind=kind)
        assert X.shape == (17, width)
        assert np.allclose(X[:, :27], 1.25, rtol=0, atol=1e-13)   # partition of unity
        assert np.array_equal(X[:, 27:30], np.eye(3)[types])
        assert not X[:, zero_from:].any()


def test_stated_features_are_the_samples_and_type_alone():
    """The stated set is the first 30 inputs of the cell set (same samples,
    same type code) and two zeros: no position inside the cell."""
    rng = np.random.default_rng(12)
    box, mesh = np.array([7.0, 8.0, 9.0]), (10, 12, 15)
    phi = rng.normal(size=mesh)
    pos = rng.uniform(-1.0, 10.0, size=(9, 3))
    types = rng.integers(0, 3, size=9).astype(np.int8)
    Xc = mlp.features(phi, pos, types, box, mesh, 5, s_in=0.8, kind="cell")
    Xs = mlp.features(phi, pos, types, box, mesh, 5, s_in=0.8, kind="stated")
    assert np.array_equal(Xs[:, :30], Xc[:, :30]) and not Xs[:, 30:].any()
    # translating the sites by one mesh cell along x and phi by one index
    # along x gives the same inputs (the samples follow the potential)
    Xs2 = mlp.features(np.roll(phi, 1, axis=0), pos + np.array([0.7, 0.0, 0.0]), types, box, mesh, 5, s_in=0.8,
                       kind="stated")
    assert np.allclose(Xs2, Xs, rtol=0, atol=1e-12)


def test_cell_offset_features():
    box, mesh = np.array([8.0, 10.0, 12.0]), (8, 5, 6)   # h = 1, 2, 2
    phi = np.zeros(mesh)
    # on a mesh point, a quarter, half and three quarters of a cell along x; y, z fixed
    pos = np.array([[3.0, 4.0, 6.0], [3.25, 5.0, 7.0], [3.5, 4.5, 6.5], [-0.25, 4.0, 6.0]])
    X = mlp.features(phi, pos, np.zeros(4, np.int8), box, mesh, 5)
    sx, cx = X[:, 30], X[:, 31]
    assert np.allclose(sx, [0.0, 1.0, 0.0, -1.0], atol=1e-12)
    assert np.allclose(cx, [1.0, 0.0, -1.0, 0.0], atol=1e-12)
    assert np.allclose(X[:, 32:34], [[0, 1], [0, -1], [1, 0], [0, 1]], atol=1e-12)   # y: 0, 1/2, 1/4, 0 cells
    assert np.allclose(X[:, 34:36], [[0, 1], [0, -1], [1, 0], [0, 1]], atol=1e-12)   # z: 0, 1/2, 1/4, 0 cells
    # the offset terms are periodic in the cell: one mesh step leaves them unchanged
    X2 = mlp.features(phi, pos + np.array([1.0, 2.0, 2.0]), np.zeros(4, np.int8), box, mesh, 5)
    assert np.allclose(X2[:, 30:36], X[:, 30:36], atol=1e-12)


@pytest.mark.parametrize("kind", ["cell", "stated"])
def test_features_at_mesh_points_are_a_discrete_convolution(kind):
    rng = np.random.default_rng(5)
    box, mesh = np.array([8.0, 8.0, 8.0]), (8, 8, 8)
    phi = rng.normal(size=mesh)
    m = rng.integers(0, 8, size=(6, 3))
    pos = m * 1.0   # h = 1: the sites sit on mesh points
    X = mlp.features(phi, pos, np.zeros(6, np.int8), box, mesh, 5, kind=kind)
    w = {0: 115 / 192, 1: 19 / 96, -1: 19 / 96, 2: 1 / 384, -2: 1 / 384}
    for i in range(6):
        k = 0
        for a in (-1, 0, 1):
            for b in (-1, 0, 1):
                for c in (-1, 0, 1):
                    ref = 0.0
                    for jx, wx in w.items():
                        for jy, wy in w.items():
                            for jz, wz in w.items():
                                ref += wx * wy * wz * phi[(m[i, 0] + a + jx) % 8, (m[i, 1] + b + jy) % 8,
                                                          (m[i, 2] + c + jz) % 8]
                    assert abs(X[i, k] - ref) < 1e-12
                    k += 1


def test_features_match_whole_mesh_brute_force():
    # phi(r) = sum over every mesh point and periodic image of M_p(u - m) phi[m]
    rng = np.random.default_rng(6)
    box, mesh = np.array([6.0, 7.0, 5.0]), (6, 7, 5)
    phi = rng.normal(size=mesh)
    pos = rng.uniform(-2.0, 9.0, size=(5, 3))
    for p in (4, 5):
        X = mlp.features(phi, pos, np.ones(5, np.int8), box, mesh, p)
        h = box / np.array(mesh)
        offs = [(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)]
        for i in range(5):
            for k, d in enumerate(offs):
                u = (pos[i] + h * np.array(d)) / h
                ref = 0.0
                for mx in range(-2 * mesh[0], 3 * mesh[0]):
                    wx = bspline_M(p, np.array([u[0] - mx]))[0]
                    if wx == 0.0:
                        continue
                    for my in range(-2 * mesh[1], 3 * mesh[1]):
                        wy = bspline_M(p, np.array([u[1] - my]))[0]
                        if wy == 0.0:
                            continue
                        for mz in range(-2 * mesh[2], 3 * mesh[2]):
                            wz = bspline_M(p, np.array([u[2] - mz]))[0]
                            if wz != 0.0:
                                ref += wx * wy * wz * phi[mx % mesh[0], my % mesh[1], mz % mesh[2]]
                assert abs(X[i, k] - ref) < 1e-12, (p, i, k)


# ---------------------------------------------------------------- Adam
def test_adam_constant_gradient_closed_form():
    # with a constant gradient g the bias-corrected moments are exactly g and
    # g^2, so every step moves each parameter by lr * g / (|g| + eps)
    rng = np.random.default_rng(7)
    theta0 = rng.normal(size=50)
    g = rng.normal(size=50) * 10.0 ** rng.uniform(-3, 2, size=50)
    theta, m, v = theta0.copy(), np.zeros(50), np.zeros(50)
    for step in range(1, 21):
        theta, m, v = mlp.adam_step(theta, m, v, g, step, lr=1e-3)
    assert np.allclose(theta, theta0 - 20 * 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-12)


def test_adam_first_step_is_a_sign_step():
    g = np.array([3.0, -0.2, 1e-3, -50.0])
    theta, _, _ = mlp.adam_step(np.zeros(4), np.zeros(4), np.zeros(4), g, 1, lr=0.01)
    assert np.allclose(theta, -0.01 * np.sign(g), rtol=1e-5)


def test_bf16_activations_stay_within_rounding_bound():
    rng = np.random.default_rng(8)
    theta = init_mlp_params(9).astype(np.float64)
    X = rng.normal(size=(64, mlp.N_IN))
    y, _ = mlp.forward(theta, X)
    ya, (_, h1, h2, p) = mlp.forward(theta, X, act_bf16=True)
    assert np.array_equal(mlp.bf16_round(h1), h1) and np.array_equal(mlp.bf16_round(h2), h2)
    # each activation moves by at most 2^-9 relative; propagate through |W|
    W2, W3 = np.abs(p["W2"]), np.abs(p["W3"])
    bound = (W3 @ (W2 @ np.abs(h1).T * 2.0 ** -9 + np.abs(h2).T * 2.0 ** -9)).T
    assert np.all(np.abs(ya - y) <= bound + 1e-15)
    assert np.any(ya != y)
