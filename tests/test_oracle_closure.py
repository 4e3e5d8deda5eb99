"""Pins of the learned-closure oracle (oracle/closure.py) against what mathematics fixes:
orthonormality and completeness of the non-conserved Hermite basis under the D2Q16 quadrature,
exact conservation of the correction and of block averaging, moments of constructed states,
neighbourhood indexing on an index field, GELU identities and an independent integral, the
network gradient against central finite differences, a hand-wired network's closed form, and
bfloat16 rounding against known values and torch's conversion."""
import math

import numpy as np
import pytest

import oracle
from oracle import closure as cl


@pytest.fixture(scope="module")
def vs():
    return oracle.velocity_set("D2Q16")


def test_basis_is_orthonormal_and_orthogonal_to_invariants(vs):
    psi = cl.nonconserved_basis(vs)
    w = vs["w"]
    G = (psi * w) @ psi.T
    assert np.max(np.abs(G - np.eye(12))) < 1e-13
    inv = np.stack([np.ones(16), vs["cx"], vs["cy"], vs["cx"] ** 2 + vs["cy"] ** 2])
    assert np.max(np.abs((psi * w) @ inv.T)) < 1e-13


def test_basis_completes_the_invariants(vs):
    inv = np.stack([np.ones(16), vs["cx"], vs["cy"], vs["cx"] ** 2 + vs["cy"] ** 2])
    full = np.vstack([inv, cl.nonconserved_basis(vs)])
    assert np.linalg.matrix_rank(full, tol=1e-10) == 16


def test_hermite_polynomials_closed_forms():
    x = np.linspace(-3, 3, 13)
    assert np.allclose(cl.hermite_e(2, x), x ** 2 - 1, atol=1e-14)
    assert np.allclose(cl.hermite_e(3, x), x ** 3 - 3 * x, atol=1e-13)


def test_correction_adds_no_mass_momentum_energy(vs):
    rng = np.random.default_rng(5)
    o = rng.normal(size=(7, 5, 12))
    d = cl.correction(o, vs)  # [16, 7, 5]
    cx = vs["cx"].reshape(-1, 1, 1)
    cy = vs["cy"].reshape(-1, 1, 1)
    for m in (np.ones_like(cx), cx, cy, cx * cx + cy * cy):
        assert np.max(np.abs((d * m).sum(axis=0))) < 1e-13


def test_project_inverts_correction_and_is_least_squares(vs):
    rng = np.random.default_rng(6)
    o = rng.normal(size=(4, 3, 12))
    assert np.max(np.abs(cl.project(cl.correction(o, vs), vs) - o)) < 1e-13
    # normal equations: the residual R - correction(project(R)) has no component along any psi_k
    R = rng.normal(size=(16, 4, 3))
    r = R - cl.correction(cl.project(R, vs), vs)
    psi = cl.nonconserved_basis(vs)
    assert np.max(np.abs(np.tensordot(psi, r, axes=([1], [0])))) < 1e-13


def test_block_average_conserves_and_keeps_uniform_states(vs):
    rng = np.random.default_rng(7)
    f = rng.uniform(0.01, 0.1, size=(16, 12, 8))
    c = cl.block_average(f, 4)
    assert c.shape == (16, 3, 2)
    assert abs(c.sum() * 16 - f.sum()) < 1e-12
    assert abs(c[:, 1, 0].mean() - f[:, 4:8, 0:4].mean()) < 1e-15
    o = oracle.Oracle(4, 4, "D2Q16")
    feq = o.equilibrium(1.02, 0.03, -0.01, 0.98)
    uni = np.broadcast_to(feq.reshape(16, 1, 1), (16, 8, 8)).copy()
    assert np.max(np.abs(cl.block_average(uni, 4) - feq.reshape(16, 1, 1))) < 1e-16


def test_features_of_equilibrium_and_of_constructed_stresses(vs):
    o = oracle.Oracle(4, 4, "D2Q16")
    rho, ux, uy, T = 1.05, 0.04, -0.02, 1.1
    feq = o.equilibrium(rho, ux, uy, T).reshape(16, 1, 1)
    F = cl.cell_features(feq, vs)[:, 0, 0]
    assert np.allclose(F, [rho, ux, uy, T, 0.0, 0.0], atol=1e-14)
    # adding a w psi_k changes only the stress it stands for: <psi_xy, c_x c_y> = 1 and
    # <psi_diff, c_x^2 - c_y^2> = 2; the conserved moments stay
    psi = cl.nonconserved_basis(vs)
    a = 1e-3
    f1 = feq + a * (vs["w"] * psi[1]).reshape(16, 1, 1)
    F1 = cl.cell_features(f1, vs)[:, 0, 0]
    assert np.allclose(F1, [rho, ux, uy, T, a, 0.0], atol=1e-14)
    f0 = feq + a * (vs["w"] * psi[0]).reshape(16, 1, 1)
    F0 = cl.cell_features(f0, vs)[:, 0, 0]
    assert np.allclose(F0, [rho, ux, uy, T, 0.0, 2 * a], atol=1e-14)
    # third-order vectors touch no feature
    f3 = feq + a * (vs["w"] * psi[2:].sum(axis=0)).reshape(16, 1, 1)
    assert np.allclose(cl.cell_features(f3, vs)[:, 0, 0], F, atol=1e-14)


def test_neighbourhood_indexing_on_an_index_field():
    ny, nx = 5, 7
    feat = np.zeros((6, ny, nx))
    yy, xx = np.mgrid[0:ny, 0:nx]
    for q in range(6):
        feat[q] = 1000 * q + 10 * yy + xx
    X = cl.neighbourhood(feat)
    assert X.shape == (ny * nx, 54)
    for (y, x) in [(0, 0), (2, 3), (4, 6), (0, 6)]:
        row = X[y * nx + x]
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                k = (dy + 1) * 3 + dx + 1
                for q in range(6):
                    want = 1000 * q + 10 * ((y + dy) % ny) + (x + dx) % nx
                    assert row[k * 6 + q] == want
    mu = np.arange(6.0)
    isg = np.arange(1.0, 7.0)
    Xn = cl.neighbourhood(feat, mu, isg)
    assert np.allclose(Xn, (X - np.tile(mu, 9)) * np.tile(isg, 9))


def test_gelu_identities_and_integral():
    z = np.linspace(-6, 6, 61)
    g = cl.gelu(z)
    assert cl.gelu(0.0) == 0.0
    assert np.max(np.abs(g - cl.gelu(-z) - z)) < 1e-14  # Phi(z) + Phi(-z) = 1
    assert abs(cl.gelu_grad(0.0) - 0.5) < 1e-15
    assert abs(cl.gelu(8.0) - 8.0) < 1e-13 and abs(cl.gelu(-8.0)) < 1e-13
    # Phi by trapezoid integration of the normal density (independent of erf)
    for zz in (-1.7, -0.3, 0.4, 2.2):
        t = np.linspace(-12.0, zz, 200001)
        phi = np.exp(-0.5 * t * t) / math.sqrt(2 * math.pi)
        Phi = float(np.sum(0.5 * (phi[1:] + phi[:-1]) * np.diff(t)))
        assert abs(cl.gelu(zz) - zz * Phi) < 1e-9
    # derivative against a central difference
    h = 1e-6
    for zz in (-2.0, -0.5, 0.7, 1.9):
        fd = (cl.gelu(zz + h) - cl.gelu(zz - h)) / (2 * h)
        assert abs(cl.gelu_grad(zz) - fd) < 1e-9


def test_gradient_matches_central_finite_differences():
    rng = np.random.default_rng(8)
    p = cl.init_params(3, scale=1.5)
    X = rng.normal(size=(7, 54))
    Ys = rng.normal(size=(7, 12)) * 0.3
    L, g = cl.loss_and_grad(p, X, Ys)
    theta = cl.pack(p)
    gflat = cl.pack(g)
    idx = rng.choice(theta.size, size=60, replace=False)
    h = 1e-5
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        Lp = cl.loss(cl.forward(cl.unpack(tp), X)[0], Ys)
        Lm = cl.loss(cl.forward(cl.unpack(tm), X)[0], Ys)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-8 + 1e-6 * abs(fd)


def test_hand_wired_network_closed_form():
    p = {name: np.zeros(shape) for name, shape in cl.PARAM_SHAPES}
    p["W1"][0, 5] = 2.0      # z1_0 = 2 x_5 + 0.1
    p["b1"][0] = 0.1
    p["W2"][3, 0] = -1.5     # z2_3 = -1.5 g(z1_0) + 0.2
    p["b2"][3] = 0.2
    p["W3"][7, 3] = 0.5      # y_7 = 0.5 g(z2_3) - 0.05, other outputs b3
    p["b3"][:] = -0.05
    x = np.zeros((1, 54))
    x[0, 5] = 0.8
    Y, _ = cl.forward(p, x)

    def g(z):
        return 0.5 * z * (1 + math.erf(z / math.sqrt(2)))
    want = 0.5 * g(-1.5 * g(2 * 0.8 + 0.1) + 0.2) - 0.05
    assert abs(Y[0, 7] - want) < 1e-15
    assert np.all(np.delete(Y[0], 7) == -0.05)


def test_bf16_rounding_known_values_and_torch():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 1.0 + 2 ** -7, -2.5, 3.0e-3, 65504.0, 0.0])
    want = np.array([1.0, 1.0, 1.0 + 2 ** -7, 1.0 + 2 ** -7, -2.5, None, 65536.0, 0.0], dtype=object)
    got = cl.bf16_round(vals)
    for g, w in zip(got, want):
        if w is not None:
            assert g == w
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(9)
    a = rng.normal(size=4096) * np.exp(rng.uniform(-20, 20, size=4096))
    ref = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cl.bf16_round(a), ref)


def test_closure_step_conserves_mass_momentum_energy():
    import workloads
    nx = ny = 12
    o = oracle.Oracle(nx, ny, "D2Q16", tau=0.6)
    o.init_moments(*workloads.random_smooth(nx, ny, seed=4, amp_u=0.05, amp_T=0.03))
    p = cl.init_params(11, scale=2.0)
    s0 = o.conserved_sums()
    coeffs = cl.closure_step(o, p, np.zeros(6), np.full(6, 10.0), np.full(12, 1e-3))
    assert np.max(np.abs(coeffs)) > 1e-5  # the correction is not trivially zero
    s1 = o.conserved_sums()
    assert np.max(np.abs(s1 - s0)) < 1e-12 * max(1.0, abs(s0[0]))


def test_noneq_coefficients_of_constructed_states(vs):
    nx, ny = 3, 2
    o = oracle.Oracle(nx, ny, "D2Q16")
    rng = np.random.default_rng(12)
    f = np.zeros((16, ny, nx))
    for y in range(ny):
        for x in range(nx):
            f[:, y, x] = o.equilibrium(1 + 0.05 * rng.normal(), 0.05 * rng.normal(), 0.05 * rng.normal(),
                                       1 + 0.05 * rng.normal())
    assert np.max(np.abs(cl.noneq_coefficients(o, f))) < 1e-15
    a = rng.normal(size=(ny, nx, 12)) * 1e-3
    g = f + cl.correction(a, vs)
    assert np.max(np.abs(cl.noneq_coefficients(o, g) - a.reshape(-1, 12))) < 1e-15


def test_closure_step_with_zero_network_is_bgk_with_unit_relaxation():
    """All-zero network output: the learned step reduces to stream + BGK with dt / tau = 1."""
    import workloads
    nx, ny = 10, 6
    fields = workloads.random_smooth(nx, ny, seed=13, amp_u=0.05, amp_T=0.03)
    a = oracle.Oracle(nx, ny, "D2Q16", tau=0.7)
    a.init_moments(*fields)
    b = oracle.Oracle(nx, ny, "D2Q16", tau=1.0)
    b.set_populations(a.f)
    p = {name: np.zeros(shape) for name, shape in cl.PARAM_SHAPES}
    cl.closure_step(a, p, np.zeros(6), np.ones(6), np.ones(12))
    b.run(1)
    assert np.max(np.abs(a.f - b.f)) < 1e-15


def test_bf16_storage_option_rounds_inputs_and_hidden_layers_only():
    """closure_coefficients(bf16=True): a network whose inputs and hidden activations are already
    BF16 values is unchanged by the option; otherwise it differs from the FP64 network by BF16
    rounding only (a few 2^-8 of the output scale); and the all-zero network gives its output
    bias exactly either way."""
    import workloads
    nx = ny = 8
    o = oracle.Oracle(nx, ny, "D2Q16", tau=0.6)
    o.init_moments(*workloads.random_smooth(nx, ny, seed=5, amp_u=0.05, amp_T=0.03))
    mu, isg, scale = np.zeros(6), np.full(6, 10.0), np.full(12, 1e-3)
    p = cl.init_params(14, scale=1.5)
    a = cl.closure_coefficients(o, p, mu, isg, scale)
    b = cl.closure_coefficients(o, p, mu, isg, scale, bf16=True)
    assert 0 < np.max(np.abs(a - b)) <= 3e-2 * np.max(np.abs(a))
    # zero first and second layers with BF16-exact biases whose GELU is BF16-exact (0): only
    # the rounding of the inputs could act, and W1 = 0 removes it
    z = {name: np.zeros(shape) for name, shape in cl.PARAM_SHAPES}
    z["b3"] = np.linspace(-1.0, 1.0, 12)
    for flag in (False, True):
        assert np.array_equal(cl.closure_coefficients(o, z, mu, isg, scale, bf16=flag),
                              np.broadcast_to(z["b3"] * scale, (nx * ny, 12)))
