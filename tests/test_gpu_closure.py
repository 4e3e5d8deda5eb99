"""GPU parity of the learned-closure path against the FP64 oracle (oracle/closure.py).

Network (tcgen05 BF16 kernels, FP32 accumulation): the forward pass is compared with the
oracle's FP64 network evaluated on the same BF16-rounded inputs and weights with its hidden
activations rounded to BF16 as the kernels store them (tolerance: a few BF16 units of the
output scale, for activations whose rounding falls on the other side); gradients are compared
with the oracle's FP64 chain rule on the same BF16-rounded operands (relative norm error, the
kernels keeping BF16 activations and BF16 back-propagated signals).  Closure kernels (features,
projection, block average, corrected coarse step) are compared element by element on FP64
storage."""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import closure as cl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1004_5059_gb300 as tv
    return tv


def bf16_params(p):
    return {k: cl.bf16_round(v) if k.startswith("W") else np.asarray(v, dtype=np.float32).astype(np.float64)
            for k, v in p.items()}


def forward_bf16_hidden(p, X):
    """The oracle network with hidden activations rounded to BF16 (the kernels' storage)."""
    H1 = cl.bf16_round(cl.gelu(X @ p["W1"].T + p["b1"]))
    H2 = cl.bf16_round(cl.gelu(H1 @ p["W2"].T + p["b2"]))
    return H2 @ p["W3"].T + p["b3"]


def random_inputs(rows, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    X = np.zeros((rows, 64))
    X[:, :54] = rng.normal(size=(rows, 54)) * scale
    return cl.bf16_round(X)


def to_dev_bf16(X):
    import torch
    return torch.from_numpy(X.astype(np.float32)).to(torch.bfloat16).cuda().contiguous()


@pytest.mark.parametrize("rows", [128, 384, 4096])
def test_forward_matches_oracle(tv, rows):
    import torch
    p = cl.init_params(21, scale=1.5)
    m = tv.Mlp(4096)
    m.set_params(cl.pack(p).astype(np.float32))
    X = random_inputs(rows, 22)
    y = torch.zeros((rows, 16), dtype=torch.float32, device="cuda")
    m.forward(to_dev_bf16(X), y)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.float64)
    pr = bf16_params(p)
    want = forward_bf16_hidden(pr, X[:, :54])
    scale = np.max(np.abs(want))
    assert np.max(np.abs(got[:, :12] - want)) <= 4e-3 * scale
    assert np.all(got[:, 12:] == 0.0)
    # the plain FP64 network (no BF16 activations) is close too
    want64, _ = cl.forward(pr, X[:, :54])
    assert np.max(np.abs(got[:, :12] - want64)) <= 3e-2 * np.max(np.abs(want64))
    m.close()


def test_params_round_trip(tv):
    p = cl.init_params(23)
    m = tv.Mlp(128)
    theta = cl.pack(p).astype(np.float32)
    m.set_params(theta)
    assert np.array_equal(m.get_params(), theta)
    m.close()


@pytest.mark.parametrize("rows", [256, 8192])
def test_loss_and_gradient_match_oracle(tv, rows):
    import torch
    p = cl.init_params(24, scale=1.5)
    m = tv.Mlp(8192)
    m.set_params(cl.pack(p).astype(np.float32))
    X = random_inputs(rows, 25)
    rng = np.random.default_rng(26)
    Ys = np.zeros((rows, 16))
    Ys[:, :12] = rng.normal(size=(rows, 12)) * 0.5
    ys_dev = torch.from_numpy(Ys.astype(np.float32)).cuda()
    loss, grad = m.loss_grad(to_dev_bf16(X), ys_dev, want_loss=True, want_grad=True)
    pr = bf16_params(p)
    L, g = cl.loss_and_grad(pr, X[:, :54], Ys[:, :12].astype(np.float32).astype(np.float64))
    assert abs(loss - L) <= 1e-2 * L
    gref = cl.pack(g)
    gg = grad.astype(np.float64)
    for name, shape in cl.PARAM_SHAPES:
        a = cl.unpack(gg)[name].ravel()
        b = cl.unpack(gref)[name].ravel()
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        assert rel < 3e-2, (name, rel)
        assert cos > 0.999, (name, cos)
    m.close()


def test_adam_training_fits_a_teacher(tv):
    """200 Adam steps on data from a random teacher network cut the loss at least tenfold."""
    import torch
    rows = 4096
    teacher = cl.init_params(30, scale=1.0)
    X = random_inputs(rows, 31)
    Y = np.zeros((rows, 16))
    Y[:, :12] = cl.forward(teacher, X[:, :54])[0]
    m = tv.Mlp(rows)
    m.set_params(cl.pack(cl.init_params(32, scale=0.5)).astype(np.float32))
    xd, yd = to_dev_bf16(X), torch.from_numpy(Y.astype(np.float32)).cuda()
    l0, _ = m.loss_grad(xd, yd)
    for _ in range(200):
        m.loss_grad(xd, yd, want_loss=False)
        m.adam(3e-3)
    l1, _ = m.loss_grad(xd, yd)
    assert l1 < 0.1 * l0, (l0, l1)
    m.close()


def test_mlp_rejects_bad_rows(tv):
    import torch
    m = tv.Mlp(256)
    x = torch.zeros((100, 64), dtype=torch.bfloat16, device="cuda")
    y = torch.zeros((100, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(tv.TvlbmError):
        m.forward(x, y)
    x = torch.zeros((384, 64), dtype=torch.bfloat16, device="cuda")
    y = torch.zeros((384, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(tv.TvlbmError):
        m.forward(x, y)
    m.close()


# ---------------------------------------------------------------------------------------------
# closure kernels on FP64 storage
# ---------------------------------------------------------------------------------------------

def make_pair(tv, nx, ny, seed, tau=0.6):
    fields = workloads.random_smooth(nx, ny, seed=seed, amp_u=0.05, amp_T=0.03)
    sim = tv.Simulation(nx, ny, "D2Q16", tau=tau, storage="fp64")
    sim.init_moments(*fields)
    o = oracle.Oracle(nx, ny, "D2Q16", tau=tau)
    o.init_moments(*fields)
    return sim, o


def test_moments_and_features_match_oracle(tv):
    import torch
    nx, ny = 48, 32
    sim, o = make_pair(tv, nx, ny, 40)
    sim.step(3)
    o.run(3)
    m6 = torch.zeros((6, ny, nx), dtype=torch.float32, device="cuda")
    tv.closure_moments(sim, m6)
    want = cl.cell_features(o.f)
    got = m6.cpu().numpy().astype(np.float64)
    for q in range(6):
        assert np.max(np.abs(got[q] - want[q])) <= 1e-6 * max(np.max(np.abs(want[q])), 1e-3), q
    mu = np.array([1.0, 0.0, 0.0, 1.0, 0.0, 0.0])
    isg = np.array([30.0, 20.0, 20.0, 30.0, 500.0, 500.0])
    x = torch.zeros((nx * ny, 64), dtype=torch.bfloat16, device="cuda")
    tv.closure_features(sim, mu, isg, x)
    gx = x.float().cpu().numpy().astype(np.float64)
    wx = cl.neighbourhood(want, mu, isg)
    # one BF16 unit (2^-8 relative) where FP32 and FP64 evaluation round to neighbours
    assert np.all(np.abs(gx[:, :54] - cl.bf16_round(wx)) <= 2.0 ** -7 * np.abs(wx) + 1e-6)
    assert np.all(gx[:, 54:] == 0.0)
    sim.close()


def test_project_matches_oracle(tv):
    import torch
    nx, ny = 32, 24
    a, oa = make_pair(tv, nx, ny, 41)
    b, ob = make_pair(tv, nx, ny, 42)
    o = torch.zeros((nx * ny, 16), dtype=torch.float32, device="cuda")
    tv.closure_project(a, b, o)
    got = o.cpu().numpy().astype(np.float64)
    want = cl.project(oa.f - ob.f).reshape(nx * ny, 12)
    assert np.max(np.abs(got[:, :12] - want)) <= 1e-6 * np.max(np.abs(want))
    assert np.all(got[:, 12:] == 0.0)
    a.close()
    b.close()


@pytest.mark.parametrize("fine_storage,coarse_storage", [("fp64", "fp64"), ("fp32_dev", "fp32_dev"), ("fp32", "fp64")])
def test_downsample_matches_block_average(tv, fine_storage, coarse_storage):
    nx, ny, mfac = 64, 48, 4
    fields = workloads.random_smooth(nx, ny, seed=43, amp_u=0.05, amp_T=0.03)
    fine = tv.Simulation(nx, ny, "D2Q16", storage=fine_storage)
    fine.init_moments(*fields)
    fine.step(5)
    coarse = tv.Simulation(nx // mfac, ny // mfac, "D2Q16", storage=coarse_storage)
    tv.downsample(fine, coarse)
    f = fine.populations_f64()
    want = cl.block_average(f, mfac)
    got = coarse.populations_f64()
    tol = 1e-14 if coarse_storage == "fp64" else 1e-7
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))
    sf, sc = fine.conserved_sums(), coarse.conserved_sums()
    for k in range(4):
        assert abs(sc[k] * mfac * mfac - sf[k]) <= (1e-12 if coarse_storage == "fp64" else 1e-6) * max(1.0, abs(sf[0]))
    # the coarse state steps like any other (frame images were written)
    coarse.step(2)
    assert np.all(np.isfinite(coarse.populations_f64()))
    fine.close()
    coarse.close()


def test_copy_state(tv):
    nx, ny = 32, 32
    a, _ = make_pair(tv, nx, ny, 44)
    a.step(3)
    b = tv.Simulation(nx, ny, "D2Q16", tau=0.6, storage="fp64")
    tv.copy_state(a, b)
    assert np.array_equal(a.raw_populations(), b.raw_populations())
    a.step(4)
    b.step(4)
    assert np.array_equal(a.raw_populations(), b.raw_populations())
    a.close()
    b.close()


def test_noneq_matches_oracle(tv):
    import torch
    nx, ny = 24, 16
    sim, o = make_pair(tv, nx, ny, 49)
    sim.step(4)
    o.run(4)
    out = torch.zeros((nx * ny, 16), dtype=torch.float32, device="cuda")
    isc = np.linspace(0.5, 2.0, 12)
    tv.closure_noneq(sim, out, isc)
    got = out.cpu().numpy().astype(np.float64)
    want = cl.noneq_coefficients(o) * isc
    assert np.max(np.abs(got[:, :12] - want)) <= 1e-6 * np.max(np.abs(want))
    assert np.all(got[:, 12:] == 0.0)
    sim.close()


def test_closure_step_matches_oracle_and_conserves(tv):
    """Three learned coarse steps, FP64 storage: populations against the oracle's closure_step
    on the same (BF16-rounded) network; conserved sums exact to rounding."""
    nx, ny = 32, 16
    sim, o = make_pair(tv, nx, ny, 45, tau=0.55)
    p = bf16_params(cl.init_params(46, scale=1.5))
    mu = np.array([1.0, 0.0, 0.0, 1.0, 0.0, 0.0])
    isg = np.array([30.0, 20.0, 20.0, 30.0, 500.0, 500.0])
    scale = np.full(12, 2e-4)
    m = tv.Mlp(nx * ny)
    m.set_params(cl.pack(p).astype(np.float32))
    o64 = oracle.Oracle(nx, ny, "D2Q16", tau=0.55)
    o64.f[...] = o.f
    s0 = sim.conserved_sums()
    coeffs = []
    for _ in range(3):
        coeffs.append(cl.closure_step(o, p, mu, isg, scale, bf16=True))
        cl.closure_step(o64, p, mu, isg, scale)
        tv.step_closure(sim, m, mu, isg, scale, 1)
    got = sim.populations_f64()
    corr_max = max(np.max(np.abs(c)) for c in coeffs)
    assert corr_max > 1e-6
    # against the oracle with BF16 inputs and activations: per step the network's FP32
    # accumulation (an occasional BF16 activation rounded the other way) <= 4e-3 of the
    # coefficient scale, times max_l w_l sum_k |psi_k(c_l)| (< 1.5 for D2Q16), over 3 steps
    assert np.max(np.abs(got - o.f)) <= 3 * 4e-3 * corr_max * 1.5
    # and against the all-FP64 network: the BF16 storage itself, <= 3e-2 of the scale per step
    assert np.max(np.abs(got - o64.f)) <= 3 * 3e-2 * corr_max * 1.5
    s1 = sim.conserved_sums()
    for k in range(4):
        assert abs(s1[k] - s0[k]) <= 1e-12 * max(1.0, abs(s0[0]))
    m.close()
    sim.close()


def test_closure_step_fp32_conserves_to_storage_rounding(tv):
    nx, ny = 64, 32
    fields = workloads.random_smooth(nx, ny, seed=47, amp_u=0.05, amp_T=0.03)
    sim = tv.Simulation(nx, ny, "D2Q16", tau=0.55, storage="fp32_dev")
    sim.init_moments(*fields)
    p = bf16_params(cl.init_params(48, scale=1.5))
    m = tv.Mlp(nx * ny)
    m.set_params(cl.pack(p).astype(np.float32))
    mu = np.array([1.0, 0.0, 0.0, 1.0, 0.0, 0.0])
    isg = np.array([30.0, 20.0, 20.0, 30.0, 500.0, 500.0])
    s0 = sim.conserved_sums()
    tv.step_closure(sim, m, mu, isg, np.full(12, 2e-4), 20)
    s1 = sim.conserved_sums()
    assert s1[4] == 0
    for k in range(4):
        assert abs(s1[k] - s0[k]) <= 2e-8 * abs(s0[0]), k
    m.close()
    sim.close()


def test_closure_graphs_equal_direct_launches(tv):
    """Learned steps replayed through the captured graphs (two steps each) equal direct launches
    bit for bit, for even and odd step counts, and follow a change of the output scale."""
    nx, ny = 64, 32
    fields = workloads.random_smooth(nx, ny, seed=50, amp_u=0.05, amp_T=0.03)
    p = bf16_params(cl.init_params(51, scale=1.5))
    m = tv.Mlp(nx * ny)
    m.set_params(cl.pack(p).astype(np.float32))
    mu = np.array([1.0, 0.0, 0.0, 1.0, 0.0, 0.0])
    isg = np.array([30.0, 20.0, 20.0, 30.0, 500.0, 500.0])
    sims = []
    for graphs in (True, False):
        s_ = tv.Simulation(nx, ny, "D2Q16", tau=0.55, storage="fp32_dev", graphs=graphs)
        s_.init_moments(*fields)
        tv.step_closure(s_, m, mu, isg, np.full(12, 2e-4), 7)
        tv.step_closure(s_, m, mu, isg, np.full(12, 1e-4), 6)
        sims.append(s_)
    assert np.array_equal(sims[0].raw_populations(), sims[1].raw_populations())
    for s_ in sims:
        s_.close()
    m.close()


def test_closure_rejects_unsupported_contexts(tv):
    m = tv.Mlp(1024)
    mu, isg, sc = np.zeros(6), np.ones(6), np.ones(12)
    for kw in [dict(velset="D2Q9"), dict(storage="fp16_dev"), dict(walls=(0.0, 1.0, 0.0, 1.0))]:
        args = dict(velset="D2Q16", storage="fp32")
        args.update(kw)
        s = tv.Simulation(32, 32, args.pop("velset"), **args)
        with pytest.raises(tv.TvlbmError):
            tv.step_closure(s, m, mu, isg, sc, 1)
        s.close()
    s = tv.Simulation(64, 32, "D2Q16", storage="fp32")  # 2048 cells > max_rows
    with pytest.raises(tv.TvlbmError):
        tv.step_closure(s, m, mu, isg, sc, 1)
    s.close()
    m.close()


def test_activation_within_its_error_bound(tv):
    """The kernels' GELU (erf by Abramowitz & Stegun eq. 7.1.26, |error| <= 1.5e-7) and its
    derivative on a dense grid: against the exact function in FP64 and against CUDA's own erff
    (torch.erf), within the approximation's bound plus FP32 rounding."""
    import torch
    from scipy.special import erf
    z = torch.linspace(-12.0, 12.0, 240001, dtype=torch.float32, device="cuda")
    g, dg = tv.mlp_activation(z)
    torch.cuda.synchronize()
    zz = z.cpu().numpy().astype(np.float64)
    phi_cdf = 0.5 * (1.0 + erf(zz / math.sqrt(2.0)))
    phi_pdf = np.exp(-0.5 * zz * zz) / math.sqrt(2.0 * math.pi)
    gg, dd = g.cpu().numpy().astype(np.float64), dg.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(gg - zz * phi_cdf) <= 3e-7 * (np.abs(zz) + 1.0))
    assert np.all(np.abs(dd - (phi_cdf + zz * phi_pdf)) <= 1e-6)
    cuda = (0.5 * z * (1.0 + torch.erf(z * 0.70710678118654752))).cpu().numpy().astype(np.float64)
    assert np.all(np.abs(gg - cuda) <= 3e-7 * (np.abs(zz) + 1.0))
    assert tv.lib.tvlbm_mlp_activation(None, None, None, 4, None) == tv.TVLBM_EINVAL
    assert tv.lib.tvlbm_mlp_activation(z.data_ptr(), None, None, -1, None) == tv.TVLBM_EINVAL
