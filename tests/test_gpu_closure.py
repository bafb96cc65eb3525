"""Learned closure (S12/S13) on the GPU through the C ABI, against the oracle.

The network runs in BF16 with FP32 accumulation on the tensor cores; the
oracle rounds weights and activations to BF16 the same way but accumulates in
FP64, so outputs and gradients are compared within 1e-2 relative (a BF16
activation that rounds the other way moves an output by about 2^-9 of its
scale).  Inputs, targets and the coupling fields are FP64 arithmetic on both
sides and are compared within FP32 / FP64 tolerances.
"""
import numpy as np
import pytest

from oracle import orc
from paper_2607_08195_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_08195_gb300 import dig  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def solver():
    s = W.config_small(seed=41)
    g = dig.Solver(s, DEV)
    yield g
    g.close()


def random_net(seed, bias=0.05, scale=1.0):
    rng = np.random.default_rng(seed)
    p = orc.mlp_init(seed) * np.float32(scale)
    p += (bias * rng.standard_normal(len(p))).astype(np.float32)
    return p


# --------------------------------------------------------------------------
# Element-wise tolerances of the BF16 network (13 -> 64 -> 64 -> 64 -> 8)
# from a propagation of the rounding differences between the CUDA kernels
# (BF16 weights, activations and deltas on the tensor cores, FP32
# accumulation, FP32 erf/exp) and the oracle (the same BF16 weights and
# activations, FP64 accumulation, FP64 deltas).  The differences are
# independent roundings, so they are propagated in quadrature, each taken
# with an RMS equal to its full size (about 3.5 times the RMS of a uniform
# rounding error): an FP32 sum of n terms errs by n 2^-24 times the sum of
# their magnitudes; an activation rounded to BF16 from slightly different
# values differs by one BF16 unit u (2^-7 of its magnitude) when the two
# values straddle a rounding boundary, which happens with probability
# |dg| / u for a difference dg < u (mean square u |dg|, at most u^2); a
# delta rounded to BF16 by half a unit (2^-8); GELU passes an input
# difference on with |GELU'| and adds 1e-6 for FP32 erf.  The tolerance of
# an element is 6 of these standard deviations.
# --------------------------------------------------------------------------
U32, ULP_BF, HALF_BF = 2.0 ** -24, 2.0 ** -7, 2.0 ** -8
SHAPES = ((13, 64), (64, 64), (64, 64), (64, 8))
NSIG = 6.0


def bf16_np(x):
    """Round to BF16, nearest even (the rule pinned in the oracle tests)."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def net_layers(p):
    out, off = [], 0
    for nin, nout in SHAPES:
        W = bf16_np(p[off:off + nin * nout]).reshape(nout, nin)
        off += nin * nout
        out.append((W, p[off:off + nout].astype(np.float64)))
        off += nout
    return out


def gelu_np(z):
    from scipy.special import erf

    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_d_np(z):
    from scipy.special import erf

    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def forward_sd(p, X):
    """Standard deviation of the GPU - oracle difference of every output
    [n, 8], with the activations, their variances and the pre-activations
    (and their variances) for the backward pass."""
    L = net_layers(p)
    a = bf16_np(X)
    v = np.zeros_like(a)
    acts, var, zs = [a], [v], []
    for l, (W, b) in enumerate(L):
        z = a @ W.T + b
        vz = v @ (W ** 2).T + ((W.shape[1] + 1) * U32 * (np.abs(a) @ np.abs(W).T + np.abs(b))) ** 2
        zs.append((z, vz))
        if l < 3:
            g = gelu_np(z)
            a = bf16_np(g)
            vg = gelu_d_np(z) ** 2 * vz + (1e-6 * np.abs(g)) ** 2  # of the value before rounding
            ulp = ULP_BF * np.abs(a)
            # rounding flips: one unit, where the two values straddle a rounding boundary
            v = vg + np.minimum(ulp ** 2, ulp * np.sqrt(vg))
            acts.append(a)
            var.append(v)
    return np.sqrt(zs[-1][1]), acts, var, zs


def gradient_sd(p, X, T):
    """Standard deviation of the GPU - oracle difference of every component
    of the gradient of the mean-square loss (layout of the parameters)."""
    L = net_layers(p)
    sy, acts, var, zs = forward_sd(p, X)
    y = zs[-1][0]
    n = len(X)
    d = 2.0 * (y - T) / (8 * n)
    vd = (2.0 * sy / (8 * n)) ** 2 + (HALF_BF * d) ** 2
    out = [None] * 4
    for l in range(3, -1, -1):
        a, va = acts[l], var[l]
        vW = vd.T @ a ** 2 + (d ** 2).T @ va + ((n + 1) * U32 * (np.abs(d).T @ np.abs(a))) ** 2
        vb = vd.sum(axis=0) + ((n + 1) * U32 * np.abs(d).sum(axis=0)) ** 2
        out[l] = (vW, vb)
        if l == 0:
            break
        W = L[l][0]
        z, vz = zs[l - 1]
        gd = gelu_d_np(z)
        s = d @ W
        vs = vd @ W ** 2 + (W.shape[0] * U32 * (np.abs(d) @ np.abs(W))) ** 2
        dn = s * gd
        vd = vs * gd ** 2 + s ** 2 * (0.8 ** 2 * vz + 1e-12) + (HALF_BF * dn) ** 2
        d = dn
    return np.sqrt(np.concatenate([np.concatenate([w.ravel(), b]) for w, b in out]))


def test_init_is_bit_exact(solver):
    """He-normal initialisation from the MLP_INIT stream: identical parameters."""
    for seed in (3, 2 ** 40 + 7):
        solver.closure_init(seed)
        assert np.array_equal(solver.closure_get(), orc.mlp_init(seed))


@pytest.mark.parametrize("n", [1, 64, 1000, 4096 + 37, 200_003])
def test_forward_parity(solver, n):
    """Forward pass (the tcgen05 inference kernel) on rows spanning several
    128-row tiles and a ragged tail; 200,003 rows give every CTA of the
    persistent grid several tiles."""
    p = random_net(n)
    solver.closure_set(p)
    rng = np.random.default_rng(n + 1)
    X = rng.standard_normal((n, 13)).astype(np.float32)
    Yg = solver.closure_forward(torch.from_numpy(X).to(DEV)).cpu().numpy().astype(np.float64)
    Yo = orc.mlp_forward(p, X, bf16=True)
    tol = NSIG * forward_sd(p, X)[0] + 1e-7
    assert np.all(np.abs(Yg - Yo) <= tol), np.max(np.abs(Yg - Yo) / tol)
    # the tolerance is not vacuous: a few per cent of an output
    assert np.median(tol / (np.abs(Yo) + 1e-3)) < 0.05
    # the FP64 network without BF16 is farther away than the BF16 oracle
    Y64 = orc.mlp_forward(p, X, bf16=False)
    assert np.abs(Yg - Yo).mean() < np.abs(Yg - Y64).mean()


def test_forward_wait_gives_up_and_context_survives(solver):
    """Failure detection of the tensor-core forward without a GPU fault: with
    its MMAs withheld the first mbarrier wait runs out after about a second,
    the kernel frees its tensor memory and returns, and the library reports
    DIG_ERR_TIMEOUT; a normal forward on the same context then still matches
    the oracle."""
    import time

    p = random_net(5)
    solver.closure_set(p)
    t0 = time.time()
    assert solver.test_forward_timeout() == -8  # DIG_ERR_TIMEOUT
    assert 0.5 < time.time() - t0 < 30.0
    rng = np.random.default_rng(9)
    X = rng.standard_normal((300, 13)).astype(np.float32)
    Yg = solver.closure_forward(torch.from_numpy(X).to(DEV)).cpu().numpy().astype(np.float64)
    Yo = orc.mlp_forward(p, X, bf16=True)
    tol = NSIG * forward_sd(p, X)[0] + 1e-7
    assert np.all(np.abs(Yg - Yo) <= tol)


@pytest.mark.parametrize("n", [777, 45_001])
def test_gradient_parity(solver, n):
    """Backward pass: every component of the gradient of the mean-square loss
    within its element-wise tolerance, the loss within 1e-3.  777 rows are
    seven 128-row tiles, one per CTA; 45,001 rows give every CTA of the
    one-per-SM grid two or three tiles, whose weight gradients accumulate in
    tensor memory before they are added to the global gradient."""
    p = random_net(9)
    solver.closure_set(p)
    rng = np.random.default_rng(10)
    X = rng.standard_normal((n, 13)).astype(np.float32)
    T = (0.5 * rng.standard_normal((n, 8))).astype(np.float32)
    lg, gg = solver.closure_grad(torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV))
    lo, go = orc.mlp_grad(p, X, T, bf16=True)
    assert abs(lg - lo) <= 1e-3 * lo
    tol = NSIG * gradient_sd(p, X, T.astype(np.float64)) + 1e-12
    assert len(tol) == dig.MLP_NPARAM
    diff = np.abs(gg.astype(np.float64) - go)
    assert np.all(diff <= tol), (np.argmax(diff / tol), np.max(diff / tol))
    assert np.median(tol / (np.abs(go) + 1e-12)) < 0.2
    # the gradient buffer is cleared afterwards: a second call gives the same
    lg2, gg2 = solver.closure_grad(torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV))
    assert np.array_equal(gg, gg2) or np.abs(gg - gg2).max() <= 1e-6 * np.abs(gg).max()


def test_adam_training_follows_oracle(solver):
    """Five Adam steps on mini-batches in a given row order: the per-epoch loss
    and the parameters track the oracle (FP64 Adam on its own gradients)."""
    p = random_net(12, scale=0.5)
    rng = np.random.default_rng(13)
    n, batch = 640, 128
    X = rng.standard_normal((n, 13)).astype(np.float32)
    T = (0.3 * rng.standard_normal((n, 8))).astype(np.float32)
    perm = rng.permutation(n).astype(np.int32)
    solver.closure_set(p)
    lr = 1e-3
    loss = solver.closure_train(torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV), epochs=1, batch=batch,
                                lr=lr, perm=torch.from_numpy(perm[None, :]).to(DEV))
    q = p.copy()
    m = np.zeros(len(q))
    v = np.zeros(len(q))
    sse = 0.0
    for k, b0 in enumerate(range(0, n, batch)):
        rows = perm[b0:b0 + batch]
        l, g = orc.mlp_grad(q, X[rows], T[rows], bf16=True)
        sse += l * len(rows)
        orc.adam(q, m, v, g, k + 1, lr=lr)
    assert abs(loss[0] - sse / n) <= 2e-3 * (sse / n)
    pg = solver.closure_get()
    step = np.abs(q.astype(np.float64) - p)
    diff = np.abs(pg.astype(np.float64) - q)
    # Adam moves each parameter by about lr per step; BF16 noise in tiny
    # gradients can change the direction of a few of them
    assert np.mean(diff <= 0.1 * 5 * lr) > 0.97, np.mean(diff <= 0.1 * 5 * lr)
    assert np.median(step) > 0.5 * lr


def test_adam_first_step_elementwise(solver):
    """One Adam step, element by element: the first step moves a parameter by
    lr g/(|g| + eps); where the oracle's gradient exceeds its element-wise
    BF16 tolerance the direction is certain and the GPU's step equals the
    oracle's within 1e-3 lr (|g| is then well above eps), elsewhere it may
    differ by up to 2 lr."""
    p = random_net(14, scale=0.5)
    rng = np.random.default_rng(15)
    n = 256
    X = rng.standard_normal((n, 13)).astype(np.float32)
    T = (0.3 * rng.standard_normal((n, 8))).astype(np.float32)
    solver.closure_set(p)
    lr = 1e-3
    solver.closure_train(torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV), epochs=1, batch=n, lr=lr,
                         perm=torch.arange(n, dtype=torch.int32, device=DEV)[None, :].clone())
    pg = solver.closure_get().astype(np.float64)
    _, go = orc.mlp_grad(p, X, T, bf16=True)
    q = p.copy()
    orc.adam(q, np.zeros(len(q)), np.zeros(len(q)), go, 1, lr=lr)
    tol = NSIG * gradient_sd(p, X, T.astype(np.float64))
    sure = np.abs(go) > tol + 1e-6
    d = np.abs(pg - q.astype(np.float64))
    assert sure.mean() > 0.5
    assert np.all(d[sure] <= 1e-3 * lr + 1e-7 * np.abs(p[sure])), np.max(d[sure])
    assert np.all(d <= 2.0 * lr + 1e-7 * np.abs(p))


def test_train_rejects_bad_perm(solver):
    """A perm entry outside [0, n) is caught on the device: DIG_ERR_ARG."""
    solver.closure_init(1)
    X = torch.zeros((100, 13), device=DEV)
    T = torch.zeros((100, 8), device=DEV)
    perm = torch.arange(100, dtype=torch.int32, device=DEV)[None, :].clone()
    perm[0, 17] = 100
    with pytest.raises(dig.DigError) as e:
        solver.closure_train(X, T, epochs=1, batch=32, perm=perm)
    assert e.value.code == -1


def test_loss_matches_oracle(solver):
    p = random_net(21)
    solver.closure_set(p)
    rng = np.random.default_rng(22)
    X = rng.standard_normal((1500, 13)).astype(np.float32)
    T = rng.standard_normal((1500, 8)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV)
    lo = orc.mlp_grad(p, X, T, bf16=True)[0]
    assert abs(solver.closure_loss(Xd, Td) - lo) <= 1e-3 * lo
    li = ((X[:, 5:13].astype(np.float64) - T) ** 2).mean()
    assert abs(solver.closure_loss(Xd, Td, identity=True) - li) <= 1e-12 * li


def window_state(scen, steps, **over):
    """Oracle after `steps` steps with moving average, window and cumulative
    sums; returns it with its particles, sums and wall fluxes."""
    o = orc.Oracle(scen, **over)
    o.init()
    o.step(steps, orc.EWMA | orc.WINDOW | orc.CUMUL)
    return o, o.read(), {w: o.moments(w) for w in (orc.PHI_EWMA, orc.PHI_WINDOW, orc.PHI_CUM)}, o.wall_flux()


def gpu_with_state(scen, steps, parts, phis, wf, **over):
    g = dig.Solver(scen, DEV, **over)
    g.init()
    g.step(steps, dig.WINDOW | dig.CUMUL | dig.SYNC)  # window / cumulative step counts as the oracle's
    g.write(*parts)
    for w, ph in phis.items():
        g.write_moments(w, ph)
    g.write_wall_flux(wf, steps)
    return g


def test_features_and_targets_parity():
    """S12 inputs from the window sums and S13 targets from the cumulative sums
    of an identical state, over stacked rows with invalid ones."""
    s = W.cavity_scenario(4, 24_000, 0.1, seed=19)
    o, parts, phis, wf = window_state(s, 30)
    g = gpu_with_state(s, 30, parts, phis, wf)
    Xg = g.closure_features(dig.PHI_WINDOW).cpu().numpy()
    Xo = o.closure_features(orc.PHI_WINDOW)
    assert np.all(np.abs(Xg - Xo) <= 1e-5 * np.abs(Xo).max(axis=0) + 1e-7), np.abs(Xg - Xo).max(axis=0)
    assert np.all(Xo[:, 0] > 0)
    Xs = np.concatenate([Xo, 1.1 * Xo, Xo])
    Xs[len(Xo) + 3] = 0.0
    Yg = g.closure_targets(dig.PHI_CUM, torch.from_numpy(Xs).to(DEV)).cpu().numpy()
    Yo = o.closure_targets(orc.PHI_CUM, Xs)
    assert np.all(Yg[len(Xo) + 3] == 0)
    assert np.all(np.abs(Yg - Yo) <= 1e-5 * np.abs(Yo).max(axis=0) + 1e-7), np.abs(Yg - Yo).max(axis=0)


def test_coupling_with_learned_closure_parity():
    """dig_couple with the learned closure: the same cells take the network's
    HoT (the rest fall back to the sampled HoT), HoT and M^{k+1} agree within
    the BF16 tolerance."""
    s = W.cavity_scenario(4, 24_000, 0.1, seed=23)
    over = dict(N_m=60, passes=2, KnD_max=1.0, closure=1)
    o, parts, phis, wf = window_state(s, 40, **over)
    g = gpu_with_state(s, 40, parts, phis, wf, **over)
    p = random_net(31, scale=0.2, bias=0.01)
    o.closure_set(p)
    g.closure_set(p)
    rg, ro = g.couple(), o.couple()
    assert ro["n_learned"] > 0.9 * o.n_tets
    assert rg["n_learned"] == ro["n_learned"]
    assert rg["n_rejected"] == ro["n_rejected"] and rg["iters"] == ro["iters"]
    Hg, Ho = g.read_couple(1), o.read_couple(1)
    sc = np.abs(Ho).max(axis=0) + 1e-30
    assert np.all(np.abs(Hg - Ho) <= 2e-2 * sc), (np.abs(Hg - Ho) / sc).max(axis=0)
    Mg, Mo = g.read_couple(2), o.read_couple(2)
    assert np.all(np.abs(Mg - Mo) <= 2e-3 * (np.abs(Mo).max(axis=0) + 1e-3)), np.abs(Mg - Mo).max(axis=0)
    # without the network the coupling is the plain DIG coupling
    g2 = gpu_with_state(s, 40, parts, phis, wf, **dict(over, closure=0))
    g2.closure_set(p)
    assert g2.couple()["n_learned"] == 0


def test_trained_closure_beats_window_average():
    """S13 end to end on the GPU: cell data generated by the solver (50-step
    windows as inputs, the long-time average as target), trained with the
    library's own kernels, reduces the error of the HoT against the long-time
    average on held-out windows well below that of the window HoT itself (the
    method without the network); the coupling then uses it."""
    s = W.cavity_scenario(6, 130_000, 0.1, seed=29)
    g = dig.Solver(s, DEV, N_m=100, closure=1)
    g.init()
    g.step(600, dig.EWMA)
    g.sample(dig.RESET_CUMUL)
    n, nwin, wsteps = g.n_tets, 100, 25
    X = torch.empty((nwin * n, 13), dtype=torch.float32, device=DEV)
    for w in range(nwin):
        g.sample(dig.RESET_WINDOW)
        g.step(wsteps, dig.EWMA | dig.WINDOW | dig.CUMUL)
        g.closure_features(dig.PHI_WINDOW, X[w * n:(w + 1) * n])
    Y = g.closure_targets(dig.PHI_CUM, X)
    ntr = 80 * n
    Xtr, Ytr, Xva, Yva = X[:ntr].contiguous(), Y[:ntr].contiguous(), X[ntr:].contiguous(), Y[ntr:].contiguous()
    assert torch.all(Xva[:, 0] > 0)
    g.closure_init(5)
    epochs = 8
    rng = np.random.default_rng(6)
    perm = torch.from_numpy(np.stack([rng.permutation(ntr) for _ in range(epochs)]).astype(np.int32)).to(DEV)
    loss = g.closure_train(Xtr, Ytr, epochs=epochs, batch=512, lr=2e-3, perm=perm)
    assert loss[-1] < 0.5 * loss[0], loss
    net = g.closure_loss(Xva, Yva)
    raw = g.closure_loss(Xva, Yva, identity=True)
    print(f"closure gain: train loss {loss[0]:.3e} -> {loss[-1]:.3e}; held-out MSE net {net:.3e} "
          f"vs window HoT {raw:.3e} (ratio {net / raw:.3f})")
    assert net < 0.6 * raw, (net, raw)
    # the coupling takes the trained closure's HoT
    g.sample(dig.RESET_WINDOW)
    g.step(wsteps, dig.EWMA | dig.WINDOW | dig.WALLFLUX)
    r = g.couple()
    assert r["n_learned"] > 0.9 * n and r["iters"] > 0


def flow_windows(U_lid, seed, nwin=60, wsteps=25):
    """Closure inputs (25-step windows) and targets (the long-time average's
    HoT) of the 6^3-hexahedra Kn = 0.1 cavity with lid speed U_lid."""
    s = W.cavity_scenario(6, 130_000, 0.1, seed=seed, U_lid=U_lid)
    g = dig.Solver(s, DEV, N_m=100)
    g.init()
    g.step(600, dig.EWMA)
    g.sample(dig.RESET_CUMUL)
    n = g.n_tets
    X = torch.empty((nwin * n, 13), dtype=torch.float32, device=DEV)
    for w in range(nwin):
        g.sample(dig.RESET_WINDOW)
        g.step(wsteps, dig.EWMA | dig.WINDOW | dig.CUMUL)
        g.closure_features(dig.PHI_WINDOW, X[w * n:(w + 1) * n])
    Y = g.closure_targets(dig.PHI_CUM, X)
    return g, X, Y


def test_trained_closure_transfers_to_another_flow():
    """S13 without leakage: the closure trained on two other flows of the
    cavity (lid 30 and 70 m/s, their own seeds) lowers the error of the HoT
    against the long-time average on the windows of a third flow it never saw
    (lid 50 m/s, another seed), compared with the window HoT itself."""
    Xs, Ys = [], []
    for U_lid, seed in ((30.0, 41), (70.0, 43)):
        g, X, Y = flow_windows(U_lid, seed)
        Xs.append(X)
        Ys.append(Y)
        g.close()
    X, Y = torch.cat(Xs).contiguous(), torch.cat(Ys).contiguous()
    gt, Xt, Yt = flow_windows(50.0, 47, nwin=20)
    gt.closure_init(5)
    epochs = 8
    rng = np.random.default_rng(6)
    perm = torch.from_numpy(np.stack([rng.permutation(len(X)) for _ in range(epochs)]).astype(np.int32)).to(DEV)
    loss = gt.closure_train(X, Y, epochs=epochs, batch=512, lr=2e-3, perm=perm)
    assert loss[-1] < 0.5 * loss[0], loss
    net = gt.closure_loss(Xt.contiguous(), Yt.contiguous())
    raw = gt.closure_loss(Xt.contiguous(), Yt.contiguous(), identity=True)
    print(f"closure transfer: held-out-flow MSE net {net:.3e} vs window HoT {raw:.3e} (ratio {net / raw:.3f})")
    assert net < 0.7 * raw, (net, raw)
