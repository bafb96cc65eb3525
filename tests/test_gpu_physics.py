"""Physics checks of the DIG coupling on the GPU (not element-wise parity):
where DSMC resolves the flow, DIG must converge to DSMC's field."""
import numpy as np
import pytest

from paper_2607_08195_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_08195_gb300 import dig  # noqa: E402


def centreline(scen, m, vol):
    """u_x(y) and u_y(x) over the hexahedra of the central half of the cavity
    in the other two directions (mass-weighted), over the lid speed."""
    nt = len(scen.mesh.tets)
    nh = round((nt // 6) ** (1.0 / 3.0))
    h = np.arange(nt) // 6
    i, j, k = h // (nh * nh), (h // nh) % nh, h % nh
    mid = lambda a: (a >= nh // 4) & (a < nh - nh // 4)  # noqa: E731
    w = m[:, 1] * vol
    out = []
    for sel, idx, q in ((mid(i) & mid(k), j, 2), (mid(j) & mid(k), i, 3)):
        den = np.bincount(idx[sel], w[sel], nh)
        out.append(np.bincount(idx[sel], w[sel] * m[sel, q], nh) / den)
    return np.concatenate(out) / 50.0


def test_dig_converges_to_the_dsmc_field_where_dsmc_is_resolved():
    """Argon cavity at Kn = 0.1 (6^3 hexes, cells 1.7 mean free paths, 200k
    particles): after 20 warm-up cycles of 200 steps, the cumulative averages
    of 40 more cycles of plain DSMC and of DIG (a coupling every cycle) give
    the same centreline profiles within 0.02 U_w (RMS; the statistical error
    is about 0.005 U_w): the synthetic solve's flux, gradients and wall
    closure do not move DSMC's steady state."""
    s = W.cavity_scenario(6, 200_000, 0.1, seed=3)
    P = s.mesh.nodes[s.mesh.tets]
    vol = np.abs(np.einsum("ni,ni->n", P[:, 1] - P[:, 0], np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]))) / 6.0
    prof = {}
    for kind in ("plain", "dig"):
        g = dig.Solver(s, "cuda:0")
        g.init()
        for c in range(60):
            if c == 20:
                g.sample(dig.RESET_CUMUL)
            g.step(200, dig.EWMA | (dig.CUMUL if c >= 20 else 0))
            if kind == "dig":
                g.couple()
        prof[kind] = centreline(s, g.moments(dig.PHI_CUM | dig.MACRO), vol)
        g.close()
    rms = float(np.sqrt(np.mean((prof["dig"] - prof["plain"]) ** 2)))
    assert np.abs(prof["plain"]).max() > 0.1  # a developed vortex
    assert rms < 0.02, (rms, prof)


def test_vss_stress_relaxation_rate_on_the_gpu():
    """VSS scattering on the CUDA path at ten times the oracle pin's size: for
    Maxwell molecules (omega = 1) in a closed specular box, the stress anisotropy
    decays as exp(-p t / mu), and with the same total cross section VSS with
    alpha = 3 has 4 alpha/((alpha + 1)(alpha + 2)) = 3/5 of it as viscosity cross
    section against 2/3 for VHS, so its decay rate is 0.9 times VHS's.  The two
    runs share the initial state and the time step."""
    import dataclasses
    import math

    K_B = W.K_B
    n = 480_000
    rates = {}
    for alpha in (1.0, 3.0):
        gas = W.Gas(mass=6.63e-26, d_ref=4.17e-10, omega=1.0, T_ref=273.0, alpha=alpha)
        mesh = W.closed_box(4, L=1e-3, kind=W.BC_SPECULAR, T_w=273.0)
        n0 = 1.677e22
        mu_vhs = dataclasses.replace(gas, alpha=1.0).mu_ref()
        s = W.Scenario(gas=gas, mesh=mesh, n_particles=n, n_init=n0, T_init=273.0, u_init=(0.0, 0.0, 0.0),
                       F_N=n0 * 1e-9 / n, dt=0.02 * mu_vhs / (n0 * K_B * 273.0), seed=41, L=1e-3, Kn=0.1,
                       capacity=2 * n)
        rng = np.random.default_rng(5)
        x, v, Ir, cell = W.random_particles(rng, s, n)
        sig = math.sqrt(K_B * 273.0 / gas.mass)
        v = (rng.standard_normal((n, 3)) * sig * np.array([1.3, 0.8, 0.8])).astype(np.float32)
        g = dig.Solver(s, "cuda:0")
        g.write(x, v, Ir, cell)

        def aniso():
            c = g.read()[1].astype(np.float64)
            c -= c.mean(0)
            m2 = (c * c).mean(0)
            return m2[0] - 0.5 * (m2[1] + m2[2]), m2.sum() / 3

        a0, th = aniso()
        T = gas.mass * th / K_B
        p = n0 * K_B * T
        mu = mu_vhs * (T / gas.T_ref) ** gas.omega
        steps = 50
        g.step(steps, dig.SYNC)
        a, _ = aniso()
        rates[alpha] = -math.log(a / a0) / (p * steps * s.dt / mu)
    assert abs(rates[1.0] - 1.0) < 0.05, rates
    assert abs(rates[3.0] / rates[1.0] - 0.9) < 0.02, rates  # statistical error ~0.007


def test_gpu_fp32_path_against_fp64_oracle_config1():
    """The precision statement of the CUDA path: config 1 (6^3-hexahedra Kn =
    0.1 argon cavity, 20,000 particles) on the GPU (FP32 velocities and FP32
    per-step cell sums into FP64 accumulators) against the oracle built with
    FP64 velocities and collision arithmetic, same seed, 10 batches of 30
    steps after 200: per cell and moment (density, velocity, temperature,
    stress deviator, heat flux) the difference in units of the two runs'
    combined batch-mean standard error has an RMS below 1.35 (Student's t
    with 9 degrees of freedom: 1.13) and under 1 % of cells beyond 4."""
    from oracle import orc
    from tests.test_oracle_precision import fp32_fp64_report

    s = W.config_small()
    g = dig.Solver(s, "cuda:0")
    g.init()
    g.step(200, 0)
    a = []
    for _ in range(10):
        g.sample(dig.RESET_CUMUL)
        g.step(30, dig.CUMUL)
        a.append(g.moments(dig.PHI_CUM | dig.MACRO))
    o = orc.Oracle(s, v64=True)
    o.init()
    o.step(200, 0)
    b = []
    for _ in range(10):
        o.sample(orc.RESET_CUMUL)
        o.step(30, orc.CUMUL)
        b.append(o.moments(orc.PHI_CUM | orc.MACRO))
    report = fp32_fp64_report(np.array(a), np.array(b))
    print("GPU FP32 vs FP64 oracle:", {k: {q: round(x, 4) for q, x in v.items()} for k, v in report.items()})
    for name, r in report.items():
        assert r["rms_z"] < 1.35 and r["tail4"] < 0.01, (name, r)
