"""Pins of the CPU oracle against things fixed outside it: published known-answer
vectors, closed forms of kinetic theory, invariants and brute force on tiny
meshes.  No GPU needed.

Each test names the property it checks and where that property comes from.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

from oracle import orc
from paper_2607_08195_gb300 import workload as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
KB = W.K_B


def box_scenario(nh=1, n_particles=6000, kind=W.BC_SPECULAR, gas=W.ARGON, T=273.0, n=1.677e22,
                 dt_factor=0.2, seed=11, L=1e-3, F_N=None):
    mesh = W.closed_box(nh, L=L, kind=kind, T_w=T)
    mu = gas.mu_ref() * (T / gas.T_ref) ** gas.omega
    p = n * KB * T
    return W.Scenario(gas=gas, mesh=mesh, n_particles=n_particles, n_init=n, T_init=T,
                      u_init=(0.0, 0.0, 0.0), F_N=F_N if F_N is not None else n * L ** 3 / n_particles,
                      dt=dt_factor * mu / p, seed=seed, L=L, Kn=0.1, capacity=2 * n_particles)


# --------------------------------------------------------------------------- RNG
def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors (Salmon et al. 2011)."""
    rows = [l.split() for l in open(os.path.join(GOLD, "philox_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = orc.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


# ------------------------------------------------------------------- own ln / exp
def test_own_log_exp_match_libm():
    """The FP32 ln/exp used in collision decisions agree with the true functions
    (closed form) to a few FP32 ulps over the ranges the collision arithmetic uses."""
    xs = np.geomspace(1e-6, 1e12, 400)
    for x in xs:
        x32 = float(np.float32(x))
        assert abs(orc.lnf(x32) - math.log(x32)) <= 2e-6 + 1e-7 * abs(math.log(x32))
    for y in np.linspace(-30.0, 30.0, 401):
        y32 = float(np.float32(y))
        assert abs(orc.expf(y32) / math.exp(y32) - 1.0) <= 5e-7
    for x in (1.0, 3.0, 1e4, 2.5e5):
        assert abs(orc.powf(x, 0.19) / x ** 0.19 - 1.0) < 2e-6


# ---------------------------------------------------------------------------- mesh
def test_mesh_tables():
    """Kuhn-split cube: volumes sum to L^3, the neighbour relation is symmetric,
    normals are unit and point away from the tet, boundary faces = 12 nh^2."""
    nh, L = 3, 1e-3
    s = box_scenario(nh=nh, L=L)
    o = orc.Oracle(s)
    mi = o.mesh_info()
    assert abs(mi["vol"].sum() / L ** 3 - 1.0) < 1e-12
    assert mi["n_bfaces"] == 12 * nh * nh
    nbr, nf = mi["nbr"], mi["nbr_face"]
    for t in range(len(nbr)):
        for f in range(4):
            if nbr[t, f] >= 0:
                assert nbr[nbr[t, f], nf[t, f]] == t
                # the shared face's normals are opposite
                assert np.allclose(mi["normals"][t, f], -mi["normals"][nbr[t, f], nf[t, f]], atol=1e-12)
    assert np.allclose(np.linalg.norm(mi["normals"], axis=2), 1.0, atol=1e-14)
    P = s.mesh.nodes[s.mesh.tets]
    cen = P.mean(axis=1)
    for f in range(4):
        # centroid is strictly inside every face plane; the opposite vertex too
        sd = mi["d"][:, f] - np.einsum("ni,ni->n", mi["normals"][:, f], cen)
        assert np.all(sd > 0)
        sv = mi["d"][:, f] - np.einsum("ni,ni->n", mi["normals"][:, f], P[:, f])
        assert np.all(sv > 0)


def test_mesh_rejects_bad_input():
    s = box_scenario(nh=1)
    bad = dataclasses.replace(s, mesh=dataclasses.replace(s.mesh, face_tag=np.full_like(s.mesh.face_tag, -1)))
    with pytest.raises(RuntimeError, match="boundary face"):
        orc.Oracle(bad)
    nodes = s.mesh.nodes.copy()
    tets = s.mesh.tets.copy()
    tets[0, 3] = tets[0, 2]  # collapse a tet
    with pytest.raises(RuntimeError, match="degenerate|non-manifold|boundary"):
        orc.Oracle(dataclasses.replace(s, mesh=dataclasses.replace(s.mesh, nodes=nodes, tets=tets)))


# ------------------------------------------------------------------- tracking
def barycentric(nodes, tets, cell, x):
    P = nodes[tets[cell]]  # [n, 4, 3]
    T = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=2)
    lam = np.linalg.solve(T, (x - P[:, 0])[..., None])[..., 0]
    return np.concatenate([1.0 - lam.sum(axis=1, keepdims=True), lam], axis=1)


def test_point_in_tet_brute_force():
    """P7: after each step every particle lies inside the tet it was tracked to,
    by barycentric coordinates computed from the nodes (independent of the
    oracle's planes); diffuse walls, a moving lid and collisions on."""
    s = W.cavity_scenario(2, 3000, 0.1, seed=5)
    o = orc.Oracle(s)
    o.init()
    for _ in range(12):
        o.step(1, orc.EWMA)
        x, v, Ir, cell = o.read()
        assert len(cell) == 3000
        lam = barycentric(s.mesh.nodes, s.mesh.tets, cell, x)
        assert lam.min() > -1e-9, lam.min()
        assert np.all(np.diff(cell) >= 0)  # sorted by cell
    c = o.counters()
    assert c["cross"] > 0 and c["wall"] > 0 and c["coll"] > 0 and c["stuck"] == 0


def test_specular_box_conserves_speed_and_free_flight():
    """P8: specular walls on the axis-aligned cube conserve every particle's speed
    exactly (the reflection flips one component); with collisions off the total
    energy is conserved bit for bit; free flight with no crossing equals x + v dt
    to 1 ulp."""
    s = box_scenario(nh=2, n_particles=2000, F_N=1e-30)
    o = orc.Oracle(s)
    o.init()
    x0, v0, _, _ = o.read()
    sp0 = np.sort(np.linalg.norm(v0.astype(np.float64), axis=1))
    o.step(30, 0)
    x1, v1, _, _ = o.read()
    assert o.counters()["coll"] == 0 and o.counters()["wall"] > 0
    sp1 = np.sort(np.linalg.norm(v1.astype(np.float64), axis=1))
    assert np.array_equal(sp0, sp1)
    lam = barycentric(s.mesh.nodes, s.mesh.tets, o.read()[3], x1)
    assert lam.min() > -1e-9
    # free flight inside one cell
    cen = s.mesh.nodes[s.mesh.tets[5]].mean(axis=0)
    v = np.array([3.0, -2.0, 1.0], np.float32)
    xn, vn, cn = o.track_one(cen, v, 5, 0, 1)
    assert cn == 5
    ref = cen + v.astype(np.float64) * s.dt
    assert np.all(np.abs(xn - ref) <= np.spacing(np.abs(ref)))


def test_diffuse_wall_distribution():
    """Diffuse re-emission at T_w: normal speed has the flux-weighted half-range
    Maxwellian law (mean sigma sqrt(pi/2), mean square 2 sigma^2); tangential
    components are N(U_w, sigma^2)."""
    s = W.cavity_scenario(1, 10, 0.1, seed=3, U_lid=100.0)
    o = orc.Oracle(s)
    mi = o.mesh_info()
    # pick a tet with a lid face (+y side); the face normal is +y
    tags = s.mesh.face_tag
    t, f = [(t, f) for t in range(len(tags)) for f in range(4) if tags[t, f] == 1][0]
    assert np.allclose(mi["normals"][t, f], [0, 1, 0])
    cen = s.mesh.nodes[s.mesh.tets[t]].mean(axis=0)
    vs = []
    for slot in range(20000):
        # particle shot straight at the lid with a short flight: one hit, then rebound
        x, v, c = o.track_one(cen, np.array([0.0, 5000.0, 0.0], np.float32), t, slot, 7)
        vs.append(v)
    v = np.array(vs, np.float64)
    sig = math.sqrt(KB * 273.0 / s.gas.mass)
    vn = -v[:, 1]
    assert np.all(vn > 0)
    n = len(vn)
    assert abs(vn.mean() - sig * math.sqrt(math.pi / 2)) < 4 * vn.std() / math.sqrt(n)
    assert abs((vn ** 2).mean() - 2 * sig ** 2) < 4 * (vn ** 2).std() / math.sqrt(n)
    assert abs(v[:, 0].mean() - 100.0) < 4 * sig / math.sqrt(n)
    assert abs(v[:, 2].mean()) < 4 * sig / math.sqrt(n)
    for comp in (0, 2):
        assert abs(v[:, comp].std() / sig - 1.0) < 4 * 0.71 / math.sqrt(n)


def test_diffuse_box_thermalises_without_collisions():
    """P9: collisionless gas in a closed box with diffuse walls at T_w relaxes to
    T = T_w and u = 0, whatever its initial temperature."""
    mesh = W.closed_box(1, L=1e-3, kind=W.BC_DIFFUSE, T_w=273.0)
    s = W.Scenario(gas=W.ARGON, mesh=mesh, n_particles=20000, n_init=1e22, T_init=500.0,
                   u_init=(30.0, 0.0, 0.0), F_N=1e-30, dt=2e-7, seed=4, L=1e-3, Kn=1.0, capacity=40000)
    o = orc.Oracle(s)
    o.init()
    o.step(300, 0)
    o.sample(orc.RESET_CUMUL)
    o.step(200, orc.CUMUL)
    Phi = o.moments(orc.PHI_CUM).sum(axis=0)
    N = Phi[0]
    u = Phi[1:4] / N
    cc = Phi[4:7] / N - u * u
    T = s.gas.mass * cc.sum() / (3 * KB)
    # particles are strongly correlated between steps; 2e4 particles x ~30
    # independent wall-to-wall flights: tolerance 1 %
    assert abs(T / 273.0 - 1.0) < 0.01, T
    assert np.all(np.abs(u) < 3.0)


# ------------------------------------------------------------------ collisions
def test_equilibrium_collision_rate():
    """P1: in an equilibrium VHS gas the NTC scheme collides at
    (1/2) N (N-1)/V F_N <sigma_T c_r> per unit time, with
    n <sigma_T c_r> = nu = 4 d^2 n sqrt(pi k T_ref/m) (T/T_ref)^(1-omega)
    (Bird 1994 eq. 4.64)."""
    s = box_scenario(nh=1, n_particles=6000)
    o = orc.Oracle(s)
    o.init()
    o.step(20, 0)  # let (sigma c_r)_max settle
    c0 = o.counters()["coll"]
    expected = 0.0
    g = s.gas
    V = s.L ** 3 / 6
    nsteps = 150
    for _ in range(nsteps):
        x, v, Ir, cell = o.read()
        vv = v.astype(np.float64)
        T = g.mass * ((vv - vv.mean(0)) ** 2).sum(1).mean() / (3 * KB)
        sc = 4 * g.d_ref ** 2 * math.sqrt(math.pi * KB * g.T_ref / g.mass) * (T / g.T_ref) ** (1 - g.omega)
        Nc = np.bincount(cell, minlength=6).astype(np.float64)
        o.step(1, 0)
        expected += (0.5 * Nc * (Nc - 1) * s.F_N * sc * s.dt / V).sum()
    got = o.counters()["coll"] - c0
    assert abs(got - expected) < 4 * math.sqrt(expected), (got, expected)


def test_collisions_conserve_momentum_energy():
    """P5: each collision conserves momentum and energy; with a time step so short
    that no particle leaves its cell (F_N raised to keep the collision count), the
    per-cell momentum and energy after a step equal those before within FP32 rounding."""
    s = box_scenario(nh=1, n_particles=3000, dt_factor=1e-6)
    s = dataclasses.replace(s, F_N=s.F_N * 2e5)
    o = orc.Oracle(s)
    o.init()
    x0, v0, _, c0 = o.read()
    o.step(1, orc.RECORD_PAIRS)
    x1, v1, _, c1 = o.read()
    assert np.array_equal(c0, c1)
    assert o.counters()["coll"] > 200
    for c in range(6):
        a, b = v0[c0 == c].astype(np.float64), v1[c1 == c].astype(np.float64)
        scale = np.abs(a).sum()
        assert np.all(np.abs(a.sum(0) - b.sum(0)) <= 8 * 2 ** -24 * scale)
        ea, eb = (a * a).sum(), (b * b).sum()
        assert abs(ea - eb) <= 8 * 2 ** -24 * ea * 4
    P = o.pairs()
    assert len(P) == o.counters()["cand"]
    assert np.all(P[:, 2] != P[:, 3])


def test_bimodal_heat_bath_relaxes_to_maxwellian():
    """P4: two counter-streaming beams relax to a Maxwellian: kurtosis
    <c^4>/<c^2>^2 -> 5/3, energy conserved to FP32 rounding."""
    s = box_scenario(nh=1, n_particles=12000)
    o = orc.Oracle(s)
    rng = np.random.default_rng(0)
    n = 12000
    sig = math.sqrt(KB * 273.0 / s.gas.mass)
    U = 2.0 * sig
    v = rng.standard_normal((n, 3)) * 0.3 * sig
    v[: n // 2, 0] += U
    v[n // 2:, 0] -= U
    cell = rng.integers(0, 6, n).astype(np.int32)
    P = s.mesh.nodes[s.mesh.tets[cell]]
    w = rng.dirichlet(np.ones(4), n)
    x = np.einsum("nk,nkc->nc", w, P)
    o.write(x, v.astype(np.float32), np.zeros(n, np.float32), cell)
    E0 = (v.astype(np.float32).astype(np.float64) ** 2).sum()
    k0 = None
    for _ in range(60):
        o.step(1, 0)
    _, v1, _, _ = o.read()
    c = v1.astype(np.float64)
    c = c - c.mean(0)
    c2 = (c * c).sum(1)
    kurt = (c2 ** 2).mean() / c2.mean() ** 2
    assert abs(kurt - 5.0 / 3.0) < 0.05, kurt
    E1 = (v1.astype(np.float64) ** 2).sum()
    assert abs(E1 / E0 - 1.0) < 1e-5


def test_maxwell_molecule_stress_relaxation():
    """P4 (second part): for Maxwell molecules (omega = 1) an anisotropic
    temperature relaxes exactly as exp(-p t / mu) with the VHS viscosity
    (Bird eq. 4.62) -- checks the collision rate and isotropic scattering."""
    gas = W.Gas(mass=6.63e-26, d_ref=4.17e-10, omega=1.0, T_ref=273.0)
    s = box_scenario(nh=1, n_particles=24000, gas=gas, dt_factor=0.05, seed=21)
    o = orc.Oracle(s)
    rng = np.random.default_rng(1)
    n = s.n_particles
    sig = math.sqrt(KB * 273.0 / gas.mass)
    v = rng.standard_normal((n, 3)) * sig * np.array([1.3, 0.8, 0.8])
    cell = rng.integers(0, 6, n).astype(np.int32)
    P = s.mesh.nodes[s.mesh.tets[cell]]
    x = np.einsum("nk,nkc->nc", rng.dirichlet(np.ones(4), n), P)
    o.write(x, v.astype(np.float32), np.zeros(n, np.float32), cell)

    def aniso():
        _, vv, _, _ = o.read()
        c = vv.astype(np.float64)
        c -= c.mean(0)
        m2 = (c * c).mean(0)
        return m2[0] - 0.5 * (m2[1] + m2[2]), m2.sum() / 3

    a0, th = aniso()
    T = gas.mass * th / KB
    mu = gas.mu_ref() * (T / gas.T_ref) ** gas.omega
    p = s.n_init * KB * T
    for k in (10, 20, 30):
        o.step(10, 0)
        a, _ = aniso()
        pred = a0 * math.exp(-p * k * s.dt / mu)
        # statistical error of the anisotropy ~ sqrt(2/n) th
        assert abs(a - pred) < 4 * math.sqrt(2.0 / n) * th * 1.5 + 0.03 * abs(a0), (k, a, pred)


def _ks_uniform(u):
    """Kolmogorov-Smirnov distance of samples u in [0, 1] from the uniform law."""
    x = np.sort(np.asarray(u, np.float64))
    n = len(x)
    return max(np.max(np.arange(1, n + 1) / n - x), np.max(x - np.arange(n) / n))


def _vss_samples(alpha, n, seed, along_x=False):
    gas = dataclasses.replace(W.ARGON, alpha=alpha)
    o = orc.Oracle(box_scenario(gas=gas))
    rng = np.random.default_rng(seed)
    if along_x:
        g = np.zeros((n, 3))
        g[:, 0] = rng.choice([-1.0, 1.0], n) * rng.uniform(1.0, 900.0, n)
    else:
        g = rng.standard_normal((n, 3)) * rng.uniform(0.1, 900.0, (n, 1))
    g = g.astype(np.float32)
    e = o.vss_directions(g).astype(np.float64)
    u = g.astype(np.float64)
    u /= np.linalg.norm(u, axis=1)[:, None]
    return u, e


def _azimuth(u, e):
    """Angle of e about u in a frame built independently of the oracle's."""
    r = np.where(np.abs(u[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    a = r - (r * u).sum(1)[:, None] * u
    a /= np.linalg.norm(a, axis=1)[:, None]
    b = np.cross(u, a)
    return np.arctan2((e * b).sum(1), (e * a).sum(1))


@pytest.mark.parametrize("alpha", [1.0, 1.4, 3.0, 0.6])
@pytest.mark.parametrize("along_x", [False, True])
def test_vss_deflection_law(alpha, along_x):
    """VSS scattering (paper Sec. 2.1; Koura & Matsumoto 1991): b/d = cos^alpha(chi/2)
    with (b/d)^2 uniform gives P(cos chi <= x) = ((1 + x)/2)^alpha, so
    <cos chi> = (alpha - 1)/(alpha + 1) and <sin^2 chi> = 4 alpha/((alpha + 1)(alpha + 2))
    (2/3 for VHS); the azimuth about g is uniform and the direction a unit vector.
    Checked on generic relative velocities and on velocities along x (the frame's
    degenerate case)."""
    n = 100_000
    u, e = _vss_samples(alpha, n, seed=5 + int(10 * alpha), along_x=along_x)
    assert np.abs(np.linalg.norm(e, axis=1) - 1.0).max() < 1e-6
    ct = np.clip((e * u).sum(1), -1.0, 1.0)
    # probability integral transform: F(cos chi) is uniform
    assert _ks_uniform(((1.0 + ct) / 2.0) ** alpha) < 1.63 / math.sqrt(n)
    m, sd = ct.mean(), ct.std() / math.sqrt(n)
    assert abs(m - (alpha - 1.0) / (alpha + 1.0)) < 4.5 * sd
    s2 = 1.0 - ct ** 2
    assert abs(s2.mean() - 4.0 * alpha / ((alpha + 1.0) * (alpha + 2.0))) < 4.5 * s2.std() / math.sqrt(n)
    phi = _azimuth(u, e)
    assert _ks_uniform((phi + math.pi) / (2.0 * math.pi)) < 1.63 / math.sqrt(n)


def test_vss_maxwell_molecule_stress_relaxation():
    """For Maxwell molecules (omega = 1) the stress anisotropy relaxes as
    exp(-p t / mu) with mu inversely proportional to the viscosity cross section:
    VSS with alpha = 3 has 4 alpha/((alpha + 1)(alpha + 2)) = 3/5 of the total cross
    section against 2/3 for VHS, so with the same collision rate its anisotropy
    decays 0.9 times as fast.  Two runs from the same state and random stream."""
    rates = {}
    for alpha in (1.0, 3.0):
        gas = W.Gas(mass=6.63e-26, d_ref=4.17e-10, omega=1.0, T_ref=273.0, alpha=alpha)
        s = box_scenario(nh=1, n_particles=48000, gas=gas, dt_factor=0.02, seed=31)
        o = orc.Oracle(s)
        rng = np.random.default_rng(3)
        n = s.n_particles
        sig = math.sqrt(KB * 273.0 / gas.mass)
        v = rng.standard_normal((n, 3)) * sig * np.array([1.3, 0.8, 0.8])
        cell = rng.integers(0, 6, n).astype(np.int32)
        P = s.mesh.nodes[s.mesh.tets[cell]]
        x = np.einsum("nk,nkc->nc", rng.dirichlet(np.ones(4), n), P)
        o.write(x, v.astype(np.float32), np.zeros(n, np.float32), cell)

        def aniso():
            _, vv, _, _ = o.read()
            c = vv.astype(np.float64)
            c -= c.mean(0)
            m2 = (c * c).mean(0)
            return m2[0] - 0.5 * (m2[1] + m2[2]), m2.sum() / 3

        a0, th = aniso()
        T = gas.mass * th / KB
        # the VHS viscosity of the same diameter fixes the time unit of both runs
        mu_vhs = dataclasses.replace(gas, alpha=1.0).mu_ref() * (T / gas.T_ref) ** gas.omega
        p = s.n_init * KB * T
        steps = 50
        o.step(steps, 0)
        a, _ = aniso()
        rates[alpha] = -math.log(a / a0) / (p * steps * s.dt / mu_vhs)
        # against the VSS viscosity itself (Gas.mu_ref carries the alpha factor)
        mu = gas.mu_ref() * (T / gas.T_ref) ** gas.omega
        assert abs(-math.log(a / a0) / (p * steps * s.dt / mu) - 1.0) < 0.05, (alpha, rates[alpha])
    assert abs(rates[3.0] / rates[1.0] - 0.9) < 0.02, rates


def test_jeans_landau_rotational_relaxation():
    """P3: homogeneous diatomic gas with T_t != T_r follows the Jeans-Landau law
    dT_r/dt = (T - T_r)/(Z_r tau), tau = mu(T_t)/p_t (paper Eq. jeans_landau),
    with T = (3 T_t + 2 T_r)/5 conserved; checks the Borgnakke-Larsen reading."""
    gas = W.NITROGEN
    s = box_scenario(nh=1, n_particles=30000, gas=gas, dt_factor=0.1, seed=8, T=300.0)
    o = orc.Oracle(s)
    rng = np.random.default_rng(2)
    n = s.n_particles
    Tt0, Tr0 = 400.0, 150.0
    sig = math.sqrt(KB * Tt0 / gas.mass)
    v = rng.standard_normal((n, 3)) * sig
    Ir = rng.exponential(Tr0, n)
    cell = rng.integers(0, 6, n).astype(np.int32)
    P = s.mesh.nodes[s.mesh.tets[cell]]
    x = np.einsum("nk,nkc->nc", rng.dirichlet(np.ones(4), n), P)
    o.write(x, v.astype(np.float32), Ir.astype(np.float32), cell)

    def temps():
        _, vv, I, _ = o.read()
        c = vv.astype(np.float64)
        c -= c.mean(0)
        return gas.mass * (c * c).sum(1).mean() / (3 * KB), I.astype(np.float64).mean()

    Tt, Tr = temps()
    Teq = (3 * Tt + 2 * Tr) / 5
    n_num = s.n_init  # number density of the box

    def rhs(Tr_):
        Tt_ = (5 * Teq - 2 * Tr_) / 3
        mu = gas.mu_ref() * (Tt_ / gas.T_ref) ** gas.omega
        tau = mu / (n_num * KB * Tt_)
        return (Teq - Tr_) / (gas.Z_rot * tau)

    Tr_ode = Tr
    t_step = s.dt
    for blk in range(6):
        for _ in range(20):
            # RK4 per time step
            k1 = rhs(Tr_ode)
            k2 = rhs(Tr_ode + 0.5 * t_step * k1)
            k3 = rhs(Tr_ode + 0.5 * t_step * k2)
            k4 = rhs(Tr_ode + t_step * k3)
            Tr_ode += t_step * (k1 + 2 * k2 + 2 * k3 + k4) / 6
        o.step(20, 0)
        Tt, Tr = temps()
        assert abs((3 * Tt + 2 * Tr) / 5 - Teq) < 1e-3 * Teq
        se = Tr / math.sqrt(n)
        assert abs(Tr - Tr_ode) < 4 * se + 0.01 * (Teq - Tr0), (blk, Tr, Tr_ode)


# -------------------------------------------------------------------- sampling
def test_moments_match_two_pass_central_moments():
    """P11: moments derived from the raw summation variables equal the direct
    two-pass central moments of the particles in each cell (Eq. dsmc_temperatures)."""
    gas = W.NITROGEN
    s = W.cavity_scenario(2, 4000, 0.1, seed=9, gas=gas)
    o = orc.Oracle(s)
    o.init()
    o.step(3, 0)
    M = o.moments(orc.PHI_INST | orc.MACRO)
    x, v, Ir, cell = o.read()
    vol = o.mesh_info()["vol"]
    m = gas.mass
    for c in range(0, len(vol), 7):
        sel = cell == c
        if sel.sum() < 2:
            continue
        vv = v[sel].astype(np.float64)
        I = Ir[sel].astype(np.float64)
        N = len(vv)
        u = vv.mean(0)
        cc = vv - u
        c2 = (cc * cc).sum(1)
        rho = m * s.F_N * N / vol[c]
        Tt = m * c2.mean() / (3 * KB)
        Tr = I.mean()
        sig = rho * (np.einsum("ni,nj->ij", cc, cc) / N - np.eye(3) * c2.mean() / 3)
        qt = 0.5 * rho * (cc * c2[:, None]).mean(0)
        qr = s.F_N * N / vol[c] * KB * (cc * I[:, None]).mean(0)
        ref = np.concatenate([[N, rho], u, [Tt, Tr, (3 * Tt + 2 * Tr) / 5],
                              [sig[0, 0], sig[1, 1], sig[2, 2], sig[0, 1], sig[0, 2], sig[1, 2]], qt, qr])
        scale = np.concatenate([[N, rho], [np.abs(vv).max()] * 3, [Tt] * 3, [rho * (vv ** 2).sum(1).mean()] * 6,
                                [rho * np.abs(vv).max() ** 3] * 3, [s.F_N * N / vol[c] * KB * I.mean() * np.abs(vv).max()] * 3])
        assert np.all(np.abs(M[c] - ref) <= 1e-9 * scale), c


def test_ewma_window_cumulative_recurrences():
    """P11: the moving average follows Eq. exponential_average_moments with n_a
    effective samples once n_a samples exist, and is the plain mean of all
    samples before (after m <= n_a steps it equals their mean); the window
    and cumulative sums are plain sums of the per-step sums."""
    s = W.cavity_scenario(2, 3000, 0.1, seed=10)
    o = orc.Oracle(s, n_a=7)
    o.init()
    ph = []
    for k in range(12):
        o.step(1, orc.EWMA | orc.WINDOW | (orc.CUMUL if k >= 4 else 0))
        ph.append(o.moments(orc.PHI_INST))
        if k == 6:
            assert np.allclose(o.moments(orc.PHI_EWMA), sum(ph) / 7.0, rtol=1e-12, atol=0)
    e = sum(ph[:7]) / 7.0
    for p in ph[7:]:
        e = (6.0 / 7.0) * e + p / 7.0
    assert np.allclose(o.moments(orc.PHI_EWMA), e, rtol=1e-12, atol=0)
    assert np.allclose(o.moments(orc.PHI_WINDOW), sum(ph), rtol=1e-12, atol=0)
    assert np.allclose(o.moments(orc.PHI_CUM), sum(ph[4:]), rtol=1e-12, atol=0)
    o.sample(orc.RESET_WINDOW)
    assert np.all(o.moments(orc.PHI_WINDOW) == 0)


def test_bookkeeping_closed_cavity():
    """P6: in the closed cavity the particle count never changes and the array
    stays sorted by cell, stayers before arrivals in every cell."""
    s = W.config_small()
    o = orc.Oracle(s)
    o.init()
    prev_x, _, _, prev_c = o.read()
    o.step(1, 0)
    x, v, Ir, cell = o.read()
    assert len(cell) == s.n_particles
    assert np.all(np.diff(cell) >= 0)
    assert o.counters()["removed"] == 0


def test_sort_by_cell_matches_stable_argsort():
    """The standalone bucket sort equals numpy's stable argsort of the cell ids
    (a library routine with the same definition), with -1 entries dropped."""
    rng = np.random.default_rng(4)
    for n, nc in ((0, 5), (1, 1), (1000, 37), (20000, 1296), (5000, 5)):
        cell = rng.integers(-1, nc, size=n).astype(np.int32)
        cs, order = orc.sort_by_cell(cell, nc)
        keep = np.flatnonzero(cell >= 0)
        ref = keep[np.argsort(cell[keep], kind="stable")]
        assert np.array_equal(order, ref)
        assert np.array_equal(cs, np.concatenate([[0], np.cumsum(np.bincount(cell[keep], minlength=nc))]))


# --------------------------------------------------------------- injection (S4)
def test_sphere_mesh_and_tracking():
    """Procedural sphere workload: the graded Delaunay mesh of the shell
    between the body (R = 0.1 m) and the far field (1 m) fills the region
    between the convex hulls of the body's and the far field's points exactly
    (no gap, no overlap; scipy's hull volumes), its boundary faces lie
    on the two spheres and carry the body-wall and free-stream tags, and after
    5 steps of the oracle (injection, body reflections, outflow) every particle
    lies inside the tet it was tracked to (P7 on an unstructured mesh)."""
    R, R_far = 0.1, 1.0
    s = W.sphere_scenario(0.02, 8000, seed=5)
    m = s.mesh
    P = m.nodes[m.tets]
    vol = np.abs(np.einsum("ni,ni->n", P[:, 1] - P[:, 0], np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]))) / 6.0
    from scipy.spatial import ConvexHull

    rn = np.linalg.norm(m.nodes, axis=1)
    hull = ConvexHull(m.nodes).volume - ConvexHull(m.nodes[rn < R * (1 + 1e-9)]).volume
    assert vol.min() > 0 and abs(vol.sum() / hull - 1.0) < 1e-9
    fc = np.stack([np.delete(P, f, axis=1).mean(axis=1) for f in range(4)], axis=1)
    r = np.linalg.norm(fc, axis=2)
    body, far = m.face_tag == 0, m.face_tag == 1
    assert body.sum() > 100 and far.sum() > 20
    assert np.all((r[body] > 0.9 * R) & (r[body] <= R * (1 + 1e-12)))
    assert np.all((r[far] > 0.9 * R_far) & (r[far] <= R_far * (1 + 1e-12)))
    o = orc.Oracle(s)
    o.init()
    o.step(5, orc.EWMA)
    x, v, I, cell = o.read()
    c = o.counters()
    assert c["stuck"] == 0 and c["injected"] > 0 and c["removed"] > 0
    assert len(cell) == s.n_particles + c["injected"] - c["removed"]
    lam = barycentric(m.nodes, m.tets, cell, x)
    assert lam.min() >= -1e-9, lam.min()


def test_capsule_mesh_and_tracking():
    """Procedural capsule (nitrogen at Mach 25, 20 degrees incidence): no tet
    lies inside the body, every body-wall face lies on the body's surface
    (within the polyhedral approximation: its centroid is at most one wall
    spacing inside or outside), the far-field faces on the far sphere; after 8
    oracle steps with Borgnakke-Larsen exchange, injection, wall reflections
    and outflow every particle lies inside the tet it was tracked to."""
    s = W.capsule_scenario(0.3, 50_000, seed=5)
    m = s.mesh
    P = m.nodes[m.tets]
    assert not W.capsule_inside(P.mean(axis=1)).any()
    fc = np.stack([np.delete(P, f, axis=1).mean(axis=1) for f in range(4)], axis=1)
    wall, far = fc[m.face_tag == 0], fc[m.face_tag == 1]
    assert len(wall) > 200 and len(far) > 50
    # a body-wall face centroid lies between the body shrunk and grown by 0.3 m
    # about its mid-axis point (spacing at the body), the far faces near 15.6 m
    a_c, tc, a_top, a_min, c0 = W._capsule_geometry()
    for sc, inside in ((1.0 - 0.3 / 2.0, False), (1.0 + 0.3 / 2.0, True)):
        q = wall.copy()
        q[:, 0] = c0 + (q[:, 0] - c0) / sc
        q[:, 1:] /= sc
        assert np.all(W.capsule_inside(q) == inside)
    rf = np.linalg.norm(far - np.array([c0, 0.0, 0.0]), axis=1)
    assert np.all((rf > 0.9 * 15.6) & (rf <= 15.6 * (1 + 1e-12)))
    o = orc.Oracle(s)
    o.init()
    o.step(8, orc.EWMA)
    x, v, I, cell = o.read()
    c = o.counters()
    assert c["stuck"] == 0 and c["injected"] > 0 and c["removed"] > 0 and c["wall"] > 0 and c["lb"] > 0
    assert len(cell) == s.n_particles + c["injected"] - c["removed"]
    assert barycentric(m.nodes, m.tets, cell, x).min() >= -1e-9


def inflow_scenario(U, T=273.0, n=1e20, sides_inflow=(0,), dt=1e-9, F_N=None, n_particles=0, L=1e-3, seed=31):
    """One-hex box: the listed sides are free-stream inflow, the others outflow;
    collisions switched off (tiny molecular diameter)."""
    gas = W.Gas(mass=6.63e-26, d_ref=1e-16, omega=0.81, T_ref=273.0)
    bcs = [dict(kind=W.BC_INFLOW, T=T, U=tuple(U), n=n), dict(kind=W.BC_OUTFLOW, T=T, U=(0.0, 0.0, 0.0), n=0.0)]
    side_bc = [0 if sd in sides_inflow else 1 for sd in range(6)]
    mesh = W.box_sides(1, L, side_bc, bcs)
    return W.Scenario(gas=gas, mesh=mesh, n_particles=n_particles, n_init=n, T_init=T, u_init=(0.0, 0.0, 0.0),
                      F_N=F_N if F_N else n * L ** 3 / 20000, dt=dt, seed=seed, L=L, Kn=1.0, capacity=400000)


def bird_flux(n, T, m, Un):
    """Bird (1994) eq. 4.22, one-sided number flux of a drifting Maxwellian."""
    from scipy.special import erf

    beta = math.sqrt(m / (2 * KB * T))
    s = beta * Un
    return n / (2 * math.sqrt(math.pi) * beta) * (math.exp(-s * s) + math.sqrt(math.pi) * s * (1 + erf(s)))


def test_injection_count_follows_bird_flux():
    """P10: particles injected per step through a face = F A dt / F_N with F
    the one-sided flux of the drifting Maxwellian (Bird eq. 4.22), remainder
    carried: after S steps the count is within one per face of S F A dt / F_N."""
    for Ux in (0.0, 400.0, -250.0):
        sc = inflow_scenario((Ux, 30.0, 0.0), F_N=1e20 * 1e-9 / 3000)
        o = orc.Oracle(sc)
        o.write(np.zeros((0, 3)), np.zeros((0, 3), np.float32), np.zeros(0, np.float32), np.zeros(0, np.int32))
        S = 7
        o.step(S, 0)
        got = o.counters()["injected"]
        # the -x side is split into two triangles of total area L^2; inward normal +x
        exp_count = S * bird_flux(1e20, 273.0, sc.gas.mass, Ux) * sc.L ** 2 * sc.dt / sc.F_N
        assert abs(got - exp_count) <= 2.0, (Ux, got, exp_count)


@pytest.mark.parametrize("Ux", [300.0, -200.0, 0.0])
def test_injected_velocity_distribution(Ux):
    """Injected particles (tiny dt: none has left yet) carry the inflow law:
    normal speed density ~ v exp(-beta^2 (v - U_n)^2) on v > 0 (moments by
    numerical integration), tangential components N(U_t, kT/m)."""
    from scipy.integrate import quad

    T = 273.0
    m = 6.63e-26
    F_N = bird_flux(1e20, T, m, Ux) * 1e-6 * 1e-12 / 20000  # ~20,000 injections in one step
    sc = inflow_scenario((Ux, 40.0, 0.0), T=T, dt=1e-12, F_N=F_N)
    o = orc.Oracle(sc)
    o.write(np.zeros((0, 3)), np.zeros((0, 3), np.float32), np.zeros(0, np.float32), np.zeros(0, np.int32))
    o.step(1, 0)
    x, v, _, cell = o.read()
    n = len(v)
    assert n > 15000
    vx = v[:, 0].astype(np.float64)
    assert np.all(vx > 0)
    beta = math.sqrt(sc.gas.mass / (2 * KB * T))
    g = lambda z: z * math.exp(-(z - beta * Ux) ** 2)
    Z = quad(g, 0, np.inf)[0]
    m1 = quad(lambda z: z * g(z), 0, np.inf)[0] / Z / beta
    m2 = quad(lambda z: z * z * g(z), 0, np.inf)[0] / Z / beta ** 2
    assert abs(vx.mean() - m1) < 4 * vx.std() / math.sqrt(n)
    assert abs((vx ** 2).mean() - m2) < 4 * (vx ** 2).std() / math.sqrt(n)
    sig = math.sqrt(KB * T / sc.gas.mass)
    assert abs(v[:, 1].mean() - 40.0) < 4 * sig / math.sqrt(n)
    assert abs(v[:, 2].mean()) < 4 * sig / math.sqrt(n)
    assert abs(v[:, 1].astype(np.float64).std() / sig - 1) < 4 * 0.71 / math.sqrt(n)
    # positions: on or just inside the inflow side x = -L/2
    assert np.all(x[:, 0] >= -0.5 * sc.L - 1e-15) and np.all(x[:, 0] < -0.5 * sc.L + 1e-8)


def test_open_box_reaches_free_stream():
    """P10: a box with free-stream inflow on all six sides and no collisions
    fills to the free-stream state: number density n, drift U, temperature T."""
    T, n, U = 300.0, 1e20, (150.0, -60.0, 0.0)
    sc = inflow_scenario(U, T=T, n=n, sides_inflow=range(6), dt=5e-8, F_N=n * 1e-9 / 20000)
    o = orc.Oracle(sc)
    o.write(np.zeros((0, 3)), np.zeros((0, 3), np.float32), np.zeros(0, np.float32), np.zeros(0, np.int32))
    o.step(600, 0)  # ~10 box-crossing times: slow molecules need long to fill the box
    o.sample(orc.RESET_CUMUL)
    o.step(400, orc.CUMUL)
    Phi = o.moments(orc.PHI_CUM).sum(axis=0) / 400
    N = Phi[0]
    dens = N * sc.F_N / sc.L ** 3
    u = Phi[1:4] / N
    T_m = sc.gas.mass * (Phi[4:7] / N - u * u).sum() / (3 * KB)
    assert abs(dens / n - 1) < 0.02, dens / n
    assert np.all(np.abs(u - np.array(U)) < 6.0), u
    assert abs(T_m / T - 1) < 0.02, T_m
    c = o.counters()
    assert c["injected"] > 0 and c["removed"] > 0


# ------------------------------------------------------------- DIG coupling (S9-S11)
def face_areas(mesh):
    """Areas of all tet faces from the nodes (face f opposite vertex f)."""
    P = mesh.nodes[mesh.tets]
    A = np.zeros(mesh.tets.shape)
    for f in range(4):
        q = [v for v in range(4) if v != f]
        A[:, f] = 0.5 * np.linalg.norm(np.cross(P[:, q[1]] - P[:, q[0]], P[:, q[2]] - P[:, q[0]]), axis=1)
    return A


def equilibrium_phi(o, scen, rho_scale=None):
    """Exact summation variables of a uniform Maxwellian at rest (per step)."""
    vol = o.mesh_info()["vol"]
    kT_m = KB * scen.T_init / scen.gas.mass
    N = scen.n_init * vol / scen.F_N
    if rho_scale is not None:
        N = N * rho_scale
    phi = np.zeros((len(vol), orc.NPHI))
    phi[:, 0] = N
    phi[:, 4:7] = (N * kT_m)[:, None]
    return phi


def wall_pressure_flux(o, scen, steps):
    """Momentum given to each wall face over `steps` steps by a gas at rest with
    pressure p = n k T: p n A t (energy 0)."""
    mi = o.mesh_info()
    A = face_areas(scen.mesh)
    p = scen.n_init * KB * scen.T_init
    rows = []
    for t in range(len(mi["nbr"])):
        for f in range(4):
            if mi["nbr"][t, f] < 0:
                rows.append([1.0, *(p * mi["normals"][t, f] * A[t, f] * steps * scen.dt), 0.0])
    return np.array(rows)


def test_synthetic_fixed_point_and_identity_recalibration():
    """P12b/P13: a uniform equilibrium at rest with HoT = 0 and walls carrying
    exactly its pressure is a steady solution of the synthetic equations: the
    solve leaves it unchanged, every cell passes the filter, and the
    recalibration leaves every particle bit-for-bit unchanged with no clones
    or deletions: every cell holds exactly the count its density stands for
    (48 equal Kuhn tets x 100 particles), so the number ratio is one."""
    s = box_scenario(nh=2, n_particles=4800, kind=W.BC_DIFFUSE)
    o = orc.Oracle(s, N_m=40, KnD_max=1e9)
    o.write(*W.particles_per_cell(np.random.default_rng(5), s, 100))
    x0, v0, I0, c0 = o.read()
    o.write_moments(orc.PHI_EWMA, equilibrium_phi(o, s))
    o.write_wall_flux(wall_pressure_flux(o, s, 10), 10)
    r = o.couple()
    half, new, flags = o.read_couple(0), o.read_couple(2), o.read_couple(3)
    assert np.all(flags == 1)
    assert np.allclose(half[:, 0], 1.0, rtol=1e-12) and np.allclose(half[:, 4], 1.0, rtol=1e-12)
    assert np.allclose(new, half, rtol=0, atol=1e-10), np.abs(new - half).max()
    assert r["n_cloned"] == 0 and r["n_deleted"] == 0
    x1, v1, I1, c1 = o.read()
    assert np.array_equal(v0, v1) and np.array_equal(x0, x1) and np.array_equal(c0, c1)


def test_synthetic_uniform_stream_is_a_fixed_point():
    """Open boundaries in the synthetic solve: a uniform drifting Maxwellian
    (u = 300 m/s along x, 273 K) in a box whose x = -L/2 side is the same free
    stream (inflow), x = +L/2 an outflow and the four other sides specular
    walls: every flux balances (the slip walls see no normal velocity, the
    inflow face the stream itself, the outflow face the cell), so the solve
    leaves the state unchanged to round-off."""
    n, T, U = 1.677e22, 273.0, 300.0
    bcs = [dict(kind=W.BC_INFLOW, T=T, U=(U, 0.0, 0.0), n=n), dict(kind=W.BC_OUTFLOW, T=T, U=(0.0, 0.0, 0.0), n=0.0),
           dict(kind=W.BC_SPECULAR, T=T, U=(0.0, 0.0, 0.0), n=0.0)]
    mesh = W.box_sides(3, 1e-3, [0, 1, 2, 2, 2, 2], bcs)
    g = W.ARGON
    mu = g.mu_ref() * (T / g.T_ref) ** g.omega
    s = W.Scenario(gas=g, mesh=mesh, n_particles=16200, n_init=n, T_init=T, u_init=(U, 0.0, 0.0),
                   F_N=n * 1e-9 / 16200, dt=0.2 * mu / (n * KB * T), seed=7, L=1e-3, Kn=0.1, capacity=40000)
    o = orc.Oracle(s, N_m=50, KnD_max=1e9)
    o.init()
    vol = o.mesh_info()["vol"]
    kT_m = KB * T / g.mass
    N = n * vol / s.F_N
    phi = np.zeros((len(vol), orc.NPHI))
    phi[:, 0] = N
    phi[:, 1] = N * U
    phi[:, 4] = N * (kT_m + U * U)
    phi[:, 5] = N * kT_m
    phi[:, 6] = N * kT_m
    phi[:, 10] = N * U * (U * U + 5.0 * kT_m)  # <v_x v^2> of a drifting Maxwellian
    o.write_moments(orc.PHI_EWMA, phi)
    r = o.couple()
    half, new, hot = o.read_couple(0), o.read_couple(2), o.read_couple(1)
    assert r["iters"] == 50 and np.all(o.read_couple(3) == 1)
    assert np.abs(hot).max() < 1e-9
    assert np.allclose(new, half, rtol=0, atol=1e-12), np.abs(new - half).max()
    assert abs(half[:, 1].mean() * math.sqrt(kT_m) - U) < 1e-9 * U


def test_synthetic_solve_conserves_mass():
    """The finite-volume update is conservative: walls carry no mass, so the
    total mass sum(rho V) after the solve equals that of M^{k+1/2}."""
    s = W.config_small(seed=4)
    o = orc.Oracle(s, N_m=60, KnD_max=1e9)
    o.init()
    o.step(40, orc.EWMA)
    o.couple()
    vol = o.mesh_info()["vol"]
    half, new = o.read_couple(0), o.read_couple(2)
    assert abs((new[:, 0] * vol).sum() / (half[:, 0] * vol).sum() - 1) < 1e-12


def test_coupling_stable_at_small_knudsen_number():
    """The first coupling of a near-continuum cavity (Kn = 0.001: cells about
    30 mean free paths, sampled stress and heat flux mostly statistical
    noise) converges to eps_m = 1e-6 and to a positive state with the mass
    it started from: the isothermal no-slip wall closure gives the synthetic
    equations a steady solution for any sampled input (a closure by the
    sampled wall fluxes has none unless they balance)."""
    s = W.cavity_scenario(6, 60_000, 0.001, seed=3)
    o = orc.Oracle(s, N_m=2000)
    o.init()
    o.step(200, orc.EWMA)
    r = o.couple()
    new, half = o.read_couple(2), o.read_couple(0)
    vol = o.mesh_info()["vol"]
    assert r["iters"] < 2000 and r["residual"] <= 1e-6
    assert new[:, 0].min() > 0.3 and new[:, 4].min() > 0.3 and np.all(np.isfinite(new))
    assert abs((new[:, 0] * vol).sum() / (half[:, 0] * vol).sum() - 1) < 1e-12


def test_synthetic_fourier_conduction():
    """P12a, Fourier limit of the synthetic equations: a gas at rest between
    diffuse walls at T1 (y = -L/2) and T2 (y = +L/2), specular (slip,
    adiabatic) sides, HoT = 0 (a learned closure that outputs zero): the steady
    solution has zero velocity, uniform pressure and the closed-form
    temperature of steady conduction with kappa ~ mu ~ T^omega, T^(1+omega)
    linear in y, at every cell centroid within 2 % of T2 - T1 (4^3 hexes)."""
    T1, T2, Tw, n = 250.0, 300.0, 273.0, 1.677e22
    wall = lambda T, kind=W.BC_DIFFUSE: dict(kind=kind, T=T, U=(0.0, 0.0, 0.0), n=0.0)
    mesh = W.box_sides(4, 1e-3, [0, 0, 1, 2, 0, 0], [wall(Tw, W.BC_SPECULAR), wall(T1), wall(T2)])
    g = W.ARGON
    mu = g.mu_ref() * (Tw / g.T_ref) ** g.omega
    s = W.Scenario(gas=g, mesh=mesh, n_particles=23040, n_init=n, T_init=Tw, u_init=(0.0, 0.0, 0.0),
                   F_N=n * 1e-9 / 23040, dt=0.2 * mu / (n * KB * Tw), seed=5, L=1e-3, Kn=0.1, capacity=46080)
    o = orc.Oracle(s, N_m=2000, eps_m=1e-12, KnD_max=1e9, closure=1)
    o.init()
    o.step(1, orc.WINDOW)
    o.write_moments(orc.PHI_EWMA, equilibrium_phi(o, s))
    o.closure_set(constant_net(np.zeros(8, np.float32)))
    r = o.couple()
    assert r["n_learned"] == o.n_tets and r["residual"] <= 1e-12 and r["iters"] < 2000, r
    new = o.read_couple(2)
    y = s.mesh.nodes[s.mesh.tets].mean(axis=1)[:, 1] / 1e-3 + 0.5
    w1 = 1.0 + g.omega
    T_exact = (T1 ** w1 + (T2 ** w1 - T1 ** w1) * y) ** (1.0 / w1)
    assert np.abs(new[:, 4] * Tw - T_exact).max() < 0.02 * (T2 - T1)
    assert np.abs(new[:, 1:4]).max() < 1e-9
    p = new[:, 0] * new[:, 4]
    assert np.abs(p / p.mean() - 1.0).max() < 1e-9


def test_reconstruction_layers():
    """Cells failing the cell-Knudsen criterion (Eq. criterion) are rebuilt layer
    by layer from available face neighbours (the paper's local passes): after P
    passes exactly the rejected cells within face-graph distance P of an
    accepted cell are reconstructed; a layer-1 cell's state is the mean of its
    accepted neighbours."""
    import collections

    s = W.cavity_scenario(3, 5000, 0.1, seed=3)
    passes = 2
    o = orc.Oracle(s, N_m=1, KnD_max=1.5, passes=passes)
    o.init()
    cen = s.mesh.nodes[s.mesh.tets].mean(axis=1)
    scale = np.where(cen[:, 0] < -0.1e-3, 0.05, 1.0)  # dilute region: large cell Knudsen number
    o.write_moments(orc.PHI_EWMA, equilibrium_phi(o, s, rho_scale=scale))
    r = o.couple()
    flags = o.read_couple(3)[:, 0]
    own = o.read_couple(4)
    half = o.read_couple(0)
    nbr = o.mesh_info()["nbr"]
    acc = flags == 1
    assert np.array_equal(acc, scale == 1.0)
    dist = np.full(len(flags), 10 ** 9)
    dq = collections.deque()
    for t in np.flatnonzero(acc):
        dist[t] = 0
        dq.append(t)
    while dq:
        t = dq.popleft()
        for nb in nbr[t]:
            if nb >= 0 and dist[nb] > dist[t] + 1:
                dist[nb] = dist[t] + 1
                dq.append(nb)
    assert np.array_equal(flags == 2, (dist >= 1) & (dist <= passes))
    assert r["n_reconstructed"] == int(((dist >= 1) & (dist <= passes)).sum()) > 0
    # the rest of the (connected) mesh is reached by the fill layers
    assert np.array_equal(flags == 3, dist > passes) and (dist > passes).any()
    for t in np.flatnonzero(dist == 1)[:20]:
        nb = [q for q in nbr[t] if q >= 0 and acc[q]]
        assert np.allclose(half[t], own[nb].mean(axis=0), rtol=1e-12)


def test_unreached_cells_take_initial_state():
    """With no accepted cell anywhere, no layer can fill a cell: every cell
    keeps flag 0 and starts the solve from the configuration's initial state
    (density n_init m, drift u_init, temperatures T_init; nondimensional 1,
    u_init / sqrt(k T_init / m), 1, 1) with zero HoT."""
    s = dataclasses.replace(W.cavity_scenario(3, 5000, 0.1, seed=3), u_init=(40.0, -15.0, 0.0))
    o = orc.Oracle(s, N_m=1, KnD_max=1.5, passes=2)
    o.init()
    o.write_moments(orc.PHI_EWMA, equilibrium_phi(o, s, rho_scale=0.05))
    r = o.couple()
    n = o.n_tets
    assert r["n_rejected"] == n and r["n_reconstructed"] == 0
    assert np.all(o.read_couple(3) == 0)
    c0 = math.sqrt(KB * s.T_init / s.gas.mass)
    want = np.array([1.0, 40.0 / c0, -15.0 / c0, 0.0, 1.0, 1.0])
    assert np.array_equal(o.read_couple(0), np.broadcast_to(want, (n, 6)))
    assert np.all(o.read_couple(1) == 0.0)


@pytest.mark.parametrize("recon", [0, 1])
def test_reconstruction_mean_arithmetic_or_logarithmic(recon):
    """A layer-1 cell with accepted neighbours of different density, drift and
    temperature: every neighbour has the same weight (Sec. 3.2); recon = 0 takes
    the arithmetic mean of every component, recon = 1 the geometric mean
    exp(mean ln) of density and temperatures (the log-mean reconstruction of
    Sec. 6) and the arithmetic mean of velocity and HoT.  By the AM-GM
    inequality the two differ wherever the neighbours differ."""
    s = W.cavity_scenario(3, 5000, 0.1, seed=3)
    o = orc.Oracle(s, N_m=1, KnD_max=1.5, passes=1, recon=recon)
    o.init()
    n = len(s.mesh.tets)
    rng = np.random.default_rng(7)
    acc_cell = rng.random(n) >= 0.3  # scattered rejected cells: many have several accepted neighbours
    scale = np.where(acc_cell, rng.uniform(0.6, 1.6, n), 0.05)
    phi = equilibrium_phi(o, s, rho_scale=scale)
    kT_m = KB * s.T_init / s.gas.mass
    Ts = rng.uniform(0.7, 1.4, n)
    ux = rng.uniform(-30.0, 30.0, n)
    N = phi[:, 0]
    phi[:, 1] = N * ux
    phi[:, 4] = N * (kT_m * Ts + ux * ux)
    phi[:, 5] = N * kT_m * Ts
    phi[:, 6] = N * kT_m * Ts
    o.write_moments(orc.PHI_EWMA, phi)
    o.couple()
    flags = o.read_couple(3)[:, 0]
    own, half, hot = o.read_couple(4), o.read_couple(0), o.read_couple(1)
    nbr = o.mesh_info()["nbr"]
    acc = flags == 1
    assert np.array_equal(acc, acc_cell)
    layer1 = [t for t in np.flatnonzero(flags == 2) if sum(1 for q in nbr[t] if q >= 0 and acc[q]) >= 2]
    assert len(layer1) > 10
    gap = 0.0
    for t in layer1:
        nb = [q for q in nbr[t] if q >= 0 and acc[q]]
        am = own[nb].mean(axis=0)
        want = am.copy()
        if recon == 1:
            for q in (0, 4, 5):
                want[q] = math.exp(np.log(own[nb, q]).mean())
        assert np.allclose(half[t], want, rtol=1e-12, atol=1e-15), (t, half[t], want)
        assert np.allclose(hot[t], hot[nb].mean(axis=0), rtol=1e-12, atol=1e-15)
        gap = max(gap, abs(am[0] - math.exp(np.log(own[nb, 0]).mean())) / am[0])
    assert gap > 1e-3  # the neighbours differ enough to tell the two means apart


@pytest.mark.parametrize("local_acc", [0, 1])
def test_local_accumulation_state(local_acc):
    """Sec. 3.2: a cell rejected by the filter enters a local accumulation state in
    which its samples are no longer forgotten.  With n_a = 10 and 20 samples
    before the coupling, a rejected cell's average afterwards is the running
    mean (10 E_0 + sum of the K new steps)/(10 + K) and its weight 10 + K; an
    accepted cell keeps the moving average E <- 0.9 E + 0.1 inst; after a
    coupling that accepts every cell all weights return to 0.  Without the
    state every cell keeps the moving average."""
    s = W.cavity_scenario(3, 5000, 0.1, seed=3)
    o = orc.Oracle(s, N_m=1, KnD_max=1.5, passes=2, n_a=10, local_acc=local_acc)
    o.init()
    o.step(20, orc.EWMA)
    cen = s.mesh.nodes[s.mesh.tets].mean(axis=1)
    dilute = cen[:, 0] < -0.1e-3
    o.write_moments(orc.PHI_EWMA, equilibrium_phi(o, s, rho_scale=np.where(dilute, 0.05, 1.0)))
    o.couple()
    rej = o.read_couple(3)[:, 0] != 1
    assert np.array_equal(rej, dilute)
    w0 = o.read_couple(5)[:, 0]
    assert np.array_equal(w0, np.where(rej, 10.0, 0.0) if local_acc else np.zeros(len(rej)))
    E0 = o.moments(orc.PHI_EWMA)
    K = 15
    inst = []
    for _ in range(K):
        o.step(1, orc.EWMA)
        inst.append(o.moments(orc.PHI_INST))
    E = o.moments(orc.PHI_EWMA)
    run = (10.0 * E0 + np.sum(inst, axis=0)) / (10.0 + K)
    mov = E0.copy()
    for ph in inst:
        mov = 0.9 * mov + 0.1 * ph
    want = np.where(rej[:, None], run, mov) if local_acc else mov
    assert np.allclose(E, want, rtol=1e-12, atol=1e-12 * np.abs(want).max())
    assert np.abs(run - mov)[rej].max() > 1e-3 * np.abs(mov).max()  # the two laws differ here
    w1 = o.read_couple(5)[:, 0]
    assert np.array_equal(w1, np.where(rej, 10.0 + K, 0.0) if local_acc else np.zeros(len(rej)))
    o.write_moments(orc.PHI_EWMA, equilibrium_phi(o, s))
    o.couple()
    assert np.all(o.read_couple(3)[:, 0] == 1)
    assert np.all(o.read_couple(5)[:, 0] == 0.0)


def test_filter_threshold_sweep_nests_rejections():
    """A sweep of Kn_D,max (the stability study's threshold of Eq. criterion): the
    cells rejected at a larger threshold are a subset of those rejected at a
    smaller one, a threshold above every cell's lambda_c/d_c rejects only the
    cells without a temperature (fewer than two particles on average), and the
    counts follow lambda_c/d_c computed here from the sampled state."""
    s = W.cavity_scenario(3, 5000, 0.1, seed=3)
    cen = s.mesh.nodes[s.mesh.tets].mean(axis=1)
    scale = np.exp(np.interp(cen[:, 0], [-0.5e-3, 0.5e-3], [math.log(0.03), 0.0]))
    prev = None
    for kmax in (0.3, 0.6, 1.2, 2.4, 1e9):
        o = orc.Oracle(s, N_m=1, KnD_max=kmax, passes=1)
        o.init()
        o.write_moments(orc.PHI_EWMA, equilibrium_phi(o, s, rho_scale=scale))
        r = o.couple()
        rej = o.read_couple(3)[:, 0] != 1
        own = o.read_couple(4)
        vol = o.mesh_info()["vol"] / s.L ** 3
        dc = 2.0 * np.cbrt(3.0 * vol / (4.0 * math.pi))
        lam = s.Kn * own[:, 4] ** (s.gas.omega - 0.5) / own[:, 0]
        nbar = equilibrium_phi(o, s, rho_scale=scale)[:, 0]
        want = (lam / dc > kmax) | (nbar < 2.0)
        assert np.array_equal(rej, want), kmax
        assert r["n_rejected"] == int(want.sum())
        if prev is not None:
            assert np.all(rej <= prev)  # nested: rejected now => rejected at the smaller threshold
        prev = rej
    assert prev.sum() == int((nbar < 2.0).sum())


def test_recalibration_number_statistics():
    """S11 number adjustment: each particle of an accepted cell is deleted with
    probability 1 - r or cloned with probability r - 1, r = rho^{k+1}/rho_N
    where rho_N = m F_N N_c / V is the density of the cell's N_c particles;
    the total change matches sum N_c (r_c - 1) within 4 standard deviations and
    the count bookkeeping is exact."""
    s = W.config_small(seed=9)
    o = orc.Oracle(s, N_m=80, KnD_max=1e9)
    o.init()
    o.step(60, orc.EWMA)
    N0 = np.bincount(o.read()[3], minlength=o.n_tets)
    r = o.couple()
    own, new, flags = o.read_couple(4), o.read_couple(2), o.read_couple(3)[:, 0]
    vol = o.mesh_info()["vol"]
    rho_N = s.gas.mass * s.F_N * N0 / vol / (s.gas.mass * s.n_init)
    rr = np.clip(new[:, 0] / np.maximum(rho_N, 1e-300), 0.5, 2.0)
    sel = flags == 1
    exp = (N0[sel] * (rr[sel] - 1)).sum()
    var = (N0[sel] * np.abs(rr[sel] - 1) * (1 - np.abs(rr[sel] - 1))).sum()
    got = r["n_cloned"] - r["n_deleted"]
    assert abs(got - exp) < 4 * math.sqrt(var) + 1, (got, exp, var)
    assert len(o.read()[3]) == N0.sum() + r["n_cloned"] - r["n_deleted"]


# ----------------------------------------------------------- learned closure (S12/S13)
def test_bf16_round_to_nearest_even():
    """BF16 = FP32 with 8 significant bits, round to nearest, ties to even."""
    assert orc.bf16(1.0 + 2 ** -8) == 1.0  # tie between 1 and 1+2^-7: even
    assert orc.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6  # tie: even mantissa
    assert orc.bf16(1.0 + 2 ** -8 + 2 ** -12) == 1.0 + 2 ** -7
    assert orc.bf16(-3.0) == -3.0 and orc.bf16(0.0) == 0.0


def test_mlp_forward_composes_gelu():
    """A network that routes one input through one unit per layer computes
    GELU(GELU(GELU(x))) with GELU(z) = z (1 + erf(z/sqrt2))/2 (closed form)."""
    from scipy.special import erf

    p = np.zeros(orc.mlp_nparam(), np.float32)
    o = 0
    p[o + 0] = 1.0  # W1[0][0]
    o += 64 * 13 + 64
    p[o + 0] = 1.0  # W2[0][0]
    o += 64 * 64 + 64
    p[o + 0] = 1.0  # W3[0][0]
    o += 64 * 64 + 64
    p[o + 0] = 1.0  # W4[0][0]
    g = lambda z: 0.5 * z * (1 + erf(z / math.sqrt(2)))
    X = np.zeros((5, 13), np.float32)
    X[:, 0] = [-2.0, -0.5, 0.0, 0.7, 3.0]
    Y = orc.mlp_forward(p, X, bf16=False)
    assert np.allclose(Y[:, 0], g(g(g(X[:, 0].astype(np.float64)))), rtol=1e-12, atol=1e-15)
    assert np.all(Y[:, 1:] == 0)


def test_mlp_gradient_matches_finite_differences():
    """P14: backpropagated gradient of the mean-square loss equals central
    finite differences of the FP64 network (no BF16 rounding) to 1e-6."""
    rng = np.random.default_rng(5)
    p = orc.mlp_init(7)
    p += (0.05 * rng.standard_normal(len(p))).astype(np.float32)  # nonzero biases too
    X = rng.standard_normal((12, 13)).astype(np.float32)
    T = rng.standard_normal((12, 8)).astype(np.float32)
    loss, g = orc.mlp_grad(p, X, T, bf16=False)
    idx = list(rng.choice(len(p), 40, replace=False)) + [len(p) - 1, len(p) - 9, 64 * 13 + 3]
    for i in idx:
        h = 3e-5 * max(1.0, abs(float(p[i])))
        pp = p.astype(np.float64)

        def L(delta):
            q = p.copy()
            q[i] = np.float32(pp[i] + delta)
            d = float(q[i]) - pp[i]
            return orc.mlp_grad(q, X, T, bf16=False)[0], d

        lp, dp = L(h)
        lm, dm = L(-h)
        fd = (lp - lm) / (dp - dm)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-10, (i, fd, g[i])


def test_adam_first_step_closed_form():
    """Adam's first step moves every parameter by lr * g / (|g| + eps) (the
    bias-corrected moments equal g and g^2), i.e. lr * sign(g)."""
    p = np.ones(orc.mlp_nparam(), np.float32)
    g = np.linspace(-2, 3, len(p))
    g[len(g) // 2] = 0.5
    m = np.zeros(len(p))
    v = np.zeros(len(p))
    orc.adam(p, m, v, g, 1, lr=1e-3)
    exp = 1.0 - 1e-3 * g / (np.abs(g) + 1e-8)
    assert np.allclose(p, exp.astype(np.float32), rtol=0, atol=2e-7)


# ------------------------------------------------------- learned closure inputs
def stressed_phi(o, scen, sigma, q, rho_scale=1.0, T=None):
    """Exact per-step summation variables of a state at rest with density
    rho_scale * m n_init, temperature T, traceless stress sigma (xx, yy, zz,
    xy, xz, yz) and heat flux q: <c_i c_j> = (kT/m) delta_ij + sigma_ij / rho,
    <c_i c^2> = 2 q_i / rho."""
    vol = o.mesh_info()["vol"]
    T = scen.T_init if T is None else T
    m = scen.gas.mass
    rho = rho_scale * m * scen.n_init
    N = scen.n_init * rho_scale * vol / scen.F_N
    phi = np.zeros((len(vol), orc.NPHI))
    phi[:, 0] = N
    for k, s in enumerate(sigma):
        phi[:, 4 + k] = N * ((KB * T / m if k < 3 else 0.0) + s / rho)
    for i in range(3):
        phi[:, 10 + i] = N * 2.0 * q[i] / rho
    return phi


SIG = np.array([0.04, -0.015, -0.025, 0.01, -0.02, 0.03])  # / p
QF = np.array([0.02, -0.01, 0.005])  # / (rho (kT/m)^{3/2})


def test_closure_features_closed_form():
    """S12 inputs of a uniform state at rest in a box whose diffuse walls are
    at the gas temperature (all gradients vanish, so the HoT is the sampled
    stress and heat flux): rho / (m n0), u / c0, T / T0, the traceless stress
    (xx, yy, xy, xz, yz) over p = rho k T / m and the heat flux over
    rho (k T / m)^{3/2}; an empty cell gives a zero row."""
    s = box_scenario(nh=2, n_particles=3000, kind=W.BC_DIFFUSE)
    o = orc.Oracle(s)
    o.init()
    o.step(1, orc.WINDOW)
    rs = 1.3
    p = rs * s.n_init * KB * s.T_init
    rho = rs * s.gas.mass * s.n_init
    kTm = KB * s.T_init / s.gas.mass
    phi = stressed_phi(o, s, SIG * p, QF * rho * kTm ** 1.5, rho_scale=rs)
    phi[3] = 0.0  # an empty cell
    o.write_moments(orc.PHI_WINDOW, phi)
    X = o.closure_features(orc.PHI_WINDOW).astype(np.float64)
    exp = np.concatenate([[rs, 0, 0, 0, 1.0], SIG[[0, 1, 3, 4, 5]], QF])
    # the empty cell's zero temperature enters its face neighbours' gradients
    nbr = o.mesh_info()["nbr"]
    ok = np.all(nbr != 3, axis=1) & (np.arange(len(X)) != 3)
    assert ok.sum() >= len(X) - 5
    assert np.all(X[3] == 0)
    assert np.allclose(X[ok], exp[None, :], rtol=2e-6, atol=1e-7), np.abs(X[ok] - exp).max(axis=0)


def test_closure_targets_normalised_by_input_row():
    """S13 targets: the HoT of the long-time (cumulative) average of cell
    r mod n divided by rho T (stress) and rho T^{3/2} (heat flux) of input row
    r, for a stack of input rows spanning several windows; rows with zero
    density or temperature are zero."""
    s = box_scenario(nh=1, n_particles=2000, kind=W.BC_DIFFUSE)
    o = orc.Oracle(s)
    o.init()
    o.step(1, orc.WINDOW | orc.CUMUL)
    p = s.n_init * KB * s.T_init
    rho = s.gas.mass * s.n_init
    kTm = KB * s.T_init / s.gas.mass
    o.write_moments(orc.PHI_CUM, stressed_phi(o, s, SIG * p, QF * rho * kTm ** 1.5))
    n = o.n_tets
    rng = np.random.default_rng(3)
    X = rng.uniform(0.5, 2.0, (3 * n, 13)).astype(np.float32)
    X[n + 2, 0] = 0.0
    X[2 * n + 1, 4] = 0.0
    Y = o.closure_targets(orc.PHI_CUM, X).astype(np.float64)
    x0, x4 = X[:, 0].astype(np.float64), X[:, 4].astype(np.float64)
    with np.errstate(divide="ignore"):
        exp = np.concatenate([np.outer(1 / (x0 * x4), SIG[[0, 1, 3, 4, 5]]), np.outer(1 / (x0 * x4 ** 1.5), QF)],
                             axis=1)
    bad = np.zeros(3 * n, bool)
    bad[[n + 2, 2 * n + 1]] = True
    exp[bad] = 0.0
    assert np.allclose(Y, exp, rtol=2e-6, atol=1e-8), np.abs(Y - exp).max()


def constant_net(y):
    """Parameters of the network whose output is the constant y: zero weights,
    zero hidden biases, output bias y (GELU(0) = 0)."""
    p = np.zeros(orc.mlp_nparam(), np.float32)
    p[-8:] = y
    return p


def closure_case(closure, y, empty=()):
    s = box_scenario(nh=2, n_particles=3000, kind=W.BC_DIFFUSE)
    o = orc.Oracle(s, N_m=5, KnD_max=1e9, closure=closure)
    o.init()
    o.step(1, orc.WINDOW)
    phi_w = stressed_phi(o, s, 0 * SIG, 0 * QF, rho_scale=1.3, T=1.2 * s.T_init)
    phi_w[list(empty)] = 0.0
    o.write_moments(orc.PHI_WINDOW, phi_w)
    p = s.n_init * KB * s.T_init
    o.write_moments(orc.PHI_EWMA, stressed_phi(o, s, 0.5 * SIG * p, 0 * QF))
    o.write_wall_flux(wall_pressure_flux(o, s, 10), 10)
    o.closure_set(constant_net(y))
    r = o.couple()
    return r, o.read_couple(1)


def test_closure_replaces_hot_in_coupling():
    """S12 in the coupling: with a network that outputs the constant y the HoT
    of each cell is y de-normalised by the window's density and temperature
    (sigma_zz = -(sigma_xx + sigma_yy)); cells with an empty window, and every
    cell when a component of y exceeds the limit, keep the sampled HoT."""
    y = np.array([0.05, -0.02, 0.01, 0.03, -0.04, 0.02, 0.01, -0.03], np.float32)
    r0, H0 = closure_case(0, y, empty=(0, 5))
    r1, H1 = closure_case(1, y, empty=(0, 5))
    n = len(H1)
    assert r0["n_learned"] == 0 and r1["n_learned"] == n - 2
    rho, T = 1.3, 1.2
    yd = y.astype(np.float64)
    s, qn = rho * T, rho * T * math.sqrt(T)
    exp = np.array([yd[0] * s, yd[1] * s, 0.0, yd[2] * s, yd[3] * s, yd[4] * s, *(yd[5:] * qn), 0, 0, 0])
    exp[2] = -(exp[0] + exp[1])
    learned = np.ones(n, bool)
    learned[[0, 5]] = False
    assert np.allclose(H1[learned], exp[None, :], rtol=1e-12, atol=1e-15)
    assert np.array_equal(H1[~learned], H0[~learned])
    y_bad = y.copy()
    y_bad[3] = 4.5  # beyond the plausibility limit
    r2, H2 = closure_case(1, y_bad)
    assert r2["n_learned"] == 0 and np.array_equal(H2, closure_case(0, y_bad)[1])
