"""Pins of the oracle's synthetic equations (paper Sec. 2.2: Eq. macro with the
NSF relations and Eq. synthetic_closure) and of the VHS mean free path,
against things fixed outside the oracle: exactness of least squares on linear
fields, the Navier-Stokes-Fourier constitutive relations written from kinetic
theory (Bird 1994 eq. 4.62 viscosity, Eucken's monatomic conductivity), a
manufactured solution of the steady equations on three meshes, and Bird's
mean free path (eq. 4.65).  No GPU needed.
"""
import math

import numpy as np
import pytest

from oracle import orc
from paper_2607_08195_gb300 import workload as W

KB = W.K_B


def wall(T, U=(0.0, 0.0, 0.0), kind=W.BC_DIFFUSE):
    return dict(kind=kind, T=T, U=tuple(U), n=0.0)


def solver_scenario(mesh, Kn=0.05, T0=273.0, gas=W.ARGON, L=1e-3):
    """A context for the synthetic equations alone: the number density follows
    from Kn by the paper's definition (Kn = mu0 / (p0 L) sqrt(pi R T0 / 2))."""
    mu0 = gas.mu_ref() * (T0 / gas.T_ref) ** gas.omega
    R = KB / gas.mass
    p0 = mu0 / (Kn * L) * math.sqrt(math.pi * R * T0 / 2.0)
    n0 = p0 / (KB * T0)
    return W.Scenario(gas=gas, mesh=mesh, n_particles=1000, n_init=n0, T_init=T0, u_init=(0.0, 0.0, 0.0),
                      F_N=n0 * L ** 3 / 1000, dt=0.2 * mu0 / p0, seed=1, L=L, Kn=Kn, capacity=2000)


def centroids(mesh, L):
    return mesh.nodes[mesh.tets].mean(axis=1) / L


def interior(o):
    return np.all(o.mesh_info()["nbr"] >= 0, axis=1)


# --------------------------------------------------------------- gradients
def test_least_squares_gradients_exact_for_linear_fields():
    """The least-squares gradient of the solve (the gradient minimising the
    squared misfit of a linear model over the four faces) reproduces every
    linear field exactly: an arbitrary linear u and T at every cell with four
    neighbours, and, for fields linear in y, also at the cells whose boundary
    faces lie on diffuse walls at y = +-L/2 that carry the field's own wall
    velocity and temperature (the face centroid is then on the linear field)."""
    L, T0 = 1e-3, 273.0
    rng = np.random.default_rng(0)
    A = rng.uniform(-0.4, 0.4, (3, 3))  # du_i/dx_j (nondimensional)
    b = rng.uniform(-0.2, 0.2, 3)
    gT = rng.uniform(-0.3, 0.3, 3)
    mesh = W.box_sides(4, L, [0, 0, 0, 0, 0, 0], [wall(T0)])
    s = solver_scenario(mesh)
    o = orc.Oracle(s)
    x = centroids(mesh, L)
    prim = np.zeros((len(x), 6))
    prim[:, 0] = 1.0 + 0.1 * x[:, 0]
    prim[:, 1:4] = x @ A.T + b
    prim[:, 4] = 1.0 + x @ gT
    prim[:, 5] = prim[:, 4]
    G = o.gradients(prim).reshape(-1, 5, 3)
    inn = interior(o)
    assert inn.sum() > 100
    assert np.abs(G[inn, 0:3, :] - A[None]).max() < 1e-12
    assert np.abs(G[inn, 3, :] - gT[None]).max() < 1e-12
    assert np.abs(G[inn, 4, :] - gT[None]).max() < 1e-12

    # fields linear in y: walls y = -L/2 (bc 1) and y = +L/2 (bc 2) carry the
    # field's values; the x and z sides are diffuse walls at rest (bc 0)
    c0 = math.sqrt(KB * T0 / s.gas.mass)
    a, u0, tg = np.array([0.3, -0.2, 0.1]), np.array([0.05, 0.0, -0.04]), 0.25
    lo, hi = wall(T0 * (1 - 0.5 * tg), c0 * (u0 - 0.5 * a)), wall(T0 * (1 + 0.5 * tg), c0 * (u0 + 0.5 * a))
    mesh = W.box_sides(4, L, [0, 0, 1, 2, 0, 0], [wall(T0), lo, hi])
    o = orc.Oracle(solver_scenario(mesh))
    x = centroids(mesh, L)
    prim[:, 1:4] = u0 + x[:, 1:2] * a
    prim[:, 4] = 1.0 + tg * x[:, 1]
    prim[:, 5] = prim[:, 4]
    G = o.gradients(prim).reshape(-1, 5, 3)
    mi = o.mesh_info()
    side = W.boundary_side(mesh.nodes, mesh.tets, L)
    ywall = (mi["nbr"] >= 0) | (side == 2) | (side == 3)
    cells = np.all(ywall, axis=1) & ~interior(o)
    assert cells.sum() > 10
    exact = np.zeros((5, 3))
    exact[0:3, 1] = a
    exact[3:5, 1] = tg
    assert np.abs(G[cells] - exact[None]).max() < 1e-12
    assert np.abs(G[interior(o)] - exact[None]).max() < 1e-12


# --------------------------------------------------------------- NSF relations
@pytest.mark.parametrize("case", ["shear", "uniaxial", "isotropic", "general"])
def test_nsf_stress_and_heat_flux(case):
    """The NSF relations of the solve (Sec. 2.2) in SI units: stress
    sigma = -mu(T) (grad u + grad u^T - 2/3 div u I) and heat flux
    q = -(15/4) (k/m) mu(T) grad T, with mu(T) the VHS viscosity of Bird (1994)
    eq. 4.62 at the cell temperature and the monatomic (Eucken) conductivity.
    A linear shear has only the off-diagonal stress mu du/dy; a uniaxial
    dilatation du_x/dx = d gives sigma_xx = -4/3 mu d and sigma_yy = sigma_zz
    = 2/3 mu d; an isotropic dilatation has no NSF stress at all."""
    L, T0, Kn = 1e-3, 273.0, 0.05
    gas = W.ARGON
    mesh = W.box_sides(3, L, [0] * 6, [wall(T0)])
    s = solver_scenario(mesh, Kn=Kn, T0=T0, gas=gas, L=L)
    o = orc.Oracle(s)
    x = centroids(mesh, L)
    A = {"shear": np.array([[0, 0.3, 0], [0, 0, 0], [0, 0, 0]]),
         "uniaxial": np.diag([0.25, 0.0, 0.0]),
         "isotropic": np.eye(3) * 0.2,
         "general": np.random.default_rng(3).uniform(-0.3, 0.3, (3, 3))}[case]
    gT = np.array([0.1, -0.2, 0.15])
    prim = np.zeros((len(x), 6))
    prim[:, 0] = 1.2
    prim[:, 1:4] = x @ A.T
    prim[:, 4] = 1.1 + x @ gT
    prim[:, 5] = prim[:, 4]
    G = o.gradients(prim)
    out = o.nsf(prim, G)
    inn = interior(o)
    # SI: velocity scale c0, lengths L, temperature T0, density m n0
    c0 = math.sqrt(KB * T0 / gas.mass)
    rho0 = gas.mass * s.n_init
    T = prim[inn, 4] * T0
    mu = gas.mu_ref() * (T / gas.T_ref) ** gas.omega
    D = A * c0 / L  # du_i/dx_j, 1/s
    sig = -mu[:, None, None] * (D + D.T - 2.0 / 3.0 * np.trace(D) * np.eye(3))[None]
    q = -(15.0 / 4.0) * (KB / gas.mass) * mu[:, None] * (gT * T0 / L)[None]
    ss, qs = rho0 * c0 ** 2, rho0 * c0 ** 3
    got = out[inn, :6] * ss
    want = np.stack([sig[:, 0, 0], sig[:, 1, 1], sig[:, 2, 2], sig[:, 0, 1], sig[:, 0, 2], sig[:, 1, 2]], axis=1)
    scale = np.abs(want).max() + mu.max() * np.abs(D).max()
    assert np.abs(got - want).max() <= 1e-11 * scale
    assert np.abs(out[inn, 6:9] * qs - q).max() <= 1e-11 * np.abs(q).max()
    assert np.all(out[:, 9:12] == 0.0)  # monatomic: no rotational heat flux
    if case == "isotropic":
        assert np.abs(got).max() <= 1e-12 * mu.max() * np.abs(D).max()
    if case == "uniaxial":
        d = D[0, 0]
        assert np.allclose(got[:, 0], -4.0 / 3.0 * mu * d, rtol=1e-11)
        assert np.allclose(got[:, 1], 2.0 / 3.0 * mu * d, rtol=1e-11)


# --------------------------------------------------------- manufactured solution
def _mms_fields(Kn, omega):
    """Exact steady state (nondimensional, monatomic) and the volume source
    that makes it one: S = div F with F the conservative fluxes of the
    compressible Navier-Stokes-Fourier equations (Eq. macro with the NSF
    relations), velocity zero and temperature one on every wall."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z", real=True)
    X = (x, y, z)
    pi = sp.pi
    phi = sp.cos(pi * x) * sp.cos(pi * y) * sp.cos(pi * z)
    rho = 1 + sp.Rational(15, 100) * sp.sin(pi * x) * sp.cos(pi * (y - sp.Rational(1, 5))) + sp.Rational(1, 10) * z
    u = [sp.Rational(3, 10) * phi * (1 + y / 2),
         -sp.Rational(1, 5) * phi * sp.sin(pi * x + sp.Rational(3, 10)),
         sp.Rational(3, 20) * phi * sp.cos(pi * (y - sp.Rational(1, 5)))]
    T = 1 + sp.Rational(1, 10) * phi * (1 + x / 2)
    mu = Kn * sp.sqrt(2 / pi) * T ** omega
    kap = sp.Rational(15, 4) * mu
    div = sum(sp.diff(u[i], X[i]) for i in range(3))
    sig = [[-mu * (sp.diff(u[i], X[j]) + sp.diff(u[j], X[i]) - sp.Rational(2, 3) * div * (1 if i == j else 0))
            for j in range(3)] for i in range(3)]
    q = [-kap * sp.diff(T, X[j]) for j in range(3)]
    p = rho * T
    E = rho * (sp.Rational(3, 2) * T + (u[0] ** 2 + u[1] ** 2 + u[2] ** 2) / 2)
    F = [[rho * u[j] for j in range(3)]]
    for i in range(3):
        F.append([rho * u[i] * u[j] + p * (1 if i == j else 0) + sig[i][j] for j in range(3)])
    F.append([(E + p) * u[j] + sum(sig[i][j] * u[i] for i in range(3)) + q[j] for j in range(3)])
    S = [sum(sp.diff(F[k][j], X[j]) for j in range(3)) for k in range(5)]
    f = sp.lambdify(X, [rho, *u, T], "numpy")
    g = sp.lambdify(X, S, "numpy")

    def exact(c):
        r = f(c[:, 0], c[:, 1], c[:, 2])
        return np.stack([np.broadcast_to(np.asarray(v, float), c[:, 0].shape) for v in r], axis=1)

    def source(c):
        r = g(c[:, 0], c[:, 1], c[:, 2])
        return np.stack([np.broadcast_to(np.asarray(v, float), c[:, 0].shape) for v in r], axis=1)

    return exact, source


def _tet_average(fn, mesh, L):
    """Cell averages by the degree-3 five-point rule on each tetrahedron."""
    P = mesh.nodes[mesh.tets] / L  # [n, 4, 3]
    cen = P.mean(axis=1)
    acc = -0.8 * fn(cen)
    for v in range(4):
        pt = (P.sum(axis=1) - P[:, v]) / 6.0 + 0.5 * P[:, v]
        acc += 0.45 * fn(pt)
    return acc


def test_manufactured_solution_converges():
    """P12c: with the source S = div F(M*) of a smooth steady state M* with
    flow (Mach up to 0.3, non-zero divergence, density and temperature
    gradients), the solve's steady state approaches M* as the mesh is refined
    (3^3, 6^3, 12^3 hexahedra): the error halves at least roughly with each
    halving of h (the scheme is first order: piecewise-constant states with
    Rusanov dissipation).  This pins the inviscid flux, the viscous flux from
    the face-averaged NSF stress and heat flux, the work of the stress, and the
    diffuse walls (no slip, isothermal, velocity zero and temperature one on
    every wall of M*).  A dropped or misweighted term leaves an O(1) error
    that does not shrink."""
    L, T0, Kn = 1e-3, 273.0, 0.05
    omega = W.ARGON.omega
    exact, source = _mms_fields(Kn, omega)
    errs = []
    for nh in (3, 6, 12):
        mesh = W.box_sides(nh, L, [0] * 6, [wall(T0)])
        o = orc.Oracle(solver_scenario(mesh, Kn=Kn, T0=T0, L=L), N_m=400_000, eps_m=1e-10)
        vol = o.mesh_info()["vol"] / L ** 3
        ex = _tet_average(exact, mesh, L)
        half = np.zeros((len(vol), 6))
        half[:, :5] = ex
        half[:, 5] = ex[:, 4]
        src = np.zeros((len(vol), 6))
        src[:, :5] = _tet_average(source, mesh, L)
        # a closed box has a steady state only if the sources add no mass: the
        # exact integral of div(rho u) is zero, its quadrature O(h^2)
        src[:, 0] -= (vol * src[:, 0]).sum() / vol.sum()
        out, it, res = o.synthetic_solve(half, src=src)
        assert res < 1e-10, (nh, it, res)
        e = np.sqrt((vol[:, None] * (out[:, :5] - ex) ** 2).sum(axis=0) / vol.sum())
        errs.append(e)
    errs = np.array(errs)  # [mesh, component]
    tot = np.sqrt((errs ** 2).sum(axis=1))
    rate = np.log2(tot[:-1] / tot[1:])
    assert np.all(rate > 0.8), (tot, rate)
    # velocity, the quantity the stress terms act on, converges as well
    uerr = np.sqrt((errs[:, 1:4] ** 2).sum(axis=1))
    assert np.all(np.log2(uerr[:-1] / uerr[1:]) > 0.8), uerr
    assert tot[-1] < 0.02


# ------------------------------------------------------------ safeguard
def _seeded_cavity_inputs():
    s = W.cavity_scenario(6, 60_000, 0.01, seed=23)
    o = orc.Oracle(s, N_m=1, passes=3, KnD_max=1.0)
    o.init()
    o.step(40, orc.EWMA)
    o.couple()
    return s, o.read_couple(0), o.read_couple(1)


def test_safeguard_returns_best_iterate_and_recovers():
    """An unstable pseudo-time step (CFL 48, no acceleration: explicit local
    steps are stable only near CFL 1): every iterate of the first 20 is worse
    than the initial state, so the solve returns M^{k+1/2} itself with
    residual 1; given iterations, the CFL halvings on divergence make it
    converge to the same fixed point as the stable step (a steady solution does
    not depend on the pseudo-time step), and the accelerated solve at CFL 12
    as well."""
    s, half, hot = _seeded_cavity_inputs()
    out, it, res = orc.Oracle(s, N_m=20, eps_m=1e-12, cfl=48.0, aa_m=0).synthetic_solve(half, hot=hot)
    assert it == 20 and res == 1.0
    assert np.allclose(out, half, rtol=1e-13, atol=1e-15)
    ref, it0, r0 = orc.Oracle(s, N_m=4000, eps_m=1e-12).synthetic_solve(half, hot=hot)
    assert r0 <= 1e-12 and it0 < 4000
    sc = np.abs(ref).max(axis=0)
    for cfl, m in ((48.0, 0), (12.0, 20)):
        new, it, res = orc.Oracle(s, N_m=4000, eps_m=1e-12, cfl=cfl, aa_m=m).synthetic_solve(half, hot=hot)
        assert res <= 1e-12 and it < 4000, (cfl, m, it, res)
        assert np.all(np.abs(new - ref) <= 1e-9 * sc), (cfl, m, np.abs(new - ref).max(axis=0))


# -------------------------------------------------------------- mean free path
def test_vhs_mean_free_path():
    """P2: in an equilibrium VHS gas the mean distance a molecule flies between
    collisions (total distance flown / molecule collisions, two per collision)
    is lambda = 1 / (sqrt(2) pi d^2 n (T_ref/T)^(omega - 1/2)) (Bird 1994
    eq. 4.65); at 400 K, away from T_ref = 273 K, so that the temperature
    factor counts.  Within 4 standard errors of the collision count."""
    from tests.test_oracle_pins import box_scenario

    T = 400.0
    s = box_scenario(nh=1, n_particles=6000, T=T)
    g = s.gas
    o = orc.Oracle(s)
    o.init()
    o.step(20, 0)
    c0 = o.counters()["coll"]
    dist = 0.0
    nsteps = 200
    for _ in range(nsteps):
        # a step moves the molecules, then collides them: the speeds read
        # before a step are the ones flown during its move (specular walls
        # keep each speed)
        _, v, _, _ = o.read()
        dist += np.linalg.norm(v.astype(np.float64), axis=1).sum() * s.dt
        o.step(1, 0)
    coll = o.counters()["coll"] - c0
    n = s.n_init
    lam = 1.0 / (math.sqrt(2.0) * math.pi * g.d_ref ** 2 * n * (g.T_ref / T) ** (g.omega - 0.5))
    got = dist / (2.0 * coll)
    assert abs(got / lam - 1.0) < 4.0 / math.sqrt(coll), (got, lam, coll)
