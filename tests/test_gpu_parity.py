"""GPU (CUDA path through the C ABI) against the CPU oracle, element by element.

The particle loop is specified as a fixed sequence of IEEE operations (no
contraction, own FP32 ln/exp, counter-based Philox streams), so cell ids,
order, positions, velocities, rotational energies and candidate-pair lists
are compared bit for bit.  The per-step cell sums are accumulated in FP32 on
the GPU and in FP64 by the oracle: they are compared within the FP32
summation bound (see tol_phi).
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import orc
from paper_2607_08195_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_08195_gb300 import dig  # noqa: E402


GPU_ONLY = ("tile_cells", "stage_cap", "wait_timeout_s", "cta_threads")


def pair(scen, **over):
    """A GPU solver and an oracle on the same scenario and overrides."""
    oo = {k: v for k, v in over.items() if k not in GPU_ONLY}
    return dig.Solver(scen, "cuda:0", **over), orc.Oracle(scen, **oo)


def assert_same_particles(g, o):
    xg, vg, Ig, cg = g.read()
    xo, vo, Io, co = o.read()
    assert len(cg) == len(co)
    assert np.array_equal(cg, co), f"cells differ at {np.flatnonzero(cg != co)[:10]}"
    bad = np.flatnonzero(np.any(xg != xo, axis=1))
    assert len(bad) == 0, f"positions differ at {bad[:10]}: {xg[bad[:3]]} vs {xo[bad[:3]]}"
    badv = np.flatnonzero(np.any(vg != vo, axis=1))
    assert len(badv) == 0, f"velocities differ at {badv[:10]}: {vg[badv[:3]]} vs {vo[badv[:3]]}"
    assert np.array_equal(Ig, Io)
    return xg, vg, Ig, cg


def tol_phi(mo, nmax):
    """FP32 sums of <= nmax terms: |error| <= nmax * 2^-24 * sum|terms| per
    component; bounded here by the oracle's magnitude scale per component."""
    scale = np.abs(mo).max(axis=0)
    return 4 * nmax * 2.0 ** -24 * np.maximum(scale, 1e-30)


def test_init_bit_exact():
    s = W.config_small()
    g, o = pair(s)
    g.init()
    o.init()
    assert_same_particles(g, o)


def test_single_step_from_written_state():
    """One step from an identical serialised state: cells, order, positions,
    velocities and every candidate pair (i, j, accept) are bit-identical."""
    s = W.config_small(seed=11)
    rng = np.random.default_rng(3)
    x, v, Ir, cell = W.random_particles(rng, s, 20_000)
    g, o = pair(s)
    g.write(x, v, Ir, cell)
    o.write(x, v, Ir, cell)
    assert_same_particles(g, o)
    g.step(1, dig.EWMA | dig.INST | dig.RECORD_PAIRS | dig.SYNC)
    o.step(1, orc.EWMA | orc.RECORD_PAIRS)
    assert_same_particles(g, o)
    pg, po = g.pairs(), o.pairs()
    assert len(pg) == len(po) > 1000
    assert np.array_equal(pg, po)
    mg, mo = g.moments(dig.PHI_INST), o.moments(orc.PHI_INST)
    nmax = np.bincount(o.read()[3]).max()
    assert np.all(np.abs(mg - mo) <= tol_phi(mo, nmax))
    cg, co = g.cell_state(), o.cell_state()
    assert np.array_equal(cg[0], co[0])
    assert np.array_equal(cg[1], co[1])


def test_multi_step_bit_exact_and_averages():
    """30 steps from the initial state: the whole particle state stays
    bit-identical; counters equal; time averages within FP32-sum tolerance."""
    s = W.config_small(seed=1)
    g, o = pair(s, n_a=50)
    g.init()
    o.init()
    fl = dig.EWMA | dig.WINDOW | dig.CUMUL | dig.INST | dig.WALLFLUX
    g.step(30, fl | dig.SYNC)
    o.step(30, orc.EWMA | orc.WINDOW | orc.CUMUL)
    assert_same_particles(g, o)
    cg, co = g.counters(), o.counters()
    for k in ("steps", "cand", "coll", "cross", "wall", "removed", "stuck"):
        assert cg[k] == co[k], (k, cg[k], co[k])
    nmax = 80
    for w in (dig.PHI_EWMA, dig.PHI_WINDOW, dig.PHI_CUM):
        mg, mo = g.moments(w), o.moments(w)
        assert np.all(np.abs(mg - mo) <= 30 * tol_phi(mo, nmax)), w
        Mg, Mo = g.moments(w | dig.MACRO), o.moments(w | dig.MACRO)
        # rho, u, T: relative 1e-5 of their natural scales
        assert np.allclose(Mg[:, 1], Mo[:, 1], rtol=1e-12)
        assert np.all(np.abs(Mg[:, 2:5] - Mo[:, 2:5]) <= 1e-3)  # m/s
        assert np.allclose(Mg[:, 5], Mo[:, 5], rtol=1e-5)
    fg, fo = g.wall_flux(), o.wall_flux()
    assert np.array_equal(fg[:, 0], fo[:, 0])
    assert np.allclose(fg, fo, rtol=1e-9, atol=1e-9 * np.abs(fo).max())


def test_diatomic_bit_exact():
    """Nitrogen with Borgnakke-Larsen exchange: rotational energies bit-exact."""
    s = W.cavity_scenario(4, 12_000, 0.05, seed=4, gas=W.NITROGEN)
    g, o = pair(s)
    g.init()
    o.init()
    g.step(12, dig.EWMA | dig.SYNC)
    o.step(12, orc.EWMA)
    assert_same_particles(g, o)
    assert g.counters()["lb"] == o.counters()["lb"] > 0


@pytest.mark.parametrize("gas", [W.ARGON_VSS, W.NITROGEN_VSS, dataclasses.replace(W.ARGON, alpha=3.0)],
                         ids=["argon-vss", "nitrogen-vss", "alpha3"])
def test_vss_scattering_bit_exact(gas):
    """VSS scattering (alpha != 1): one step from a written state with every
    candidate pair, then 12 more steps, bit-identical to the oracle."""
    s = W.cavity_scenario(4, 12_000, 0.05, seed=9, gas=gas)
    rng = np.random.default_rng(9)
    x, v, Ir, cell = W.random_particles(rng, s, 12_000)
    g, o = pair(s)
    g.write(x, v, Ir, cell)
    o.write(x, v, Ir, cell)
    g.step(1, dig.EWMA | dig.RECORD_PAIRS | dig.SYNC)
    o.step(1, orc.EWMA | orc.RECORD_PAIRS)
    assert_same_particles(g, o)
    pg, po = g.pairs(), o.pairs()
    assert len(pg) == len(po) > 100
    assert np.array_equal(pg, po)
    g.step(12, dig.EWMA | dig.SYNC)
    o.step(12, orc.EWMA)
    assert_same_particles(g, o)
    cg, co = g.counters(), o.counters()
    for k in ("cand", "coll", "lb", "cross", "wall"):
        assert cg[k] == co[k], (k, cg[k], co[k])
    assert co["coll"] > 1000


@pytest.mark.parametrize("tile_cells,stage_cap,threads", [(1, 4096, 256), (7, 512, 256), (256, 8192, 256),
                                                          (0, 1024, 64), (5, 1536, 128)])
def test_tiling_does_not_change_results(tile_cells, stage_cap, threads):
    """Ragged tiles (cells not a multiple of the tile) and small shared-memory
    stages (cells grouped several times per CTA) give identical results."""
    s = W.cavity_scenario(5, 15_000, 0.1, seed=6)
    g, o = pair(s, tile_cells=tile_cells, stage_cap=stage_cap, cta_threads=threads)
    g.init()
    o.init()
    g.step(4, dig.EWMA | dig.SYNC)
    o.step(4, orc.EWMA)
    assert_same_particles(g, o)


def test_edge_cases():
    s = W.config_small(seed=5)
    # no particles at all
    g = dig.Solver(s, "cuda:0")
    g.write(np.zeros((0, 3)), np.zeros((0, 3), np.float32), np.zeros(0, np.float32), np.zeros(0, np.int32))
    g.step(3, dig.EWMA | dig.SYNC)
    assert g.count() == 0
    # one particle; two particles in one cell
    g2, o2 = pair(s)
    cen = s.mesh.nodes[s.mesh.tets[17]].mean(axis=0)
    x = np.array([cen, cen + 1e-9])
    v = np.array([[300.0, -50.0, 20.0], [-100.0, 10.0, 0.0]], np.float32)
    for n in (1, 2):
        g2.write(x[:n], v[:n], np.zeros(n, np.float32), np.full(n, 17, np.int32))
        o2.write(x[:n], v[:n], np.zeros(n, np.float32), np.full(n, 17, np.int32))
        g2.step(5, dig.EWMA | dig.SYNC)
        o2.step(5, orc.EWMA)
        assert_same_particles(g2, o2)
    # velocity components that are zero, negative zero or FP32 subnormal
    # (their exact FP64 value enters x + v dt)
    rng = np.random.default_rng(12)
    n = 64
    P = s.mesh.nodes[s.mesh.tets[17]]
    x = rng.dirichlet(np.ones(4), size=n) @ P
    v = (rng.standard_normal((n, 3)) * 300.0).astype(np.float32)
    v[:8, 0] = 0.0
    v[8:16, 1] = -0.0
    v[16:32, 2] = np.float32(1e-40) * rng.integers(1, 1000, 16).astype(np.float32)
    v[32:40, :] = np.float32(-3e-39)
    g3, o3 = pair(s)
    g3.write(x, v, np.zeros(n, np.float32), np.full(n, 17, np.int32))
    o3.write(x, v, np.zeros(n, np.float32), np.full(n, 17, np.int32))
    g3.step(1, dig.EWMA | dig.SYNC)
    o3.step(1, orc.EWMA)
    assert_same_particles(g3, o3)


@pytest.mark.parametrize("gas", [W.ARGON, W.NITROGEN])
def test_dense_cells_take_both_collision_paths(gas):
    """Cells with more NTC candidates than a chunk of precomputed candidate
    records holds (about 1,000 particles per cell and a time step near the
    mean collision time) run the per-candidate loop; cells with fewer run on
    precomputed records; both give the oracle's pairs, acceptances and
    velocities bit for bit, with and without rotational exchange."""
    T, n = 273.0, 1.677e22
    mu = gas.mu_ref() * (T / gas.T_ref) ** gas.omega
    npart = 6000
    s = W.Scenario(gas=gas, mesh=W.closed_box(1, 1e-3, W.BC_DIFFUSE), n_particles=npart, n_init=n, T_init=T,
                   u_init=(0.0, 0.0, 0.0), F_N=n * 1e-9 / npart, dt=1.2 * mu / (n * W.K_B * T), seed=21, L=1e-3,
                   Kn=0.1, capacity=2 * npart)
    g, o = pair(s)
    g.init()
    o.init()
    g.step(2, dig.EWMA | dig.RECORD_PAIRS | dig.SYNC)
    o.step(2, orc.EWMA | orc.RECORD_PAIRS)
    assert_same_particles(g, o)
    pg, po = g.pairs(), o.pairs()
    assert np.array_equal(pg, po)
    per_cell = np.bincount(po[:, 0])
    assert per_cell.max() > 600 and per_cell.min() > 0
    assert g.counters()["coll"] == o.counters()["coll"]


def test_one_cell_holding_many_particles():
    """600 particles written into one cell (far more than a move tile aims
    at, stage_cap = 256): the cell's NTC loop, the gather and the move give
    the oracle's particles and pairs bit for bit over two steps."""
    s = W.config_small(seed=2)
    g, o = pair(s, stage_cap=256)
    n = 600
    rng = np.random.default_rng(8)
    P = s.mesh.nodes[s.mesh.tets[40]]
    w = rng.dirichlet(np.ones(4), size=n)
    x = w @ P
    v = (rng.standard_normal((n, 3)) * 300.0).astype(np.float32)
    for h in (g, o):
        h.write(x, v, np.zeros(n, np.float32), np.full(n, 40, np.int32))
    g.step(2, dig.EWMA | dig.RECORD_PAIRS | dig.SYNC)
    o.step(2, orc.EWMA | orc.RECORD_PAIRS)
    assert_same_particles(g, o)
    pg, po = g.pairs(), o.pairs()
    assert len(po) > 500 and np.array_equal(pg, po)


def test_crossing_limit_matches_oracle():
    """With a crossing cap of 1 per step the truncated tracks are identical on
    both sides and the GPU reports DIG_ERR_STUCK."""
    s = W.config_small(seed=8)
    g, o = dig.Solver(s, "cuda:0", max_cross=1), orc.Oracle(s, max_cross=1)
    g.init()
    o.init()
    with pytest.raises(dig.DigError, match="STUCK"):
        g.step(1, dig.SYNC)
    o.step(1, 0)
    assert g.counters()["stuck"] == o.counters()["stuck"] > 0
    assert_same_particles(g, o)


def test_full_size_workload_one_step():
    """The 8M-particle, 162,000-tet cavity (the benchmarked workload, same
    launch configuration as bench.py): one step from the initial state,
    bit-identical to the oracle over every particle."""
    s = W.config_c2()
    g, o = pair(s)
    g.init()
    o.init()
    g.step(1, dig.EWMA | dig.SYNC)
    o.step(1, orc.EWMA)
    xg, vg, Ig, cg = assert_same_particles(g, o)
    assert len(cg) == s.n_particles
    cg_, co_ = g.counters(), o.counters()
    assert cg_["coll"] == co_["coll"] and cg_["cross"] == co_["cross"]


@pytest.mark.parametrize("n,n_cells", [(0, 7), (1, 1), (5000, 37), (200_000, 1296), (1_000_000, 162_000), (30_000, 3)])
def test_sort_by_cell_matches_oracle(n, n_cells):
    """Standalone bucket sort (C ABI dig_sort_by_cell) against the oracle's
    stable counting sort: cell_start and order bit-identical; -1 dropped;
    small and very large segments (n/n_cells up to 10^4)."""
    rng = np.random.default_rng(n + n_cells)
    cell = rng.integers(-1, n_cells, size=n).astype(np.int32)
    cs_o, ord_o = orc.sort_by_cell(cell, n_cells)
    cs_g, ord_g = dig.sort_by_cell(torch.from_numpy(cell).cuda(), n_cells)
    assert np.array_equal(cs_g.cpu().numpy(), cs_o)
    assert np.array_equal(ord_g.cpu().numpy(), ord_o)


@pytest.mark.parametrize("n,n_cells,heavy", [(65_536, 1, 0), (65_536, 64, 0.9), (1_000_000, 4096, 0.5),
                                             (4_000, 100, 1.0)])
def test_sort_by_cell_heavy_segments(n, n_cells, heavy):
    """The bucket sort on skewed input: a fraction `heavy` of the elements in
    one cell (all of them in a single cell at n = 65,536), the rest spread:
    cell_start and order identical to numpy's stable argsort, and the long
    segments sorted in time linear in their length (the whole call well under
    a second)."""
    import time

    rng = np.random.default_rng(n + n_cells)
    cell = rng.integers(-1, n_cells, size=n).astype(np.int32)
    cell[rng.random(n) < heavy] = n_cells // 2
    keep = cell >= 0
    want = np.flatnonzero(keep)[np.argsort(cell[keep], kind="stable")]
    want_cs = np.concatenate([[0], np.cumsum(np.bincount(cell[keep], minlength=n_cells))])
    dcell = torch.from_numpy(cell).cuda()
    dig.sort_by_cell(dcell, n_cells)  # warm
    t0 = time.perf_counter()
    cs_g, ord_g = dig.sort_by_cell(dcell, n_cells)
    dt = time.perf_counter() - t0
    assert np.array_equal(cs_g.cpu().numpy(), want_cs)
    assert np.array_equal(ord_g.cpu().numpy(), want)
    assert dt < 0.5, dt


def inflow_box(gas, U, sides_inflow, nh=2, n=1.677e22, T=273.0, n_particles=6000, seed=13):
    bcs = [dict(kind=W.BC_INFLOW, T=T, U=tuple(U), n=n), dict(kind=W.BC_OUTFLOW, T=T, U=(0.0, 0.0, 0.0), n=0.0)]
    mesh = W.box_sides(nh, 1e-3, [0 if sd in sides_inflow else 1 for sd in range(6)], bcs)
    mu = gas.mu_ref() * (T / gas.T_ref) ** gas.omega
    return W.Scenario(gas=gas, mesh=mesh, n_particles=n_particles, n_init=n, T_init=T, u_init=tuple(U),
                      F_N=n * 1e-9 / n_particles, dt=0.2 * mu / (n * W.K_B * T), seed=seed, L=1e-3, Kn=0.1,
                      capacity=8 * n_particles)


@pytest.mark.parametrize("gas,U,sides", [(W.ARGON, (200.0, -50.0, 30.0), range(6)),
                                         (W.NITROGEN, (500.0, 0.0, 0.0), (0,)),
                                         (W.ARGON, (-150.0, 0.0, 0.0), (0, 2))])
def test_injection_bit_exact(gas, U, sides):
    """Free-stream injection and outflow removal (S4): from the same initial
    state, 15 steps give identical particles (injected ones included), counts
    of injected / removed particles and collision counters."""
    s = inflow_box(gas, U, sides)
    g, o = pair(s)
    g.init()
    o.init()
    g.step(15, dig.EWMA | dig.SYNC)
    o.step(15, orc.EWMA)
    assert_same_particles(g, o)
    cg, co = g.counters(), o.counters()
    for k in ("injected", "removed", "cand", "coll", "cross", "lb"):
        assert cg[k] == co[k], (k, cg[k], co[k])
    assert cg["injected"] > 0 and cg["removed"] > 0


def seeded_dig_state(scen, steps=60, **over):
    """Oracle state after `steps` DSMC steps (moving average, wall fluxes on);
    returns the oracle and its particles, sums and wall fluxes."""
    o = orc.Oracle(scen, **over)
    o.init()
    o.step(steps, orc.EWMA)
    return o, o.read(), o.moments(orc.PHI_EWMA), o.wall_flux()


def converged_pair(rg, ro, N_m, eps):
    """Both solves stopped on the residual test, not on N_m.  Their iteration
    counts are not compared: the accelerated iteration's path moves with the
    last bits of its inputs (fused multiply-adds and summation order differ
    between the two sides), and so does the iteration at which it crosses
    eps_m; its converged state does not."""
    for r in (rg, ro):
        assert r["iters"] < N_m and r["residual"] <= eps, r


@pytest.mark.parametrize("nh,kn,passes,kmax,gas,recon", [(4, 0.1, 3, 0.6, W.ARGON, 0), (5, 0.05, 2, 0.4, W.ARGON, 0),
                                                         (4, 0.1, 3, 0.6, W.NITROGEN, 0),
                                                         (5, 0.05, 2, 0.4, W.ARGON, 1),
                                                         (4, 0.1, 3, 0.6, W.NITROGEN, 1)])
def test_couple_parity_from_written_state(nh, kn, passes, kmax, gas, recon):
    """S9-S11 from an identical written state (particles, moving-average sums,
    wall fluxes), the synthetic solve converged to eps_m = 1e-12: identical
    filter flags, rejection/reconstruction counts, clone/delete decisions and
    particle cells; FP64 fields within 1e-9.  Nitrogen carries the rotational
    energy equation and heat flux; recon = 1 reconstructs density and
    temperatures by their logarithmic mean."""
    s = W.cavity_scenario(nh, 30 * 6 * nh ** 3, kn, seed=17, gas=gas)
    over = dict(N_m=4000, eps_m=1e-12, passes=passes, KnD_max=kmax, recon=recon)
    o, (x, v, Ir, cell), phi, wf = seeded_dig_state(s, **over)
    g = dig.Solver(s, "cuda:0", **over)
    g.write(x, v, Ir, cell)
    g.write_moments(dig.PHI_EWMA, phi)
    g.write_wall_flux(wf, 60)
    rg = g.couple()
    ro = o.couple()
    converged_pair(rg, ro, 4000, 1e-12)
    for k in ("n_rejected", "n_reconstructed", "n_cloned", "n_deleted"):
        assert rg[k] == ro[k], (k, rg[k], ro[k])
    assert ro["n_rejected"] > 0 and ro["n_cloned"] + ro["n_deleted"] > 0
    assert np.array_equal(g.read_couple(3), o.read_couple(3))
    for which in (4, 0, 1, 2):
        a, b = g.read_couple(which), o.read_couple(which)
        scale = np.abs(b).max(axis=0) + 1e-30
        assert np.all(np.abs(a - b) <= 1e-9 * scale), (which, np.abs(a - b).max())
    xg, vg, Ig, cg = g.read()
    xo, vo, Io, co = o.read()
    assert np.array_equal(cg, co)
    assert np.array_equal(xg, xo)
    assert np.allclose(vg, vo, rtol=1e-6, atol=1e-4)


@pytest.mark.parametrize("N_m", [20, 4000])
def test_couple_safeguard_parity(N_m):
    """The synthetic solve's best-iterate safeguard on the GPU (CFL 48 without
    acceleration: explicit local steps are stable only near CFL 1).  With
    N_m = 20 every iterate is worse than the initial state, so M^{k+1} is
    M^{k+1/2} itself and the residual 1, on both sides; with N_m = 4000 the
    CFL halvings on divergence let both converge to 1e-12, to the same fixed
    point within 1e-9."""
    s = W.cavity_scenario(6, 60_000, 0.01, seed=23)
    over = dict(N_m=N_m, eps_m=1e-12, passes=3, KnD_max=1.0, cfl=48.0, aa_m=0)
    o, (x, v, Ir, cell), phi, wf = seeded_dig_state(s, steps=40, **over)
    g = dig.Solver(s, "cuda:0", **over)
    g.write(x, v, Ir, cell)
    g.write_moments(dig.PHI_EWMA, phi)
    g.write_wall_flux(wf, 40)
    rg, ro = g.couple(), o.couple()
    assert np.array_equal(g.read_couple(3), o.read_couple(3))
    if N_m == 20:
        assert rg["iters"] == ro["iters"] == 20 and rg["residual"] == ro["residual"] == 1.0, (rg, ro)
        for side in (g, o):
            assert np.allclose(side.read_couple(2), side.read_couple(0), rtol=1e-13, atol=1e-15)
    else:
        converged_pair(rg, ro, N_m, 1e-12)
        a, b = g.read_couple(2), o.read_couple(2)
        assert np.all(np.abs(a - b) <= 1e-9 * np.abs(b).max(axis=0)), np.abs(a - b).max(axis=0)


def test_couple_parity_benchmarked_solve():
    """The coupling at the synthetic-solve configuration the bench runs (N_m =
    500, eps_m = 1e-6, Anderson depth 20, CFL 1.5) on the 48,000-tet cavity at
    Kn = 0.01, from a written state (480,000 particles after 40 DSMC steps).
    Filter flags, rejection counts and the solve's inputs (own state,
    M^{k+1/2}, HoT) agree within 1e-9.  Both solves stop at N_m above eps_m,
    and an unconverged accelerated iteration's state moves with the last bits
    of its inputs: the test measures that spread on the oracle itself (a second
    oracle solve from inputs perturbed by 2e-16 relative; about 3e-3 of each
    component's scale here) and requires the GPU's solved state to lie within
    10 times it of the oracle's, its residual within a factor 2, and its
    clone and delete counts (and the per-cell particle counts after them)
    within a few plus 10 times that spread of the oracle's counts."""
    s = W.cavity_scenario(20, 480_000, 0.01, seed=23)
    over = dict(N_m=500, passes=3, KnD_max=1.0)
    o, (x, v, Ir, cell), phi, wf = seeded_dig_state(s, steps=40, **over)
    g = dig.Solver(s, "cuda:0", **over)
    g.write(x, v, Ir, cell)
    g.write_moments(dig.PHI_EWMA, phi)
    rg, ro = g.couple(), o.couple()
    assert rg["iters"] == ro["iters"] == 500 and ro["residual"] > 1e-6
    assert 0.5 < rg["residual"] / ro["residual"] < 2.0, (rg["residual"], ro["residual"])
    for k in ("n_rejected", "n_reconstructed"):
        assert rg[k] == ro[k], (k, rg[k], ro[k])
    assert np.array_equal(g.read_couple(3), o.read_couple(3))
    for which in (4, 0, 1):
        a, b = g.read_couple(which), o.read_couple(which)
        scale = np.abs(b).max(axis=0) + 1e-30
        assert np.all(np.abs(a - b) <= 1e-9 * scale), (which, np.abs(a - b).max())
    half, hot, new_o = o.read_couple(0), o.read_couple(1), o.read_couple(2)
    f = 1.0 + np.random.default_rng(1).choice([-1.0, 1.0], half.shape) * 2e-16
    new_p, it_p, _ = orc.Oracle(s, **over).synthetic_solve(half * f, hot=hot)
    scale = np.abs(new_o).max(axis=0) + 1e-30
    spread = (np.abs(new_p - new_o) / scale).max(axis=0)
    diff = (np.abs(g.read_couple(2) - new_o) / scale).max(axis=0)
    assert it_p == 500 and np.all(diff <= 10 * spread + 1e-9), (diff, spread)
    # clone/delete decisions follow the solved density ratio: a relative
    # change d of the state moves about d of them
    for k in ("n_cloned", "n_deleted"):
        assert abs(rg[k] - ro[k]) <= 3 + 10 * spread.max() * ro[k], (k, rg[k], ro[k])
    n_o = np.bincount(o.read()[3], minlength=o.n_tets)
    n_g = np.bincount(g.read()[3], minlength=o.n_tets)
    assert np.abs(n_g - n_o).sum() <= 6 + 20 * spread.max() * (ro["n_cloned"] + ro["n_deleted"])


def test_local_accumulation_state_parity():
    """Local accumulation state (Sec. 3.2, local_acc = 1): a coupling that rejects
    the dilute part of the cavity puts the same cells into the state with the
    same weight as the oracle; 15 more steps from identical particles (the
    oracle's, written to both) leave identical weights and moving averages
    within the FP32-sum tolerance, the rejected cells on the running mean."""
    s = W.cavity_scenario(3, 5000, 0.1, seed=3)
    over = dict(N_m=1, KnD_max=1.5, passes=2, n_a=10, local_acc=1)
    g, o = pair(s, **over)
    g.init()
    o.init()
    g.step(20, dig.EWMA | dig.SYNC)
    o.step(20, orc.EWMA)
    vol = o.mesh_info()["vol"]
    cen = s.mesh.nodes[s.mesh.tets].mean(axis=1)
    dilute = cen[:, 0] < -0.1e-3
    kT_m = W.K_B * s.T_init / s.gas.mass
    N = s.n_init * vol / s.F_N * np.where(dilute, 0.05, 1.0)
    phi = np.zeros((len(vol), dig.NPHI))
    phi[:, 0] = N
    phi[:, 4:7] = (N * kT_m)[:, None]
    g.write_moments(dig.PHI_EWMA, phi)
    o.write_moments(orc.PHI_EWMA, phi)
    g.couple()
    o.couple()
    assert np.array_equal(g.read_couple(3), o.read_couple(3))
    wg, wo = g.read_couple(5), o.read_couple(5)
    assert np.array_equal(wg, wo)
    assert np.array_equal(wo[:, 0] > 0, dilute)
    x, v, Ir, cell = o.read()
    g.write(x, v, Ir, cell)
    g.write_moments(dig.PHI_EWMA, o.moments(orc.PHI_EWMA))
    g.step(15, dig.EWMA | dig.SYNC)
    o.step(15, orc.EWMA)
    assert_same_particles(g, o)
    assert np.array_equal(g.read_couple(5), o.read_couple(5))
    assert np.all(o.read_couple(5)[dilute, 0] == 25.0)
    mg, mo = g.moments(dig.PHI_EWMA), o.moments(orc.PHI_EWMA)
    assert np.all(np.abs(mg - mo) <= 30 * tol_phi(mo, 80))


def test_couple_fixed_point_identity_on_gpu():
    """Uniform equilibrium with the exact wall pressure: the GPU coupling leaves
    the state and every particle unchanged (no clones or deletions); every
    cell holds exactly the count its density stands for (48 x 100)."""
    s = W.Scenario(gas=W.ARGON, mesh=W.closed_box(2, 1e-3, W.BC_DIFFUSE), n_particles=4800, n_init=1.677e22,
                   T_init=273.0, u_init=(0.0, 0.0, 0.0), F_N=1.677e22 * 1e-9 / 4800, dt=6.7e-8, seed=5, L=1e-3,
                   Kn=0.1, capacity=9600)
    g = dig.Solver(s, "cuda:0", N_m=40, KnD_max=1e9)
    g.write(*W.particles_per_cell(np.random.default_rng(5), s, 100))
    x0, v0, I0, c0 = g.read()
    vol = orc.Oracle(s).mesh_info()["vol"]
    kT_m = W.K_B * s.T_init / s.gas.mass
    N = s.n_init * vol / s.F_N
    phi = np.zeros((len(vol), dig.NPHI))
    phi[:, 0] = N
    phi[:, 4:7] = (N * kT_m)[:, None]
    g.write_moments(dig.PHI_EWMA, phi)
    # exact pressure on every wall face
    mi = orc.Oracle(s).mesh_info()
    P = s.mesh.nodes[s.mesh.tets]
    rows = []
    p = s.n_init * W.K_B * s.T_init
    for t in range(len(vol)):
        for f in range(4):
            if mi["nbr"][t, f] < 0:
                q = [k for k in range(4) if k != f]
                A = 0.5 * np.linalg.norm(np.cross(P[t, q[1]] - P[t, q[0]], P[t, q[2]] - P[t, q[0]]))
                rows.append([1.0, *(p * mi["normals"][t, f] * A * 10 * s.dt), 0.0])
    g.write_wall_flux(np.array(rows), 10)
    r = g.couple()
    assert r["n_cloned"] == 0 and r["n_deleted"] == 0 and r["n_rejected"] == 0
    assert np.allclose(g.read_couple(2), g.read_couple(0), rtol=0, atol=1e-10)
    x1, v1, I1, c1 = g.read()
    assert np.array_equal(v0, v1) and np.array_equal(x0, x1) and np.array_equal(c0, c1)


def uniform_phi(vol, scen, scale):
    """Summation variables of a Maxwellian at rest at T_init, n_init * scale."""
    kT_m = W.K_B * scen.T_init / scen.gas.mass
    N = scen.n_init * vol / scen.F_N * scale
    phi = np.zeros((len(vol), dig.NPHI))
    phi[:, 0] = N
    phi[:, 4:7] = (N * kT_m)[:, None]
    return phi


def test_deep_fill_layers_match_oracle():
    """One accepted corner of the 48,000-tet cavity, every other cell dilute
    (rejected): after 3 reconstruction passes the rest of the mesh is reached
    only by fill layers, about 75 of them, so the GPU's fill runs past its
    first chunk of 64 layers.  Flags and counts agree exactly, M^{k+1/2} and
    HoT within the tolerance of the other coupling tests (the fill is a chain
    of neighbour means, summed in the same order on both sides)."""
    s = W.cavity_scenario(20, 480_000, 0.1, seed=3)
    over = dict(N_m=5, passes=3, KnD_max=5.0)
    o = orc.Oracle(s, **over)
    o.init()
    g = dig.Solver(s, "cuda:0", **over)
    g.write(*o.read())
    vol = o.mesh_info()["vol"]
    cen = s.mesh.nodes[s.mesh.tets].mean(axis=1) / s.L
    scale = np.where((cen < -0.45).all(axis=1), 1.0, 0.05)
    phi = uniform_phi(vol, s, scale)
    phi[:, 1] = phi[:, 0] * 20.0 * cen[:, 1]  # a drift that varies, so the means carry information
    phi[:, 4] += phi[:, 1] ** 2 / np.maximum(phi[:, 0], 1e-300)
    g.write_moments(dig.PHI_EWMA, phi)
    o.write_moments(orc.PHI_EWMA, phi)
    rg, ro = g.couple(), o.couple()
    fl = o.read_couple(3)[:, 0]
    assert np.array_equal(g.read_couple(3)[:, 0], fl)
    assert (fl == 1).sum() == int((scale == 1.0).sum()) and (fl == 0).sum() == 0
    assert (fl == 3).sum() > 0.9 * len(fl)
    for k in ("n_rejected", "n_reconstructed"):
        assert rg[k] == ro[k], (k, rg[k], ro[k])
    # the accepted cells' own states differ by the rounding of their moments
    # (relative 1e-9 as in the other coupling tests; the HoT of a gas at rest
    # is round-off itself, hence the absolute 1e-12 in nondimensional units)
    for which in (0, 1):
        a, b = g.read_couple(which), o.read_couple(which)
        sc = np.abs(b).max(axis=0)
        assert np.all(np.abs(a - b) <= 1e-9 * sc + 1e-12), (which, np.abs(a - b).max())


def test_unreached_cells_take_initial_state_on_gpu():
    """No accepted cell anywhere: every cell keeps flag 0 and starts the solve
    from the configuration's initial state with zero HoT, as in the oracle."""
    s = dataclasses.replace(W.cavity_scenario(3, 5000, 0.1, seed=3), u_init=(40.0, -15.0, 0.0))
    over = dict(N_m=1, passes=2, KnD_max=1.5)
    o = orc.Oracle(s, **over)
    o.init()
    g = dig.Solver(s, "cuda:0", **over)
    g.write(*o.read())
    phi = uniform_phi(o.mesh_info()["vol"], s, 0.05)
    g.write_moments(dig.PHI_EWMA, phi)
    o.write_moments(orc.PHI_EWMA, phi)
    rg, ro = g.couple(), o.couple()
    assert rg["n_rejected"] == ro["n_rejected"] == o.n_tets and rg["n_reconstructed"] == 0
    assert np.all(g.read_couple(3) == 0)
    assert np.array_equal(g.read_couple(0), o.read_couple(0))
    assert np.all(g.read_couple(1) == 0.0)


# ----------------------------------------------------------- hypersonic sphere
def test_sphere_bit_exact():
    """Hypersonic argon sphere (Mach 10 free stream, diffuse body at 500 K) on
    a small graded Delaunay mesh (13,012 tets): 8 steps with free-stream
    injection over the far field, wall reflections on the body and outflow
    removal give particles and counters identical to the oracle's."""
    s = W.sphere_scenario(0.02, 60_000, seed=4)
    g, o = pair(s)
    g.init()
    o.init()
    g.step(8, dig.EWMA | dig.SYNC)
    o.step(8, orc.EWMA)
    assert_same_particles(g, o)
    cg, co = g.counters(), o.counters()
    for k in ("injected", "removed", "cand", "coll", "cross", "wall", "stuck"):
        assert cg[k] == co[k], (k, cg[k], co[k])
    assert cg["injected"] > 0 and cg["removed"] > 0 and cg["wall"] > 0 and cg["stuck"] == 0


def test_sphere_full_size_properties():
    """The full sphere workload (about 2M tets graded 20x toward the body,
    100M particles), two steps in the bench's launch configuration: the count
    follows N = N_0 + injected - removed, no particle exceeds the crossing
    limit, and 4,096 sampled particles lie inside the tets they were tracked
    to (barycentric coordinates >= -1e-9)."""
    s = W.config_c4()
    g = dig.Solver(s, "cuda:0")
    g.init()
    n0 = g.count()
    g.step(2, dig.EWMA | dig.SYNC)
    c = g.counters()
    n1 = g.count()
    assert n0 == s.n_particles and n1 == n0 + c["injected"] - c["removed"]
    assert c["stuck"] == 0 and c["injected"] > 0 and c["removed"] > 0 and c["coll"] > 0
    x, v, I, cell = g.read()
    rng = np.random.default_rng(4)
    k = rng.choice(len(cell), 4096, replace=False)
    P = s.mesh.nodes[s.mesh.tets[cell[k]]]
    T = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=2)
    lam = np.linalg.solve(T, (x[k] - P[:, 0])[..., None])[..., 0]
    bary = np.concatenate([1.0 - lam.sum(axis=1, keepdims=True), lam], axis=1)
    assert bary.min() >= -1e-9, bary.min()
    assert np.all(np.isfinite(v[k]))


def test_couple_parity_sphere():
    """DIG coupling on the hypersonic sphere (13,012 tets, 60,000 particles),
    the solve converged to eps_m = 1e-12: free-stream faces in the synthetic
    solve, cells rejected for holding
    fewer than two particles on average, reconstruction layers and fill
    layers beyond them; identical flags and counts, FP64 fields within 1e-9,
    identical recalibrated particle cells."""
    s = W.sphere_scenario(0.02, 60_000, seed=4)
    over = dict(N_m=6000, eps_m=1e-12, passes=3, KnD_max=1.0)
    o, (x, v, Ir, cell), phi, wf = seeded_dig_state(s, steps=40, **over)
    g = dig.Solver(s, "cuda:0", **over)
    g.write(x, v, Ir, cell)
    g.write_moments(dig.PHI_EWMA, phi)
    rg, ro = g.couple(), o.couple()
    converged_pair(rg, ro, 6000, 1e-12)
    for k in ("n_rejected", "n_reconstructed", "n_cloned", "n_deleted"):
        assert rg[k] == ro[k], (k, rg[k], ro[k])
    flags = o.read_couple(3)[:, 0]
    assert np.array_equal(g.read_couple(3)[:, 0], flags)
    assert (flags == 3).sum() > 0 and (flags == 2).sum() > 0 and (flags == 1).sum() > 0
    # the solve's inputs within 1e-9; the converged state within 1e-8: the
    # oracle's own converged state moves by 1.6e-9 of each component's scale
    # when the solve's inputs are perturbed by 2e-16 relative (graded mesh,
    # Mach 10; 1e-11 on the cavity)
    for which, tol in ((4, 1e-9), (0, 1e-9), (1, 1e-9), (2, 1e-8)):
        a, b = g.read_couple(which), o.read_couple(which)
        scale = np.abs(b).max(axis=0) + 1e-30
        assert np.all(np.abs(a - b) <= tol * scale), (which, np.abs(a - b).max())
    assert np.array_equal(g.read()[3], o.read()[3])


# ----------------------------------------------------------- diatomic capsule
def test_capsule_bit_exact():
    """Nitrogen at Mach 25 over the capsule at 20 degrees incidence (14,381
    tets, 50,000 particles): 8 steps with Borgnakke-Larsen exchange, free-stream
    injection, wall reflections and outflow give particles (rotational
    energies included) and counters identical to the oracle's."""
    s = W.capsule_scenario(0.3, 50_000, seed=5)
    g, o = pair(s)
    g.init()
    o.init()
    g.step(8, dig.EWMA | dig.SYNC)
    o.step(8, orc.EWMA)
    assert_same_particles(g, o)
    cg, co = g.counters(), o.counters()
    for k in ("injected", "removed", "cand", "coll", "cross", "wall", "lb", "stuck"):
        assert cg[k] == co[k], (k, cg[k], co[k])
    assert cg["lb"] > 0 and cg["wall"] > 0 and cg["stuck"] == 0


def test_couple_parity_capsule():
    """DIG coupling on the nitrogen capsule at Mach 25 (14,381 tets, 50,000
    particles after 40 steps), the solve converged to eps_m = 1e-12 (about
    5,900 iterations): rotational energy equation and heat flux, free-stream
    and outflow faces, a wall at 500 K; most cells filled (few particles per
    cell this early).  Identical flags and counts, the solve's inputs within
    1e-9 and its converged state within 1e-8 (as on the sphere), identical
    recalibrated particle cells."""
    s = W.capsule_scenario(0.3, 50_000, seed=5)
    over = dict(N_m=12000, eps_m=1e-12, passes=3, KnD_max=1.0)
    o, (x, v, Ir, cell), phi, wf = seeded_dig_state(s, steps=40, **over)
    g = dig.Solver(s, "cuda:0", **over)
    g.write(x, v, Ir, cell)
    g.write_moments(dig.PHI_EWMA, phi)
    rg, ro = g.couple(), o.couple()
    converged_pair(rg, ro, 12000, 1e-12)
    for k in ("n_rejected", "n_reconstructed", "n_cloned", "n_deleted"):
        assert rg[k] == ro[k], (k, rg[k], ro[k])
    flags = o.read_couple(3)[:, 0]
    assert np.array_equal(g.read_couple(3)[:, 0], flags)
    assert (flags == 3).sum() > 0 and (flags == 2).sum() > 0 and (flags == 1).sum() > 0
    for which, tol in ((4, 1e-9), (0, 1e-9), (1, 1e-9), (2, 1e-8)):
        a, b = g.read_couple(which), o.read_couple(which)
        scale = np.abs(b).max(axis=0) + 1e-30
        assert np.all(np.abs(a - b) <= tol * scale), (which, np.abs(a - b).max(axis=0))
    assert np.array_equal(g.read()[3], o.read()[3])


def test_capsule_medium_size_properties():
    """The capsule at a medium size (about 0.4M tets, 20M particles), three
    steps: count bookkeeping, no particle over the crossing limit, sampled
    particles inside their tets, finite velocities and rotational energies."""
    s = W.capsule_scenario(0.1, 20_000_000, seed=5)
    g = dig.Solver(s, "cuda:0")
    g.init()
    n0 = g.count()
    g.step(3, dig.EWMA | dig.SYNC)
    c = g.counters()
    assert g.count() == n0 + c["injected"] - c["removed"] and c["stuck"] == 0 and c["lb"] > 0
    x, v, I, cell = g.read()
    k = np.random.default_rng(5).choice(len(cell), 4096, replace=False)
    P = s.mesh.nodes[s.mesh.tets[cell[k]]]
    T = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=2)
    lam = np.linalg.solve(T, (x[k] - P[:, 0])[..., None])[..., 0]
    assert np.concatenate([1.0 - lam.sum(axis=1, keepdims=True), lam], axis=1).min() >= -1e-9
    assert np.all(np.isfinite(v[k])) and np.all(np.isfinite(I[k])) and I[k].min() >= 0.0


def test_couple_open_boundaries_uniform_stream():
    """A uniform drifting stream between a free-stream inflow side, an outflow
    side and four specular walls is a fixed point of the GPU's synthetic solve
    too (both open-boundary kinds), within 1e-12 of the written state and of
    the oracle's result."""
    n, T, U = 1.677e22, 273.0, 300.0
    bcs = [dict(kind=W.BC_INFLOW, T=T, U=(U, 0.0, 0.0), n=n), dict(kind=W.BC_OUTFLOW, T=T, U=(0.0, 0.0, 0.0), n=0.0),
           dict(kind=W.BC_SPECULAR, T=T, U=(0.0, 0.0, 0.0), n=0.0)]
    mesh = W.box_sides(3, 1e-3, [0, 1, 2, 2, 2, 2], bcs)
    gas = W.ARGON
    mu = gas.mu_ref() * (T / gas.T_ref) ** gas.omega
    s = W.Scenario(gas=gas, mesh=mesh, n_particles=16200, n_init=n, T_init=T, u_init=(U, 0.0, 0.0),
                   F_N=n * 1e-9 / 16200, dt=0.2 * mu / (n * W.K_B * T), seed=7, L=1e-3, Kn=0.1, capacity=40000)
    g, o = pair(s, N_m=50, KnD_max=1e9)
    o.init()
    g.write(*o.read())
    vol = o.mesh_info()["vol"]
    kT_m = W.K_B * T / gas.mass
    N = n * vol / s.F_N
    phi = np.zeros((len(vol), orc.NPHI))
    phi[:, 0] = N
    phi[:, 1] = N * U
    phi[:, 4] = N * (kT_m + U * U)
    phi[:, 5] = N * kT_m
    phi[:, 6] = N * kT_m
    phi[:, 10] = N * U * (U * U + 5.0 * kT_m)
    g.write_moments(dig.PHI_EWMA, phi)
    o.write_moments(orc.PHI_EWMA, phi)
    rg, ro = g.couple(), o.couple()
    assert rg["iters"] == ro["iters"] == 50
    half, new = g.read_couple(0), g.read_couple(2)
    assert np.allclose(new, half, rtol=0, atol=1e-12), np.abs(new - half).max()
    assert np.allclose(new, o.read_couple(2), rtol=0, atol=1e-12)
    assert np.array_equal(g.read()[3], o.read()[3])


def test_surface_quantities_of_a_gas_at_rest():
    """dig_surface on a closed box of gas at rest at the wall temperature
    (diffuse walls): it converts the oracle's and the GPU's (identical)
    wall-flux sums into the number flux n c_mean / 4, the pressure n k T, zero
    shear and zero heat flux, box-wide means within 5 % of those values (about
    460,000 wall hits: the statistical error is near 0.2 %)."""
    s = W.Scenario(gas=W.ARGON, mesh=W.closed_box(1, 1e-3, W.BC_DIFFUSE), n_particles=60_000, n_init=1.677e22,
                   T_init=273.0, u_init=(0.0, 0.0, 0.0), F_N=1.677e22 * 1e-9 / 60_000, dt=6.7e-8, seed=21, L=1e-3,
                   Kn=0.1, capacity=120_000)
    g, o = pair(s)
    g.init()
    o.init()
    g.step(200, dig.WALLFLUX | dig.SYNC)
    o.step(200, orc.EWMA)
    assert_same_particles(g, o)
    surf = g.surface()
    mi = o.mesh_info()
    P = s.mesh.nodes[s.mesh.tets]
    wf = g.wall_flux()
    ib = 0
    t = 200 * s.dt
    for tt in range(len(s.mesh.tets)):
        for f in range(4):
            if mi["nbr"][tt, f] >= 0:
                continue
            q = [k for k in range(4) if k != f]
            A = 0.5 * np.linalg.norm(np.cross(P[tt, q[1]] - P[tt, q[0]], P[tt, q[2]] - P[tt, q[0]]))
            nrm = mi["normals"][tt, f]
            G = wf[ib, 1:4] / (A * t)
            p = G @ nrm
            exp = [wf[ib, 0] * s.F_N / (A * t), p, *(G - p * nrm), wf[ib, 4] / (A * t)]
            assert np.allclose(surf[ib], exp, rtol=1e-9, atol=1e-9 * np.abs(exp).max())
            ib += 1
    kT = W.K_B * s.T_init
    p_exact = s.n_init * kT
    flux_exact = s.n_init * math.sqrt(8.0 * kT / (math.pi * s.gas.mass)) / 4.0
    # the box's 12 faces have equal areas: face means are box-wide means
    assert abs(surf[:, 0].mean() - flux_exact) < 0.05 * flux_exact
    assert abs(surf[:, 1].mean() - p_exact) < 0.05 * p_exact
    assert np.abs(surf[:, 2:5].mean(axis=0)).max() < 0.05 * p_exact
    assert abs(surf[:, 5].mean()) < 0.05 * p_exact * math.sqrt(2 * kT / s.gas.mass)
