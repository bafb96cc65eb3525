"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds no step of the DSMC/DIG method itself: it builds the procedural
meshes (node coordinates, tetrahedra, boundary tags) and the scenario parameters
(gas constants, number density, time step, particle weight) that both sides take
as inputs.  Everything is plain numpy; nothing here touches a GPU.

Workloads (lid-driven cavity, paper Sec. 5.1, rescaled to a 1 mm argon cube):

* ``cavity(nh)``: the cube [-L/2, L/2]^3 split into nh^3 hexahedra, each cut into
  six Kuhn (Freudenthal) tetrahedra along its (0,0,0)-(1,1,1) diagonal, so the
  triangulation is conforming across hexahedra.  All six walls are diffuse at
  T_w; the wall y = +L/2 moves with velocity (U_w, 0, 0).
* ``open_box(nh)``: the same mesh with every boundary face a free-stream inflow
  face (used for the injection/outflow checks).

Hypersonic sphere (paper Sec. 5.2's sphere, procedural): ``sphere_mesh`` builds a
Delaunay triangulation of seeded points on concentric shells graded toward the
body; the far field is a free-stream face set, the body a diffuse wall.
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

K_B = 1.380649e-23  # J/K

# boundary-condition kinds (same integer values in include/dig.h and the oracle header)
BC_DIFFUSE, BC_SPECULAR, BC_INFLOW, BC_OUTFLOW = 0, 1, 2, 3


@dataclasses.dataclass
class Gas:
    mass: float
    d_ref: float
    omega: float
    T_ref: float
    rot_dof: int = 0
    Z_rot: float = 1.0
    alpha: float = 1.0

    def mu_ref(self) -> float:
        """Viscosity at T_ref, the scenario's mu_0: the VHS value (Bird 1994,
        eq. 4.62) times (alpha + 1)(alpha + 2) / (6 alpha) for a VSS gas, the
        ratio of the VHS viscosity cross section (2/3 of the total) to the VSS
        one (4 alpha / ((alpha + 1)(alpha + 2)) of the total)."""
        w = self.omega
        mu = 15.0 * math.sqrt(math.pi * self.mass * K_B * self.T_ref) / (
            2.0 * math.pi * self.d_ref ** 2 * (5.0 - 2.0 * w) * (7.0 - 2.0 * w))
        a = self.alpha
        if a != 1.0:
            mu *= (a + 1.0) * (a + 2.0) / (6.0 * a)
        return mu


ARGON = Gas(mass=6.63e-26, d_ref=4.17e-10, omega=0.81, T_ref=273.0)
NITROGEN = Gas(mass=4.65e-26, d_ref=4.17e-10, omega=0.74, T_ref=273.0, rot_dof=2, Z_rot=5.0)
# VSS parameters of Bird 1994, Table A1
ARGON_VSS = Gas(mass=6.63e-26, d_ref=4.11e-10, omega=0.81, T_ref=273.0, alpha=1.40)
NITROGEN_VSS = Gas(mass=4.65e-26, d_ref=4.11e-10, omega=0.74, T_ref=273.0, rot_dof=2, Z_rot=5.0, alpha=1.36)


@dataclasses.dataclass
class Mesh:
    nodes: np.ndarray      # [n_nodes, 3] float64
    tets: np.ndarray       # [n_tets, 4] int32
    face_tag: np.ndarray   # [n_tets, 4] int32: -1 interior, else index into bcs; face f is opposite vertex f
    bcs: list              # list of dicts: kind, T, U(3), n


def kuhn_cube(nh: int, L: float):
    """Nodes and Kuhn tetrahedra of the cube [-L/2, L/2]^3 cut into nh^3 hexahedra."""
    g = np.linspace(-0.5 * L, 0.5 * L, nh + 1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    nodes = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float64)

    def nid(i, j, k):
        return (i * (nh + 1) + j) * (nh + 1) + k

    i, j, k = np.meshgrid(np.arange(nh), np.arange(nh), np.arange(nh), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    tets = []
    for perm in itertools.permutations(range(3)):
        # path v000 -> +e_p0 -> +e_p0+e_p1 -> v111
        off = np.zeros((4, 3), dtype=np.int64)
        off[1, perm[0]] = 1
        off[2] = off[1]
        off[2, perm[1]] = 1
        off[3] = 1
        tets.append(np.stack([nid(i + o[0], j + o[1], k + o[2]) for o in off], axis=1))
    # hex-major order: the six tets of one hex are consecutive
    tets = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return nodes, tets


def boundary_side(nodes, tets, L):
    """For each (tet, local face) the cube side it lies on (0..5 = -x,+x,-y,+y,-z,+z) or -1."""
    h = 0.5 * L
    side = np.full(tets.shape, -1, dtype=np.int32)
    for f in range(4):
        verts = [tets[:, v] for v in range(4) if v != f]
        P = np.stack([nodes[v] for v in verts], axis=1)  # [n, 3 verts, 3 coords]
        for ax in range(3):
            for s, val in ((0, -h), (1, h)):
                on = np.all(np.abs(P[:, :, ax] - val) <= 1e-12 * L, axis=1)
                side[on, f] = 2 * ax + s
    return side


def cavity(nh: int, L: float = 1e-3, T_w: float = 273.0, U_lid: float = 50.0) -> Mesh:
    nodes, tets = kuhn_cube(nh, L)
    side = boundary_side(nodes, tets, L)
    face_tag = np.where(side < 0, -1, 0).astype(np.int32)
    face_tag[side == 3] = 1  # lid y = +L/2
    bcs = [dict(kind=BC_DIFFUSE, T=T_w, U=(0.0, 0.0, 0.0), n=0.0),
           dict(kind=BC_DIFFUSE, T=T_w, U=(U_lid, 0.0, 0.0), n=0.0)]
    return Mesh(nodes, tets, face_tag, bcs)


def closed_box(nh: int, L: float = 1e-3, kind: int = BC_SPECULAR, T_w: float = 273.0) -> Mesh:
    nodes, tets = kuhn_cube(nh, L)
    side = boundary_side(nodes, tets, L)
    face_tag = np.where(side < 0, -1, 0).astype(np.int32)
    bcs = [dict(kind=kind, T=T_w, U=(0.0, 0.0, 0.0), n=0.0)]
    return Mesh(nodes, tets, face_tag, bcs)


def open_box(nh: int, L: float, n_inf: float, T_inf: float, U_inf=(0.0, 0.0, 0.0)) -> Mesh:
    nodes, tets = kuhn_cube(nh, L)
    side = boundary_side(nodes, tets, L)
    face_tag = np.where(side < 0, -1, 0).astype(np.int32)
    bcs = [dict(kind=BC_INFLOW, T=T_inf, U=tuple(U_inf), n=n_inf)]
    return Mesh(nodes, tets, face_tag, bcs)


def box_sides(nh: int, L: float, side_bc, bcs) -> Mesh:
    """Cube whose six sides (0..5 = -x,+x,-y,+y,-z,+z) carry bcs[side_bc[side]]."""
    nodes, tets = kuhn_cube(nh, L)
    side = boundary_side(nodes, tets, L)
    face_tag = np.full(tets.shape, -1, dtype=np.int32)
    for sd in range(6):
        face_tag[side == sd] = side_bc[sd]
    return Mesh(nodes, tets, face_tag, list(bcs))


def _shell_points(n: int, r: float, rng: np.random.Generator) -> np.ndarray:
    """n points spread evenly over the sphere of radius r (Fibonacci lattice),
    turned by a random rotation (random unit quaternion)."""
    i = np.arange(n) + 0.5
    phi = np.arccos(1.0 - 2.0 * i / n)
    th = math.pi * (1.0 + 5.0 ** 0.5) * i
    p = np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], axis=1)
    a, b, c, d = rng.standard_normal(4)
    q = math.sqrt(a * a + b * b + c * c + d * d)
    a, b, c, d = a / q, b / q, c / q, d / q
    rot = np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                    [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                    [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])
    return r * (p @ rot.T)


def sphere_mesh(h_w: float, R: float = 0.1, R_far: float = 1.0, grading: float = 20.0, seed: int = 4,
                T_w: float = 500.0, n_inf: float = 1e21, T_inf: float = 200.0, U_inf=(2635.0, 0.0, 0.0)) -> Mesh:
    """Sphere of radius R in a spherical far field of radius R_far: Delaunay
    tetrahedra of a seeded point cloud on concentric shells whose spacing grows
    geometrically from h_w at the body to grading * h_w at the far field; the
    tetrahedra inside the body are removed.  Boundary faces nearer the body than
    the far field are the body wall (diffuse at T_w, bcs[0]); the others are
    free-stream faces (n_inf, T_inf, U_inf; bcs[1])."""
    import os
    import tempfile

    from scipy.spatial import Delaunay

    bcs = [dict(kind=BC_DIFFUSE, T=T_w, U=(0.0, 0.0, 0.0), n=0.0),
           dict(kind=BC_INFLOW, T=T_inf, U=tuple(U_inf), n=n_inf)]
    # the triangulation of a large point cloud takes a minute: cached per parameters
    cache = os.path.join(os.environ.get("DIG_MESH_CACHE", tempfile.gettempdir()),
                         f"dig_sphere_{h_w:.6g}_{R:.6g}_{R_far:.6g}_{grading:.6g}_{seed}.npz")
    if os.path.exists(cache):
        z = np.load(cache)
        return Mesh(z["nodes"], z["tets"], z["face_tag"], bcs)
    rng = np.random.default_rng(seed)
    a = math.log(grading) / math.log(R_far / R)
    radii = [R]
    while True:
        h = h_w * (radii[-1] / R) ** a
        if radii[-1] + h >= R_far - 0.3 * h:
            break
        radii.append(radii[-1] + h)
    radii.append(R_far)
    pts = []
    for r in radii:
        h = h_w * (r / R) ** a
        pts.append(_shell_points(max(12, int(round(4.0 * math.pi * r * r / (0.866 * h * h)))), r, rng))
    nodes = np.concatenate(pts).astype(np.float64)
    tets = Delaunay(nodes).simplices.astype(np.int64)
    tets = tets[np.linalg.norm(nodes[tets].mean(axis=1), axis=1) > R]
    # boundary faces: the faces (opposite vertex f) that no other kept tet shares
    nt = len(tets)
    tri = np.stack([np.delete(tets, f, axis=1) for f in range(4)], axis=1).reshape(-1, 3)
    tri.sort(axis=1)
    key = (tri[:, 0] * (len(nodes) + 1) + tri[:, 1]) * (len(nodes) + 1) + tri[:, 2]
    order = np.argsort(key, kind="stable")
    ks = key[order]
    dup = np.zeros(len(ks), bool)
    dup[1:] |= ks[1:] == ks[:-1]
    dup[:-1] |= ks[:-1] == ks[1:]
    boundary = np.empty(len(ks), bool)
    boundary[order] = ~dup
    boundary = boundary.reshape(nt, 4)
    fc = np.stack([nodes[np.delete(tets, f, axis=1)].mean(axis=1) for f in range(4)], axis=1)
    far = np.linalg.norm(fc, axis=2) > 0.5 * (R + R_far)
    face_tag = np.where(boundary, np.where(far, 1, 0), -1).astype(np.int32)
    tets = tets.astype(np.int32)
    try:
        tmp = cache + f".{os.getpid()}.npz"
        np.savez(tmp, nodes=nodes, tets=tets, face_tag=face_tag)
        os.replace(tmp, cache)
    except OSError:
        pass
    return Mesh(nodes, tets, face_tag, bcs)


# capsule body (the paper's Apollo case, Sec. 5.3, procedural): spherical cap
# of radius 2 m meeting a 33-degree conical frustum at the base radius 1.95 m;
# the frustum narrows to a flat top of radius 0.5 m.  Axis x, cap toward -x.
CAPSULE_RC, CAPSULE_RB, CAPSULE_CONE_DEG, CAPSULE_RTOP = 2.0, 1.95, 33.0, 0.5


def _capsule_geometry():
    a_c = math.sqrt(CAPSULE_RC ** 2 - CAPSULE_RB ** 2)  # cap centre on the axis
    tc = math.tan(math.radians(CAPSULE_CONE_DEG))
    a_top = (CAPSULE_RB - CAPSULE_RTOP) / tc
    a_min = a_c - CAPSULE_RC
    return a_c, tc, a_top, a_min, 0.5 * (a_min + a_top)


def capsule_inside(p: np.ndarray) -> np.ndarray:
    """True for points inside the capsule body."""
    a_c, tc, a_top, a_min, _ = _capsule_geometry()
    a = p[:, 0]
    r = np.hypot(p[:, 1], p[:, 2])
    cap = (a <= 0.0) & (a >= a_min) & ((a - a_c) ** 2 + r ** 2 <= CAPSULE_RC ** 2)
    cone = (a > 0.0) & (a <= a_top) & (r <= CAPSULE_RB - a * tc)
    return cap | cone


def _capsule_meridian(h: float, s: float) -> np.ndarray:
    """(a, r) points along the body's meridian scaled by s about the body's
    mid-axis point, spacing about h: cap arc, frustum line, top radius."""
    a_c, tc, a_top, a_min, c0 = _capsule_geometry()
    th_max = math.asin(CAPSULE_RB / CAPSULE_RC)
    pts = []
    n = max(2, int(math.ceil(s * CAPSULE_RC * th_max / h)))
    pts += [(a_c - CAPSULE_RC * math.cos(th_max * i / n), CAPSULE_RC * math.sin(th_max * i / n)) for i in range(n)]
    n = max(2, int(math.ceil(s * math.hypot(a_top, CAPSULE_RB - CAPSULE_RTOP) / h)))
    pts += [(a_top * i / n, CAPSULE_RB - (CAPSULE_RB - CAPSULE_RTOP) * i / n) for i in range(n)]
    n = max(2, int(math.ceil(s * CAPSULE_RTOP / h)))
    pts += [(a_top, CAPSULE_RTOP * (1.0 - i / n)) for i in range(n + 1)]
    m = np.array(pts)
    m[:, 0] = c0 + s * (m[:, 0] - c0)
    m[:, 1] *= s
    return m


def capsule_mesh(h_w: float, R_far: float = 15.6, grading: float = 20.0, seed: int = 5, T_w: float = 500.0,
                 n_inf: float = 1e20, T_inf: float = 142.2, U_inf=(6000.0, 0.0, 0.0)) -> Mesh:
    """Capsule in a spherical far field of radius R_far about the body's
    mid-axis point: Delaunay tetrahedra of seeded points on copies of the body
    surface scaled about that point (spacing growing from h_w at the body
    toward grading * h_w at the far field; each surface of revolution sampled
    along its meridian and around the axis with a random phase) and on the far
    sphere; tetrahedra inside the body removed.  Boundary faces nearer the
    body than half the far-field radius are the body wall (diffuse at T_w,
    bcs[0]); the others are free-stream faces (bcs[1])."""
    import os
    import tempfile

    from scipy.spatial import Delaunay

    bcs = [dict(kind=BC_DIFFUSE, T=T_w, U=(0.0, 0.0, 0.0), n=0.0),
           dict(kind=BC_INFLOW, T=T_inf, U=tuple(U_inf), n=n_inf)]
    cache = os.path.join(os.environ.get("DIG_MESH_CACHE", tempfile.gettempdir()),
                         f"dig_capsule_{h_w:.6g}_{R_far:.6g}_{grading:.6g}_{seed}.npz")
    if os.path.exists(cache):
        z = np.load(cache)
        return Mesh(z["nodes"], z["tets"], z["face_tag"], bcs)
    rng = np.random.default_rng(seed)
    _, _, _, _, c0 = _capsule_geometry()
    R_eq = 2.0
    a = math.log(grading) / math.log(R_far / R_eq)
    h_far = h_w * (R_far / R_eq) ** a
    pts = []
    s = 1.0
    while True:
        h = h_w * s ** a
        for am, rm in _capsule_meridian(h, s):
            n = max(1, int(round(2.0 * math.pi * rm / h))) if rm > 1e-12 else 1
            t = rng.uniform(0.0, 2.0 * math.pi) + 2.0 * math.pi * np.arange(n) / n
            pts.append(np.stack([np.full(n, am), rm * np.cos(t), rm * np.sin(t)], axis=1))
        s_next = s + h / R_eq
        if s_next * 2.4 > R_far - h_far:
            break
        s = s_next
    far = _shell_points(max(12, int(round(4.0 * math.pi * R_far ** 2 / (0.866 * h_far * h_far)))), R_far, rng)
    far[:, 0] += c0
    pts.append(far)
    nodes = np.concatenate(pts).astype(np.float64)
    tets = Delaunay(nodes).simplices.astype(np.int64)
    tets = tets[~capsule_inside(nodes[tets].mean(axis=1))]
    nt = len(tets)
    tri = np.stack([np.delete(tets, f, axis=1) for f in range(4)], axis=1).reshape(-1, 3)
    tri.sort(axis=1)
    key = (tri[:, 0] * (len(nodes) + 1) + tri[:, 1]) * (len(nodes) + 1) + tri[:, 2]
    order = np.argsort(key, kind="stable")
    ks = key[order]
    dup = np.zeros(len(ks), bool)
    dup[1:] |= ks[1:] == ks[:-1]
    dup[:-1] |= ks[:-1] == ks[1:]
    boundary = np.empty(len(ks), bool)
    boundary[order] = ~dup
    boundary = boundary.reshape(nt, 4)
    fc = np.stack([nodes[np.delete(tets, f, axis=1)].mean(axis=1) for f in range(4)], axis=1)
    fc[..., 0] -= c0
    far_face = np.linalg.norm(fc, axis=2) > 0.5 * R_far
    face_tag = np.where(boundary, np.where(far_face, 1, 0), -1).astype(np.int32)
    tets = tets.astype(np.int32)
    try:
        tmp = cache + f".{os.getpid()}.npz"
        np.savez(tmp, nodes=nodes, tets=tets, face_tag=face_tag)
        os.replace(tmp, cache)
    except OSError:
        pass
    return Mesh(nodes, tets, face_tag, bcs)


@dataclasses.dataclass
class Scenario:
    """Everything a run needs besides the mesh; the same values feed both sides."""
    gas: Gas
    mesh: Mesh
    n_particles: int
    n_init: float          # number density of the initial state, 1/m^3
    T_init: float
    u_init: tuple
    F_N: float             # real molecules per simulation particle
    dt: float              # s
    seed: int
    L: float
    Kn: float
    capacity: int = 0      # particle capacity (0: 2x n_particles)
    name: str = ""


def cavity_scenario(nh: int, n_particles: int, Kn: float, seed: int, L: float = 1e-3,
                    gas: Gas = ARGON, T0: float = 273.0, U_lid: float = 50.0,
                    dt_factor: float = 0.2, name: str = "") -> Scenario:
    """Cavity at global Knudsen number Kn (paper eq. for Kn: mu0/(p0 L) sqrt(pi R T0 / 2)).

    dt = dt_factor * mu0/p0 (the paper's mean collision time tau = mu/p_t)."""
    mu0 = gas.mu_ref() * (T0 / gas.T_ref) ** gas.omega
    R = K_B / gas.mass
    p0 = mu0 / (Kn * L) * math.sqrt(math.pi * R * T0 / 2.0)
    n0 = p0 / (K_B * T0)
    F_N = n0 * L ** 3 / n_particles
    dt = dt_factor * mu0 / p0
    mesh = cavity(nh, L=L, T_w=T0, U_lid=U_lid)
    return Scenario(gas=gas, mesh=mesh, n_particles=n_particles, n_init=n0, T_init=T0,
                    u_init=(0.0, 0.0, 0.0), F_N=F_N, dt=dt, seed=seed, L=L, Kn=Kn,
                    capacity=2 * n_particles, name=name or f"cavity{nh}")


# The five configurations used by the tests and the bench.
def config_small(seed: int = 1) -> Scenario:
    """Argon cavity, 6^3 hexes x 6 tets = 1,296 tets, Kn = 0.1, 20,000 particles."""
    return cavity_scenario(6, 20_000, 0.1, seed, name="cavity-6x6x6-Kn0.1-20k")


def config_c2(seed: int = 2) -> Scenario:
    """Argon cavity, 30^3 hexes x 6 tets = 162,000 tets, Kn = 0.01, 8M particles."""
    return cavity_scenario(30, 8_000_000, 0.01, seed, name="cavity-30x30x30-Kn0.01-8M")


def config_c3(seed: int = 3) -> Scenario:
    """Argon cavity, 20^3 hexes x 6 tets = 48,000 tets, Kn = 0.001, 3M particles."""
    return cavity_scenario(20, 3_000_000, 0.001, seed, name="cavity-20x20x20-Kn0.001-3M")


def sphere_scenario(h_w: float, n_particles: int, seed: int = 4, gas: Gas = ARGON, R: float = 0.1,
                    R_far: float = 1.0, n_inf: float = 1e21, T_inf: float = 200.0, U: float = 2635.0,
                    T_w: float = 500.0, name: str = "") -> Scenario:
    """Hypersonic argon over a sphere (Mach 10 at 200 K: U = 2635 m/s along +x,
    n = 1e21 m^-3, diffuse wall at 500 K), initial state the free stream.
    dt = min(0.2 tau, 0.2 h_w / (U + 3 sqrt(2 k T / m))) with tau = mu / p of
    the free stream; L_ref = 2R and Kn from the cavity's Kn definition."""
    mesh = sphere_mesh(h_w, R=R, R_far=R_far, seed=seed, T_w=T_w, n_inf=n_inf, T_inf=T_inf, U_inf=(U, 0.0, 0.0))
    mu = gas.mu_ref() * (T_inf / gas.T_ref) ** gas.omega
    p = n_inf * K_B * T_inf
    dt = min(0.2 * mu / p, 0.2 * h_w / (U + 3.0 * math.sqrt(2.0 * K_B * T_inf / gas.mass)))
    P = mesh.nodes[mesh.tets]
    V = float(np.abs(np.einsum("ni,ni->n", P[:, 1] - P[:, 0], np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]))).sum()) / 6.0
    L = 2.0 * R
    Kn = mu / (p * L) * math.sqrt(math.pi * K_B / gas.mass * T_inf / 2.0)
    return Scenario(gas=gas, mesh=mesh, n_particles=n_particles, n_init=n_inf, T_init=T_inf, u_init=(U, 0.0, 0.0),
                    F_N=n_inf * V / n_particles, dt=dt, seed=seed, L=L, Kn=Kn, capacity=2 * n_particles,
                    name=name or f"sphere-{len(mesh.tets)}tets")


def config_c4(seed: int = 4) -> Scenario:
    """Hypersonic argon sphere: R = 0.1 m, far field 1 m, ~2M tets graded 20x toward the wall, 100M particles."""
    return sphere_scenario(0.0036, 100_000_000, seed, name="sphere-R0.1-Ma10-2Mtets-100M")


def capsule_scenario(h_w: float, n_particles: int, seed: int = 5, gas: Gas = NITROGEN, Ma: float = 25.0,
                     T_inf: float = 142.2, Kn: float = 0.01, incidence_deg: float = 20.0, T_w: float = 500.0,
                     name: str = "") -> Scenario:
    """Nitrogen (Borgnakke-Larsen, Z_rot = 5) at Mach 25 over the capsule at
    20 degrees incidence: free stream at 142.2 K with the number density that
    gives Kn = 0.01 on the diameter L = 3.9 m (the cavity's Kn definition),
    diffuse wall at 500 K, initial state the free stream.
    dt = min(0.2 tau, 0.2 h_w / (U + 3 sqrt(2 k T / m)))."""
    R = K_B / gas.mass
    gam = (5.0 + gas.rot_dof) / (3.0 + gas.rot_dof)
    U = Ma * math.sqrt(gam * R * T_inf)
    inc = math.radians(incidence_deg)
    Uv = (U * math.cos(inc), U * math.sin(inc), 0.0)
    L = 2.0 * CAPSULE_RB
    mu = gas.mu_ref() * (T_inf / gas.T_ref) ** gas.omega
    p = mu / (Kn * L) * math.sqrt(math.pi * R * T_inf / 2.0)
    n_inf = p / (K_B * T_inf)
    mesh = capsule_mesh(h_w, seed=seed, T_w=T_w, n_inf=n_inf, T_inf=T_inf, U_inf=Uv)
    dt = min(0.2 * mu / p, 0.2 * h_w / (U + 3.0 * math.sqrt(2.0 * K_B * T_inf / gas.mass)))
    P = mesh.nodes[mesh.tets]
    V = float(np.abs(np.einsum("ni,ni->n", P[:, 1] - P[:, 0], np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]))).sum()) / 6.0
    return Scenario(gas=gas, mesh=mesh, n_particles=n_particles, n_init=n_inf, T_init=T_inf, u_init=Uv,
                    F_N=n_inf * V / n_particles, dt=dt, seed=seed, L=L, Kn=Kn,
                    capacity=int(1.25 * n_particles), name=name or f"capsule-{len(mesh.tets)}tets")


def config_c5(seed: int = 5) -> Scenario:
    """Nitrogen capsule at Mach 25, 20 degrees incidence: ~8M tets graded 20x
    toward the body, 1e9 particles (44 GB of particle state per buffer set)."""
    return capsule_scenario(0.0365, 1_000_000_000, seed, name="capsule-Ma25-8Mtets-1G")


def random_particles(rng: np.random.Generator, scen: Scenario, n: int):
    """Arbitrary test states: uniform points inside random tets, Maxwellian velocities.

    Returns (x[n,3] f64, v[n,3] f32, Ir[n] f32, cell[n] i32); order is random."""
    m = scen.mesh
    cell = rng.integers(0, len(m.tets), size=n).astype(np.int32)
    w = rng.dirichlet(np.ones(4), size=n)
    P = m.nodes[m.tets[cell]]  # [n, 4, 3]
    x = np.einsum("nk,nkc->nc", w, P)
    s = math.sqrt(K_B * scen.T_init / scen.gas.mass)
    v = (rng.standard_normal((n, 3)) * s).astype(np.float32)
    Ir = (rng.exponential(scen.T_init, size=n)).astype(np.float32)
    return x, v, Ir, cell


def particles_per_cell(rng: np.random.Generator, scen: Scenario, k: int):
    """Exactly k particles in every tet (uniform points, Maxwellian velocities
    at T_init, zero rotational energy), cell-major order.

    Returns (x f64 [n,3], v f32 [n,3], Ir f32 [n], cell i32 [n]), n = k * n_tets."""
    m = scen.mesh
    cell = np.repeat(np.arange(len(m.tets), dtype=np.int32), k)
    w = rng.dirichlet(np.ones(4), size=len(cell))
    x = np.einsum("nk,nkc->nc", w, m.nodes[m.tets[cell]])
    s = math.sqrt(K_B * scen.T_init / scen.gas.mass)
    v = (rng.standard_normal((len(cell), 3)) * s).astype(np.float32)
    return x, v, np.zeros(len(cell), np.float32), cell
