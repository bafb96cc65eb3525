"""ctypes wrapper of the CPU oracle (liborc.so).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py.  The product package never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liborc.so")

PHI_INST, PHI_EWMA, PHI_WINDOW, PHI_CUM, MACRO = 0, 1, 2, 3, 16
EWMA, WINDOW, CUMUL, RECORD_PAIRS = 1, 2, 4, 8
RESET_WINDOW, RESET_CUMUL, RESET_EWMA = 1, 2, 4
NPHI, NMAC = 17, 20
COUNTERS = ["steps", "cand", "coll", "cross", "wall", "removed", "injected", "stuck", "lb"]


class OrcConfig(C.Structure):
    _fields_ = [
        ("mass", C.c_double), ("d_ref", C.c_double), ("omega", C.c_double), ("T_ref", C.c_double),
        ("alpha", C.c_double), ("Z_rot", C.c_double), ("rot_dof", C.c_int32), ("max_cross", C.c_int32),
        ("F_N", C.c_double), ("dt", C.c_double), ("seed", C.c_uint64), ("n_init", C.c_double),
        ("T_init", C.c_double), ("u_init", C.c_double * 3), ("mu_ref", C.c_double), ("Kn", C.c_double),
        ("L_ref", C.c_double), ("n_a", C.c_int32), ("N_s", C.c_int32), ("N_m", C.c_int32),
        ("passes", C.c_int32), ("eps_m", C.c_double), ("KnD_max", C.c_double), ("capacity", C.c_int64),
        ("closure", C.c_int32), ("recon", C.c_int32),
        ("local_acc", C.c_int32), ("aa_m", C.c_int32), ("cfl", C.c_double),
    ]


class CoupleReport(C.Structure):
    _fields_ = [("iters", C.c_int32), ("n_learned", C.c_int32), ("residual", C.c_double), ("n_rejected", C.c_int64),
                ("n_reconstructed", C.c_int64), ("n_cloned", C.c_int64), ("n_deleted", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class OrcBC(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("T", C.c_double), ("U", C.c_double * 3),
                ("n", C.c_double)]


LIB64 = os.path.join(HERE, "liborc64.so")


def build(force: bool = False, v64: bool = False) -> str:
    """liborc.so (FP32 velocities, as the method states them), or with v64
    liborc64.so: the same oracle with FP64 velocities, rotational energies
    and collision, wall and injection arithmetic (the FP64 reference run)."""
    src = os.path.join(HERE, "orc.c")
    out = LIB64 if v64 else LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(HERE, "orc.h"))):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-D_DEFAULT_SOURCE", *(["-DORC_V64"] if v64 else []), "-fPIC", "-shared", "-Wall",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


_libs = {}


def lib(v64: bool = False):
    if v64 not in _libs:
        L = C.CDLL(build(v64=v64))
        P = C.c_void_p
        L.orc_create.restype = P
        L.orc_create.argtypes = [C.POINTER(OrcConfig)]
        L.orc_destroy.argtypes = [P]
        L.orc_last_error.restype = C.c_char_p
        L.orc_last_error.argtypes = [P]
        L.orc_mesh_load.argtypes = [P, P, C.c_int64, P, C.c_int64, P, P, C.c_int32]
        L.orc_particles_init.argtypes = [P, C.c_int64]
        L.orc_write_particles.argtypes = [P, P, P, P, P, C.c_int64]
        L.orc_read_particles.argtypes = [P, P, P, P, P, C.c_int64, P]
        L.orc_dsmc_step.argtypes = [P, C.c_int32, C.c_int32]
        L.orc_sample.argtypes = [P, C.c_int32]
        L.orc_read_moments.argtypes = [P, C.c_int32, P, C.c_int64]
        L.orc_read_pairs.argtypes = [P, P, P, P, P, P, C.c_int64, P]
        L.orc_read_counters.argtypes = [P, P, C.c_int32]
        L.orc_cell_state.argtypes = [P, P, P, C.c_int32]
        L.orc_wall_flux.argtypes = [P, P, C.c_int64, P]
        L.orc_step_index.restype = C.c_int64
        L.orc_step_index.argtypes = [P]
        L.orc_philox.argtypes = [P, P, P]
        L.orc_lnf.restype = C.c_float
        L.orc_lnf.argtypes = [C.c_float]
        L.orc_expf.restype = C.c_float
        L.orc_expf.argtypes = [C.c_float]
        L.orc_powf.restype = C.c_float
        L.orc_powf.argtypes = [C.c_float, C.c_float]
        L.orc_mesh_info.argtypes = [P, P, P, P, P, P]
        L.orc_locate.restype = C.c_int32
        L.orc_locate.argtypes = [P, P, C.c_double]
        L.orc_track_one.argtypes = [P, P, P, P, C.c_int64, C.c_int64]
        L.orc_sort_by_cell.argtypes = [P, C.c_int64, C.c_int32, P, P]
        L.orc_couple.argtypes = [P, P]
        L.orc_vss_directions.argtypes = [P, P, C.c_int64, P]
        L.orc_mlp_nparam.restype = C.c_int32
        L.orc_bf16.restype = C.c_double
        L.orc_bf16.argtypes = [C.c_double]
        L.orc_mlp_init.argtypes = [P, C.c_uint64]
        L.orc_mlp_forward.argtypes = [P, P, C.c_int64, C.c_int32, P]
        L.orc_mlp_grad.restype = C.c_double
        L.orc_mlp_grad.argtypes = [P, P, P, C.c_int64, C.c_int32, P]
        L.orc_adam.argtypes = [P, P, P, P, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_double]
        L.orc_read_couple.argtypes = [P, C.c_int32, P, C.c_int64]
        L.orc_write_moments.argtypes = [P, C.c_int32, P]
        L.orc_write_wall_flux.argtypes = [P, P, C.c_int64]
        L.orc_closure_set.argtypes = [P, P]
        L.orc_closure_features.argtypes = [P, C.c_int32, P]
        L.orc_closure_targets.argtypes = [P, C.c_int32, P, C.c_int64, P]
        L.orc_gradients.argtypes = [P, P, P]
        L.orc_nsf.argtypes = [P, P, P, P]
        L.orc_synthetic_solve.argtypes = [P, P, P, P, P, P, P]
        L.orc_synthetic_residual.argtypes = [P, P, P, P, P, P]
        _libs[v64] = L
    return _libs[v64]


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_p(c), _p(k), _p(o))
    return o


def make_config(scen, **over) -> OrcConfig:
    g = scen.gas
    cfg = OrcConfig()
    cfg.mass, cfg.d_ref, cfg.omega, cfg.T_ref = g.mass, g.d_ref, g.omega, g.T_ref
    cfg.alpha, cfg.Z_rot, cfg.rot_dof = g.alpha, g.Z_rot, g.rot_dof
    cfg.max_cross = 4096
    cfg.F_N, cfg.dt, cfg.seed = scen.F_N, scen.dt, scen.seed
    cfg.n_init, cfg.T_init = scen.n_init, scen.T_init
    for i in range(3):
        cfg.u_init[i] = scen.u_init[i]
    cfg.mu_ref = g.mu_ref()
    cfg.Kn, cfg.L_ref = scen.Kn, scen.L
    cfg.n_a, cfg.N_s, cfg.N_m, cfg.passes = 1000, 100, 500, 3
    cfg.eps_m, cfg.KnD_max = 1e-6, 1.0
    cfg.aa_m, cfg.cfl = 20, 1.5
    cfg.capacity = scen.capacity or 2 * scen.n_particles
    for k, v in over.items():
        setattr(cfg, k, v)
    return cfg


class Oracle:
    """One oracle simulation context on the host."""

    def __init__(self, scen, v64=False, **over):
        """v64: the FP64-velocity build (liborc64.so)."""
        self.scen = scen
        self.cfg = make_config(scen, **over)
        self.L = lib(v64)
        self.h = self.L.orc_create(C.byref(self.cfg))
        m = scen.mesh
        self.n_tets = len(m.tets)
        bcs = (OrcBC * max(1, len(m.bcs)))()
        for i, b in enumerate(m.bcs):
            bcs[i].kind, bcs[i].T, bcs[i].n = b["kind"], b["T"], b["n"]
            for q in range(3):
                bcs[i].U[q] = b["U"][q]
        nodes = np.ascontiguousarray(m.nodes, dtype=np.float64)
        tets = np.ascontiguousarray(m.tets, dtype=np.int32)
        tag = np.ascontiguousarray(m.face_tag, dtype=np.int32)
        self._check(self.L.orc_mesh_load(self.h, _p(nodes), len(nodes), _p(tets), len(tets), _p(tag),
                                         C.cast(bcs, C.c_void_p), len(m.bcs)))

    def _check(self, rc):
        if rc != 0:
            raise RuntimeError(f"oracle error {rc}: {self.L.orc_last_error(self.h).decode()}")

    def close(self):
        if self.h:
            self.L.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vss_directions(self, g):
        """Unit post-collision directions [n, 3] of the scattering law for the
        relative velocities g [n, 3] (non-zero), with this context's alpha."""
        g = np.ascontiguousarray(g, np.float32)
        e = np.zeros_like(g)
        self._check(self.L.orc_vss_directions(self.h, _p(g), len(g), _p(e)))
        return e

    def init(self, n=None):
        self._check(self.L.orc_particles_init(self.h, self.scen.n_particles if n is None else n))

    def write(self, x, v, Ir, cell):
        x = np.ascontiguousarray(x, np.float64)
        v = np.ascontiguousarray(v, np.float32)
        Ir = np.ascontiguousarray(Ir, np.float32)
        cell = np.ascontiguousarray(cell, np.int32)
        self._check(self.L.orc_write_particles(self.h, _p(x), _p(v), _p(Ir), _p(cell), len(cell)))

    def read(self):
        n = C.c_int64(0)
        self.L.orc_read_particles(self.h, None, None, None, None, 0, C.byref(n))
        N = n.value
        x = np.zeros((N, 3), np.float64)
        v = np.zeros((N, 3), np.float32)
        Ir = np.zeros(N, np.float32)
        cell = np.zeros(N, np.int32)
        self._check(self.L.orc_read_particles(self.h, _p(x), _p(v), _p(Ir), _p(cell), N, C.byref(n)))
        return x, v, Ir, cell

    def step(self, n=1, flags=EWMA):
        self._check(self.L.orc_dsmc_step(self.h, n, flags))

    def sample(self, action):
        self._check(self.L.orc_sample(self.h, action))

    def moments(self, which):
        k = NMAC if which & MACRO else NPHI
        out = np.zeros((self.n_tets, k), np.float64)
        self._check(self.L.orc_read_moments(self.h, which, _p(out), out.size))
        return out

    def pairs(self):
        n = C.c_int64(0)
        self.L.orc_read_pairs(self.h, None, None, None, None, None, 0, C.byref(n))
        N = n.value
        a = [np.zeros(N, np.int32) for _ in range(4)]
        acc = np.zeros(N, np.uint8)
        self._check(self.L.orc_read_pairs(self.h, *[_p(x) for x in a], _p(acc), N, C.byref(n)))
        return np.stack(a + [acc.astype(np.int32)], axis=1)

    def counters(self):
        out = np.zeros(len(COUNTERS), np.int64)
        self.L.orc_read_counters(self.h, _p(out), len(COUNTERS))
        return dict(zip(COUNTERS, out.tolist()))

    def cell_state(self, cmax=None, rem=None):
        if cmax is None:
            cm = np.zeros(self.n_tets, np.float32)
            rm = np.zeros(self.n_tets, np.float64)
            self.L.orc_cell_state(self.h, _p(cm), _p(rm), 0)
            return cm, rm
        cm = np.ascontiguousarray(cmax, np.float32)
        rm = np.ascontiguousarray(rem, np.float64)
        self.L.orc_cell_state(self.h, _p(cm), _p(rm), 1)

    def wall_flux(self):
        n = C.c_int64(0)
        self.L.orc_wall_flux(self.h, None, 0, C.byref(n))
        out = np.zeros((n.value, 5), np.float64)
        self._check(self.L.orc_wall_flux(self.h, _p(out), out.size, C.byref(n)))
        return out

    def mesh_info(self):
        n = self.n_tets
        nbr = np.zeros((n, 4), np.int32)
        nf = np.zeros((n, 4), np.int8)
        nrm = np.zeros((n, 4, 3), np.float64)
        d = np.zeros((n, 4), np.float64)
        vol = np.zeros(n, np.float64)
        nbf = self.L.orc_mesh_info(self.h, _p(nbr), _p(nf), _p(nrm), _p(d), _p(vol))
        return dict(nbr=nbr, nbr_face=nf, normals=nrm, d=d, vol=vol, n_bfaces=nbf)

    def locate(self, x, tol):
        x = np.ascontiguousarray(x, np.float64)
        return self.L.orc_locate(self.h, _p(x), tol)

    def track_one(self, x, v, cell, slot, step):
        x = np.array(x, np.float64)
        v = np.array(v, np.float32)
        c = np.array([cell], np.int32)
        self.L.orc_track_one(self.h, _p(x), _p(v), _p(c), slot, step)
        return x, v, int(c[0])

    def couple(self):
        r = CoupleReport()
        self._check(self.L.orc_couple(self.h, C.byref(r)))
        return r.as_dict()

    def read_couple(self, which):
        k = {0: 6, 1: 12, 2: 6, 3: 1, 4: 6, 5: 1}[which]
        out = np.zeros((self.n_tets, k), np.float64)
        self._check(self.L.orc_read_couple(self.h, which, _p(out), out.size))
        return out

    def write_moments(self, which, phi):
        phi = np.ascontiguousarray(phi, np.float64)
        assert phi.shape == (self.n_tets, NPHI)
        self._check(self.L.orc_write_moments(self.h, which, _p(phi)))

    def write_wall_flux(self, flux, steps):
        flux = np.ascontiguousarray(flux, np.float64)
        self._check(self.L.orc_write_wall_flux(self.h, _p(flux), steps))

    def closure_set(self, params):
        params = np.ascontiguousarray(params, np.float32)
        assert params.size == mlp_nparam()
        self._check(self.L.orc_closure_set(self.h, _p(params)))

    def closure_features(self, which):
        X = np.zeros((self.n_tets, 13), np.float32)
        self._check(self.L.orc_closure_features(self.h, which, _p(X)))
        return X

    def closure_targets(self, which, X):
        X = np.ascontiguousarray(X, np.float32)
        Y = np.zeros((len(X), 8), np.float32)
        self._check(self.L.orc_closure_targets(self.h, which, _p(X), len(X), _p(Y)))
        return Y

    # harness of the synthetic-equation pins (nondimensional rows per cell)
    def gradients(self, prim):
        prim = np.ascontiguousarray(prim, np.float64)
        assert prim.shape == (self.n_tets, 6)
        g = np.zeros((self.n_tets, 15), np.float64)
        self._check(self.L.orc_gradients(self.h, _p(prim), _p(g)))
        return g

    def nsf(self, prim, grad):
        prim = np.ascontiguousarray(prim, np.float64)
        grad = np.ascontiguousarray(grad, np.float64)
        out = np.zeros((self.n_tets, 12), np.float64)
        self._check(self.L.orc_nsf(self.h, _p(prim), _p(grad), _p(out)))
        return out

    def synthetic_solve(self, half, hot=None, src=None):
        half = np.ascontiguousarray(half, np.float64)
        hot = np.zeros((self.n_tets, 12)) if hot is None else np.ascontiguousarray(hot, np.float64)
        src = None if src is None else np.ascontiguousarray(src, np.float64)
        out = np.zeros((self.n_tets, 6), np.float64)
        it = C.c_int32(0)
        res = C.c_double(0.0)
        self._check(self.L.orc_synthetic_solve(self.h, _p(half), _p(hot), _p(src), _p(out), C.byref(it),
                                               C.byref(res)))
        return out, it.value, res.value

    def synthetic_residual(self, prim, hot=None, src=None):
        prim = np.ascontiguousarray(prim, np.float64)
        hot = np.zeros((self.n_tets, 12)) if hot is None else np.ascontiguousarray(hot, np.float64)
        src = None if src is None else np.ascontiguousarray(src, np.float64)
        R = np.zeros((self.n_tets, 6), np.float64)
        dtl = np.zeros(self.n_tets, np.float64)
        self._check(self.L.orc_synthetic_residual(self.h, _p(prim), _p(hot), _p(src), _p(R), _p(dtl)))
        return R, dtl

    @property
    def step_index(self):
        return self.L.orc_step_index(self.h)


def lnf(x):
    return lib().orc_lnf(float(x))


def expf(x):
    return lib().orc_expf(float(x))


def powf(x, a):
    return lib().orc_powf(float(x), float(a))


def sort_by_cell(cell, n_cells):
    """Stable counting sort by cell; -1 entries are dropped."""
    cell = np.ascontiguousarray(cell, np.int32)
    cs = np.zeros(n_cells + 1, np.int32)
    order = np.zeros(max(1, int((cell >= 0).sum())), np.int32)
    rc = lib().orc_sort_by_cell(_p(cell), len(cell), n_cells, _p(cs), _p(order))
    if rc != 0:
        raise ValueError("orc_sort_by_cell: bad input")
    return cs, order[: cs[-1]]


# ------------------------------------------------------------- learned closure
def mlp_nparam():
    return lib().orc_mlp_nparam()


def mlp_init(seed):
    p = np.zeros(mlp_nparam(), np.float32)
    lib().orc_mlp_init(_p(p), seed)
    return p


def mlp_forward(params, X, bf16=True):
    params = np.ascontiguousarray(params, np.float32)
    X = np.ascontiguousarray(X, np.float32)
    Y = np.zeros((len(X), 8), np.float64)
    lib().orc_mlp_forward(_p(params), _p(X), len(X), int(bf16), _p(Y))
    return Y


def mlp_grad(params, X, T, bf16=True):
    params = np.ascontiguousarray(params, np.float32)
    X = np.ascontiguousarray(X, np.float32)
    T = np.ascontiguousarray(T, np.float32)
    g = np.zeros(mlp_nparam(), np.float64)
    loss = lib().orc_mlp_grad(_p(params), _p(X), _p(T), len(X), int(bf16), _p(g))
    return loss, g


def adam(params, m, v, g, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    lib().orc_adam(_p(params), _p(m), _p(v), _p(np.ascontiguousarray(g, np.float64)), t, lr, b1, b2, eps)


def bf16(x):
    return lib().orc_bf16(float(x))
