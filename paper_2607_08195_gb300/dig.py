"""Thin Python binding of libdig.so (include/dig.h).

Argument marshalling only: every step of the particle loop runs in the CUDA
kernels of libdig.so.  PyTorch supplies the device memory (one uint8 tensor,
the arena) and the stream.  There is no CPU fallback: without the compiled
library or a CUDA device the constructor raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdig.so")

EWMA, WINDOW, CUMUL, RECORD_PAIRS, INST, WALLFLUX, SYNC, TIMING = 1, 2, 4, 8, 16, 32, 64, 128
RESET_WINDOW, RESET_CUMUL, RESET_EWMA = 1, 2, 4
PHI_INST, PHI_EWMA, PHI_WINDOW, PHI_CUM, MACRO = 0, 1, 2, 3, 16
NPHI, NMAC = 17, 20
COUNTERS = ["steps", "cand", "coll", "cross", "wall", "removed", "injected", "stuck", "lb"]
ERRORS = {-1: "DIG_ERR_ARG", -2: "DIG_ERR_MESH", -3: "DIG_ERR_CAPACITY", -4: "DIG_ERR_STUCK",
          -5: "DIG_ERR_SOLVE", -6: "DIG_ERR_CUDA", -7: "DIG_ERR_STATE", -8: "DIG_ERR_TIMEOUT"}


class DigError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class DigConfig(C.Structure):
    _fields_ = [
        ("mass", C.c_double), ("d_ref", C.c_double), ("omega", C.c_double), ("T_ref", C.c_double),
        ("alpha", C.c_double), ("Z_rot", C.c_double), ("rot_dof", C.c_int32), ("max_cross", C.c_int32),
        ("F_N", C.c_double), ("dt", C.c_double), ("seed", C.c_uint64), ("n_init", C.c_double),
        ("T_init", C.c_double), ("u_init", C.c_double * 3), ("mu_ref", C.c_double), ("Kn", C.c_double),
        ("L_ref", C.c_double), ("n_a", C.c_int32), ("N_s", C.c_int32), ("N_m", C.c_int32),
        ("passes", C.c_int32), ("eps_m", C.c_double), ("KnD_max", C.c_double), ("capacity", C.c_int64),
        ("wait_timeout_s", C.c_double), ("stage_cap", C.c_int32), ("tile_cells", C.c_int32),
        ("cta_threads", C.c_int32), ("closure", C.c_int32), ("recon", C.c_int32), ("local_acc", C.c_int32),
        ("aa_m", C.c_int32), ("cfl", C.c_double),
    ]


class CoupleReport(C.Structure):
    _fields_ = [("iters", C.c_int32), ("n_learned", C.c_int32), ("residual", C.c_double), ("n_rejected", C.c_int64),
                ("n_reconstructed", C.c_int64), ("n_cloned", C.c_int64), ("n_deleted", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TrainConfig(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("eps", C.c_double), ("perm", C.c_void_p)]


MLP_NIN, MLP_NOUT, MLP_NPARAM = 13, 8, 9736
CLOSURE_YMAX = 4.0


class DigBC(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("T", C.c_double), ("U", C.c_double * 3),
                ("n", C.c_double)]


# every symbol include/dig.h declares
EXPORTS = ["dig_create", "dig_destroy", "dig_last_error", "dig_set_stream", "mesh_load", "dig_arena_bytes",
           "dig_bind_arena", "particles_init", "write_particles", "read_particles", "dsmc_step", "sample",
           "read_moments", "read_pairs", "read_counters", "dig_cell_state", "dig_wall_flux",
           "dig_particle_count", "dig_synchronize", "dig_launch_count", "dig_kernel_time",
           "dig_sort_scratch_bytes", "dig_sort_by_cell", "dig_sort_by_cell_noalloc", "dig_couple",
           "dig_read_couple", "dig_write_moments", "dig_write_wall_flux", "closure_init", "closure_set",
           "closure_get", "closure_features", "closure_targets", "closure_forward", "closure_loss", "closure_grad",
           "closure_train", "dig_checkpoint_bytes", "dig_save", "dig_load", "dig_surface",
           "dig_test_forward_timeout"]

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libdig.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not built: run paper_2607_08195_gb300.build.build() (needs nvcc)")
    L = C.CDLL(path)
    P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
    sig = {
        "dig_create": [P, P], "dig_destroy": [P], "dig_set_stream": [P, P],
        "mesh_load": [P, P, I64, P, I64, P, P, I32], "dig_arena_bytes": [P, P],
        "dig_bind_arena": [P, P, I64], "particles_init": [P, I64],
        "write_particles": [P, P, P, P, P, I64], "read_particles": [P, P, P, P, P, I64, P],
        "dsmc_step": [P, I32, I32], "sample": [P, I32], "read_moments": [P, I32, P, I64],
        "read_pairs": [P, P, P, P, P, P, I64, P], "read_counters": [P, P, I32],
        "dig_cell_state": [P, P, P, I32], "dig_wall_flux": [P, P, I64, P], "dig_particle_count": [P, P],
        "dig_synchronize": [P], "dig_launch_count": [P, P], "dig_kernel_time": [P, P, P],
        "dig_sort_scratch_bytes": [I64, I32, P], "dig_sort_by_cell": [P, I64, I32, P, P, P, I64, P],
        "dig_sort_by_cell_noalloc": [P, I64, I32, P, P, P],
        "dig_couple": [P, P], "dig_read_couple": [P, I32, P, I64], "dig_write_moments": [P, I32, P],
        "dig_write_wall_flux": [P, P, I64],
        "closure_init": [P, C.c_uint64], "closure_set": [P, P, I64], "closure_get": [P, P, I64],
        "closure_features": [P, I32, P], "closure_targets": [P, I32, P, I64, P], "closure_forward": [P, P, I64, P],
        "closure_loss": [P, P, P, I64, I32, P], "closure_grad": [P, P, P, I64, P, P],
        "closure_train": [P, P, P, P, I64, P],
        "dig_checkpoint_bytes": [P, P], "dig_save": [P, P, I64], "dig_load": [P, P, I64],
        "dig_surface": [P, P, I64, P], "dig_test_forward_timeout": [P],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.dig_last_error.argtypes = [P]
    L.dig_last_error.restype = C.c_char_p
    _lib = L
    return L


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def make_config(scen, **over) -> DigConfig:
    g = scen.gas
    cfg = DigConfig()
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
    cfg.wait_timeout_s = 600.0
    for k, v in over.items():
        setattr(cfg, k, v)
    return cfg


class Solver:
    """One DSMC context on one CUDA device (the C ABI, with torch-owned memory)."""

    def __init__(self, scen, device: str = "cuda:0", stream=None, **over):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("paper_2607_08195_gb300.Solver needs a CUDA device (no CPU fallback)")
        self.L = load_library()
        self.scen = scen
        self.device = torch.device(device)
        self.cfg = make_config(scen, **over)
        h = C.c_void_p()
        self._check(self.L.dig_create(C.byref(self.cfg), C.byref(h)), None)
        self.h = h
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._check(self.L.dig_set_stream(self.h, C.c_void_p(self.stream.cuda_stream)))
        m = scen.mesh
        self.n_tets = len(m.tets)
        bcs = (DigBC * max(1, len(m.bcs)))()
        for i, b in enumerate(m.bcs):
            bcs[i].kind, bcs[i].T, bcs[i].n = b["kind"], b["T"], b["n"]
            for q in range(3):
                bcs[i].U[q] = b["U"][q]
        nodes = np.ascontiguousarray(m.nodes, np.float64)
        tets = np.ascontiguousarray(m.tets, np.int32)
        tag = np.ascontiguousarray(m.face_tag, np.int32)
        self._check(self.L.mesh_load(self.h, _p(nodes), len(nodes), _p(tets), len(tets), _p(tag),
                                     C.cast(bcs, C.c_void_p), len(m.bcs)))
        nb = C.c_int64(0)
        self._check(self.L.dig_arena_bytes(self.h, C.byref(nb)))
        self.arena_bytes = nb.value
        self.arena = torch.empty(self.arena_bytes + 256, dtype=torch.uint8, device=self.device)
        ptr = self.arena.data_ptr()
        ptr = (ptr + 255) & ~255
        self._check(self.L.dig_bind_arena(self.h, C.c_void_p(ptr), self.arena_bytes))

    # ---------------------------------------------------------------- basics
    def _check(self, rc, h=-1):
        if rc != 0:
            hh = self.h if h == -1 else h
            msg = self.L.dig_last_error(hh).decode() if hh else ""
            raise DigError(rc, msg)

    def close(self):
        if getattr(self, "h", None):
            self.L.dig_synchronize(self.h)
            self.L.dig_destroy(self.h)
            self.h = None
            self.arena = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- particles
    def init(self, n=None):
        self._check(self.L.particles_init(self.h, self.scen.n_particles if n is None else n))

    def write(self, x, v, Ir, cell):
        x = np.ascontiguousarray(x, np.float64)
        v = np.ascontiguousarray(v, np.float32)
        Ir = None if Ir is None else np.ascontiguousarray(Ir, np.float32)
        cell = np.ascontiguousarray(cell, np.int32)
        self._check(self.L.write_particles(self.h, _p(x), _p(v), _p(Ir), _p(cell), len(cell)))

    def count(self):
        n = C.c_int64(0)
        self._check(self.L.dig_particle_count(self.h, C.byref(n)))
        return n.value

    def read(self):
        N = self.count()
        x = np.zeros((N, 3), np.float64)
        v = np.zeros((N, 3), np.float32)
        Ir = np.zeros(N, np.float32)
        cell = np.zeros(N, np.int32)
        n = C.c_int64(0)
        self._check(self.L.read_particles(self.h, _p(x), _p(v), _p(Ir), _p(cell), N, C.byref(n)))
        return x, v, Ir, cell

    def step(self, n=1, flags=EWMA):
        self._check(self.L.dsmc_step(self.h, n, flags))

    def sample(self, action):
        self._check(self.L.sample(self.h, action))

    def synchronize(self):
        self._check(self.L.dig_synchronize(self.h))

    def moments(self, which, out=None):
        k = NMAC if which & MACRO else NPHI
        if out is None:
            out = np.zeros((self.n_tets, k), np.float64)
        self._check(self.L.read_moments(self.h, which, _p(out), out.size))
        return out

    def pairs(self):
        n = C.c_int64(0)
        self._check(self.L.read_pairs(self.h, None, None, None, None, None, 0, C.byref(n)))
        N = n.value
        a = [np.zeros(N, np.int32) for _ in range(4)]
        acc = np.zeros(N, np.uint8)
        self._check(self.L.read_pairs(self.h, *[_p(x) for x in a], _p(acc), N, C.byref(n)))
        return np.stack(a + [acc.astype(np.int32)], axis=1)

    def counters(self):
        out = np.zeros(len(COUNTERS), np.int64)
        self._check(self.L.read_counters(self.h, _p(out), len(COUNTERS)))
        return dict(zip(COUNTERS, out.tolist()))

    def cell_state(self, cmax=None, rem=None):
        if cmax is None:
            cm = np.zeros(self.n_tets, np.float32)
            rm = np.zeros(self.n_tets, np.float64)
            self._check(self.L.dig_cell_state(self.h, _p(cm), _p(rm), 0))
            return cm, rm
        cm = np.ascontiguousarray(cmax, np.float32)
        rm = np.ascontiguousarray(rem, np.float64)
        self._check(self.L.dig_cell_state(self.h, _p(cm), _p(rm), 1))

    def wall_flux(self):
        n = C.c_int64(0)
        self.L.dig_wall_flux(self.h, None, 0, C.byref(n))
        out = np.zeros((n.value, 5), np.float64)
        self._check(self.L.dig_wall_flux(self.h, _p(out), out.size, C.byref(n)))
        return out

    def surface(self):
        """[n_bfaces][6]: number flux, pressure, shear (3), heat flux per boundary face (dig_surface)."""
        n = C.c_int64(0)
        self.L.dig_surface(self.h, None, 0, C.byref(n))
        out = np.zeros((n.value, 6), np.float64)
        self._check(self.L.dig_surface(self.h, _p(out), out.size, C.byref(n)))
        return out

    def couple(self):
        r = CoupleReport()
        self._check(self.L.dig_couple(self.h, C.byref(r)))
        return r.as_dict()

    def read_couple(self, which):
        k = {0: 6, 1: 12, 2: 6, 3: 1, 4: 6, 5: 1}[which]
        out = np.zeros((self.n_tets, k), np.float64)
        self._check(self.L.dig_read_couple(self.h, which, _p(out), out.size))
        return out

    def save(self):
        """The context's checkpoint (numpy uint8 array): see dig_save."""
        nb = C.c_int64(0)
        self._check(self.L.dig_checkpoint_bytes(self.h, C.byref(nb)))
        buf = np.empty(nb.value, np.uint8)
        self._check(self.L.dig_save(self.h, _p(buf), buf.size))
        return buf

    def load(self, buf):
        """Resume from a checkpoint made by save() on the same configuration and mesh."""
        buf = np.ascontiguousarray(buf, np.uint8)
        self._check(self.L.dig_load(self.h, _p(buf), buf.size))

    def write_moments(self, which, phi):
        phi = np.ascontiguousarray(phi, np.float64)
        assert phi.shape == (self.n_tets, NPHI)
        self._check(self.L.dig_write_moments(self.h, which, _p(phi)))

    def write_wall_flux(self, flux, steps):
        flux = np.ascontiguousarray(flux, np.float64)
        self._check(self.L.dig_write_wall_flux(self.h, _p(flux), steps))

    def kernel_time(self):
        ms, n = C.c_double(0), C.c_int64(0)
        self._check(self.L.dig_kernel_time(self.h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def launches(self):
        n = C.c_int64(0)
        self._check(self.L.dig_launch_count(self.h, C.byref(n)))
        return n.value

    # ---------------------------------------------------------------- learned closure
    def _dev(self, t, dtype, cols=None):
        import torch

        assert t.is_cuda and t.dtype == dtype and t.is_contiguous(), "expected a contiguous device tensor"
        if cols is not None:
            assert t.dim() == 2 and t.shape[1] == cols
        return C.c_void_p(t.data_ptr())

    def closure_init(self, seed):
        self._check(self.L.closure_init(self.h, seed))

    def closure_set(self, params):
        params = np.ascontiguousarray(params, np.float32)
        self._check(self.L.closure_set(self.h, _p(params), params.size))

    def closure_get(self):
        p = np.zeros(MLP_NPARAM, np.float32)
        self._check(self.L.closure_get(self.h, _p(p), p.size))
        return p

    def closure_features(self, which, X=None):
        """X[n_tets][13] (device tensor, filled) from the sums `which`."""
        import torch

        if X is None:
            X = torch.empty((self.n_tets, MLP_NIN), dtype=torch.float32, device=self.device)
        assert X.shape[0] == self.n_tets
        self._check(self.L.closure_features(self.h, which, self._dev(X, torch.float32, MLP_NIN)))
        return X

    def closure_targets(self, which, X, Y=None):
        import torch

        if Y is None:
            Y = torch.empty((X.shape[0], MLP_NOUT), dtype=torch.float32, device=self.device)
        self._check(self.L.closure_targets(self.h, which, self._dev(X, torch.float32, MLP_NIN), X.shape[0],
                                           self._dev(Y, torch.float32, MLP_NOUT)))
        return Y

    def test_forward_timeout(self):
        """The failure path of the tensor-core forward (its MMAs withheld, so
        its first wait gives up); returns the library's status code."""
        return self.L.dig_test_forward_timeout(self.h)

    def closure_forward(self, X, Y=None):
        import torch

        if Y is None:
            Y = torch.empty((X.shape[0], MLP_NOUT), dtype=torch.float32, device=self.device)
        self._check(self.L.closure_forward(self.h, self._dev(X, torch.float32, MLP_NIN), X.shape[0],
                                           self._dev(Y, torch.float32, MLP_NOUT)))
        return Y

    def closure_loss(self, X, Y, identity=False):
        import torch

        loss = C.c_double(0)
        self._check(self.L.closure_loss(self.h, self._dev(X, torch.float32, MLP_NIN),
                                        self._dev(Y, torch.float32, MLP_NOUT), X.shape[0], int(identity),
                                        C.byref(loss)))
        return loss.value

    def closure_grad(self, X, Y):
        import torch

        g = np.zeros(MLP_NPARAM, np.float32)
        loss = C.c_double(0)
        self._check(self.L.closure_grad(self.h, self._dev(X, torch.float32, MLP_NIN),
                                        self._dev(Y, torch.float32, MLP_NOUT), X.shape[0], _p(g),
                                        C.byref(loss)))
        return loss.value, g

    def closure_train(self, X, Y, epochs, batch, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, perm=None):
        """Adam over mini-batches; perm: device int32 [epochs][n] row orders
        (None: rows in order).  Returns the per-epoch training losses."""
        import torch

        n = X.shape[0]
        cfg = TrainConfig()
        cfg.epochs, cfg.batch, cfg.lr, cfg.beta1, cfg.beta2, cfg.eps = epochs, batch, lr, beta1, beta2, eps
        if perm is not None:
            assert perm.shape == (epochs, n)
            cfg.perm = self._dev(perm, torch.int32).value
        loss = np.zeros(epochs, np.float64)
        self._check(self.L.closure_train(self.h, C.byref(cfg), self._dev(X, torch.float32, MLP_NIN),
                                         self._dev(Y, torch.float32, MLP_NOUT), n, _p(loss)))
        return loss


def sort_by_cell(cell, n_cells: int, stream=None):
    """Stable counting sort of a device int32 tensor of cell ids (C ABI
    dig_sort_by_cell); returns (cell_start, order) device tensors.  Scratch is
    a torch allocation on the same device."""
    import torch

    L = load_library()
    assert cell.dtype == torch.int32 and cell.is_cuda and cell.is_contiguous()
    n = cell.numel()
    nb = C.c_int64(0)
    rc = L.dig_sort_scratch_bytes(n, n_cells, C.byref(nb))
    if rc:
        raise DigError(rc, L.dig_last_error(None).decode())
    scratch = torch.empty(nb.value + 256, dtype=torch.uint8, device=cell.device)
    sp = (scratch.data_ptr() + 255) & ~255
    cs = torch.empty(n_cells + 1, dtype=torch.int32, device=cell.device)
    order = torch.empty(max(n, 1), dtype=torch.int32, device=cell.device)
    s = stream if stream is not None else torch.cuda.current_stream(cell.device)
    rc = L.dig_sort_by_cell(C.c_void_p(cell.data_ptr()), n, n_cells, C.c_void_p(cs.data_ptr()),
                            C.c_void_p(order.data_ptr()), C.c_void_p(sp), nb.value, C.c_void_p(s.cuda_stream))
    if rc:
        raise DigError(rc, L.dig_last_error(None).decode())
    s.synchronize()
    return cs, order[: int(cs[-1].item())]
