"""The C-ABI library builds, loads without a GPU and exports every symbol that
include/dig.h declares; the binding's structs match the header's layout.
No compute calls (no GPU here)."""
import ctypes
import os
import re
import shutil

import pytest

from paper_2607_08195_gb300 import dig

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dig.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", txt, flags=re.M)
    return sorted(set(n for n in names if n not in ("defined",)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2607_08195_gb300 import build

    build.build()
    return dig.load_library()


def test_header_lists_match_binding():
    assert declared_functions() == sorted(dig.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def _c_layout(struct, fields):
    """sizeof and offsetof of every field of a struct of include/dig.h, from the C compiler."""
    import shutil
    import subprocess
    import tempfile

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(ROOT, "include")
    body = "".join(f'  printf("%zu\\n", offsetof({struct}, {f}));\n' for f in fields)
    src = ("#include <stddef.h>\n#include <stdio.h>\n#include \"dig.h\"\nint main(void) {\n"
           f'  printf("%zu\\n", sizeof({struct}));\n' + body + "  return 0;\n}\n")
    with tempfile.TemporaryDirectory() as d:
        c, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        open(c, "w").write(src)
        subprocess.check_call([cc, "-I", inc, c, "-o", exe])
        out = [int(x) for x in subprocess.check_output([exe]).split()]
    return out[0], out[1:]


@pytest.mark.parametrize("struct, cls", [("dig_config", "DigConfig"), ("dig_bc", "DigBC"),
                                         ("dig_couple_report", "CoupleReport")])
def test_struct_layout_matches_header(struct, cls):
    """The binding's ctypes mirrors have the size and field offsets that the C
    compiler gives the structs of include/dig.h."""
    py = getattr(dig, cls)
    names = [f for f, _ in py._fields_]
    size, offs = _c_layout(struct, names)
    assert ctypes.sizeof(py) == size
    assert [getattr(py, f).offset for f in names] == offs


def test_create_rejects_bad_config(lib):
    cfg = dig.DigConfig()
    h = ctypes.c_void_p()
    assert lib.dig_create(ctypes.byref(cfg), ctypes.byref(h)) == -1  # zero mass / dt
    from paper_2607_08195_gb300 import workload as W

    for alpha in (0.0, -1.0, float("nan")):  # the VSS exponent 1/alpha needs alpha > 0
        cfg = dig.make_config(W.config_small())
        cfg.alpha = alpha
        assert lib.dig_create(ctypes.byref(cfg), ctypes.byref(h)) == -1, alpha
    for field, value in (("recon", 2), ("local_acc", -1), ("tile_cells", 4096), ("rot_dof", 1), ("aa_m", -1),
                         ("aa_m", 33)):
        cfg = dig.make_config(W.config_small())
        setattr(cfg, field, value)
        assert lib.dig_create(ctypes.byref(cfg), ctypes.byref(h)) == -1, field


def test_mesh_load_host_validation(lib):
    """mesh_load runs on the host: bad meshes are rejected without a GPU."""
    import numpy as np

    from paper_2607_08195_gb300 import workload as W

    s = W.config_small()
    cfg = dig.make_config(s)
    h = ctypes.c_void_p()
    assert lib.dig_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
    m = s.mesh
    bcs = (dig.DigBC * 2)()
    tag = np.full_like(m.face_tag, -1)
    nodes = np.ascontiguousarray(m.nodes)
    tets = np.ascontiguousarray(m.tets)
    rc = lib.mesh_load(h, nodes.ctypes.data, len(nodes), tets.ctypes.data, len(tets), tag.ctypes.data,
                       ctypes.cast(bcs, ctypes.c_void_p), 2)
    assert rc == -2
    assert b"boundary face" in lib.dig_last_error(h)
    tag = np.ascontiguousarray(m.face_tag)
    rc = lib.mesh_load(h, nodes.ctypes.data, len(nodes), tets.ctypes.data, len(tets), tag.ctypes.data,
                       ctypes.cast(bcs, ctypes.c_void_p), 2)
    assert rc == 0
    nb = ctypes.c_int64(0)
    assert lib.dig_arena_bytes(h, ctypes.byref(nb)) == 0
    assert nb.value > 40 * cfg.capacity * 2
    lib.dig_destroy(h)


def test_closure_structs_layout():
    assert ctypes.sizeof(dig.TrainConfig) == 4 * 2 + 8 * 4 + 8
    assert ctypes.sizeof(dig.CoupleReport) == 4 * 2 + 8 + 8 * 4


def test_closure_host_validation(lib):
    """The closure entry points validate their arguments on the host: a wrong
    parameter count or training constants are rejected before any GPU work,
    and calls before an arena is bound report DIG_ERR_STATE."""
    import numpy as np

    from paper_2607_08195_gb300 import workload as W

    s = W.config_small()
    cfg = dig.make_config(s)
    h = ctypes.c_void_p()
    assert lib.dig_create(ctypes.byref(cfg), ctypes.byref(h)) == 0
    p = np.zeros(dig.MLP_NPARAM, np.float32)
    assert lib.closure_set(h, p.ctypes.data, dig.MLP_NPARAM - 1) == -1
    assert lib.closure_set(h, p.ctypes.data, dig.MLP_NPARAM) == -7
    assert lib.closure_init(h, 3) == -7
    tc = dig.TrainConfig()
    tc.epochs, tc.batch, tc.lr, tc.beta1, tc.beta2, tc.eps = 0, 16, 1e-3, 0.9, 0.999, 1e-8
    loss = np.zeros(1)
    fake = ctypes.c_void_p(256)  # never dereferenced: the call fails validation first
    assert lib.closure_train(h, ctypes.byref(tc), fake, fake, 10, loss.ctypes.data) == -1
    tc.epochs, tc.beta1 = 1, 1.0
    assert lib.closure_train(h, ctypes.byref(tc), fake, fake, 10, loss.ctypes.data) == -1
    assert lib.closure_features(h, 7, fake) == -1
    out = np.zeros(8)
    assert lib.dig_read_couple(h, 6, out.ctypes.data, 8) == -1  # selectors are 0..5
    assert lib.dig_read_couple(h, 5, out.ctypes.data, 8) == -7  # no arena bound yet
    assert lib.dig_destroy(h) == 0
