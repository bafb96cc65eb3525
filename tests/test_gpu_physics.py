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
