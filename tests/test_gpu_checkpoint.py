"""Checkpoint / resume through the C ABI (dig_save / dig_load): a run resumed
from a checkpoint continues bit for bit, across DSMC steps, moving and
cumulative averages and a DIG coupling; a checkpoint of another
configuration or a truncated one is refused."""
import dataclasses

import numpy as np
import pytest

from paper_2607_08195_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2607_08195_gb300 import dig  # noqa: E402

FL = dig.EWMA | dig.CUMUL


def tail(g):
    """Continue a run: 20 steps, one coupling, 10 steps; return its state."""
    g.step(20, FL)
    r = g.couple()
    g.step(10, FL)
    x, v, I, c = g.read()
    return r, x, v, I, c, g.moments(dig.PHI_EWMA), g.moments(dig.PHI_CUM)


def test_resume_is_bit_exact():
    s = W.config_small(seed=5)
    g = dig.Solver(s, "cuda:0", N_m=40)
    g.init()
    g.step(30, FL)
    g.couple()
    g.step(10, FL)
    ck = g.save()
    a = tail(g)
    h = dig.Solver(s, "cuda:0", N_m=40)
    h.load(ck)
    b = tail(h)
    assert a[0] == b[0]
    for u, w in zip(a[1:], b[1:]):
        assert np.array_equal(u, w)


def test_load_refuses_other_configuration_and_truncation():
    s = W.config_small(seed=5)
    g = dig.Solver(s, "cuda:0")
    g.init()
    g.step(3, FL)
    ck = g.save()
    other = dig.Solver(W.config_small(seed=6), "cuda:0")
    with pytest.raises(RuntimeError):
        other.load(ck)
    # settings that change results but not the arena: refused, the field named
    for over in (dict(alpha=1.4), dict(local_acc=1), dict(N_m=77), dict(cfl=1.0), dict(KnD_max=0.5)):
        if "alpha" in over:
            sc = W.config_small(seed=5)
            sc.gas = dataclasses.replace(sc.gas, alpha=1.4)
            h = dig.Solver(sc, "cuda:0")
        else:
            h = dig.Solver(s, "cuda:0", **over)
        with pytest.raises(RuntimeError, match="different dig_config." + list(over)[0]):
            h.load(ck)
    same = dig.Solver(s, "cuda:0")
    with pytest.raises(RuntimeError):
        same.load(ck[: len(ck) // 2])
    with pytest.raises(RuntimeError):
        same.load(np.zeros(64, np.uint8))
