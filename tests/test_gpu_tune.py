"""lat_tune: the step-kernel autotuner.

It times every kernel shape that can run a lattice on that lattice's own state,
keeps the fastest and remembers it per (N, precision, stencil, split storage,
expansion). These tests check that the sweep leaves the state and the scalar
block exactly as it found them (any odd or even step), that the chosen shape is
the one reported and reproduces a lattice set to it by hand bit for bit, that it
agrees with the oracle, and that handles created later with the same key start
with it while other keys do not.
"""
import numpy as np
import pytest

from gpu_helpers import compare_states
from oracle.oracle import Oracle
from paper_0911_5692_gb300 import Lattice
from paper_0911_5692_gb300.workloads import lphi4, m2phi2, random_state

pytestmark = pytest.mark.gpu


def _state(n, seed):
    return random_state(n, seed, precision=32, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-3), pi_mean=(0.5, 0.0),
                        pi_amp=(1e-3, 1e-3))


def _shape(info):
    return (info["variant"], info["ty"], info["depth"])


@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("odd", [False, True])
def test_tune_keeps_state_and_reports_its_shape(odd, split):
    n = 64
    p = lphi4(n, precision=32, split=split)
    g = Lattice(p)
    h = Lattice(p)        # created before the tune: the same starting shape as g
    g.set_state(*_state(n, 7), t=0.0, a=1.05, ad=0.5)
    g.evolve(3 if odd else 4)
    before = [x.copy() for x in g.get_state()]
    sc = g.scalars()
    bg = g.background() if split else None
    r = g.tune(steps=8)
    assert r["candidates"] >= 2
    assert 0 < r["best_ms"] <= r["slowest_ms"]
    info = g.kernel_info()
    assert (r["variant"], r["ty"], r["zr"], r["depth"], r["blocks"]) == (
        info["variant"], info["ty"], info["zr"], info["depth"], info["blocks"])
    assert g.scalars() == sc
    if split:
        assert g.background() == bg
    for a, b in zip(g.get_state(), before):
        assert np.array_equal(a, b)
    # the tuned lattice steps on exactly like one that ran the same kernels by
    # hand: h's starting shape first (h was created before the tune), then the
    # chosen one (each kernel's sums reduce in its own order, so the scalars
    # follow the kernel history)
    h.set_state(*_state(n, 7), t=0.0, a=1.05, ad=0.5)
    h.evolve(3 if odd else 4)
    h.set_kernel(r["variant"], r["ty"], 0, r["depth"])   # the automatic zr, as the tuner sets it
    g.evolve(40)
    h.evolve(40)
    for a, b in zip(g.get_state(), h.get_state()):
        assert np.array_equal(a, b)
    assert g.scalars() == h.scalars()


def test_tuned_lattice_matches_oracle():
    n = 48
    p = m2phi2(n, precision=32)
    st = random_state(n, 11, precision=32, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-4), pi_mean=(0.3, 0.0),
                      pi_amp=(1e-3, 1e-2))
    g = Lattice(p)
    g.set_state(*st, t=0.0, a=1.0, ad=0.3)
    g.tune(steps=4)
    g.evolve(5)
    o = Oracle(p)
    o.set_state(*st, t=0.0, a=1.0, ad=0.3)
    o.step(5)
    compare_states(g, o, 5 * 2e-6, f"tuned kernel {g.kernel_info()}")


def test_tuned_shape_is_taken_by_new_handles_of_the_same_key():
    n = 40
    p = lphi4(n, precision=32, seed=3)
    g = Lattice(p)
    g.init_fields()
    r = g.tune(steps=4)
    # same key (N, precision, stencil, split, expansion), other seed and L
    q = Lattice(dict(lphi4(n, precision=32, seed=9, L=12.0)))
    assert _shape(q.kernel_info()) == (r["variant"], r["ty"], r["depth"])
    # a handle of another key starts with the default shape
    other = lphi4(n, precision=64)
    fresh_default = _shape(Lattice(other).kernel_info())
    t = Lattice(other)
    t.set_kernel(0)
    assert _shape(t.kernel_info()) == fresh_default


def test_tune_27_point():
    n = 48
    p = dict(lphi4(n, precision=32), stencil=27)
    g = Lattice(p)
    st = _state(n, 5)
    g.set_state(*st, t=0.0, a=1.1, ad=0.45)
    r = g.tune(steps=4)
    assert r["variant"] == 2 and r["candidates"] >= 2
    g.evolve(2)
    o = Oracle(p)
    o.set_state(*st, t=0.0, a=1.1, ad=0.45)
    o.step(2)
    compare_states(g, o, 2 * 2e-6, "tuned 27-point kernel")
