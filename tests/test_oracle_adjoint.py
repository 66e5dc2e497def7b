"""Pins for the oracle's reverse-mode derivative of the leapfrog (Oracle.vjp).

The adjoint is checked against the oracle's own forward map by central finite
differences (the derivative's definition), in FP64 on 16^3 lattices:
* the gradient of the final <chi^2> with respect to g^2 and along random
  directions of the initial (f, pi), with expansion on and off and for both
  potentials (the contract asks rel <= 1e-5; FP64 central differences reach
  1e-8, which is what is asserted);
* the dot-product test <v, J u> = <J^T v, u> for a single step, with the scale
  factor a and a' included in both u and v;
* a linear case (m^2 phi^2, g^2 = 0, no expansion) in which the step map is
  linear, so central differences of the quadratic observable are exact and the
  adjoint must reproduce them to rounding.
A dropped term of the adjoint (for instance the feedback of the volume sums
through a'' into later steps, or a Hessian cross term) moves the directional
derivative by far more than these tolerances.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_0911_5692_gb300.workloads import lphi4, m2phi2, random_state

N = 16


def _case(name):
    if name == "lphi4_expanding":
        p = lphi4(N, precision=64)
        st = random_state(N, 3, 64, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-3), pi_mean=(0.5, 0.0), pi_amp=(1e-3, 1e-3))
        return p, st, dict(t=0.0, a=1.1, ad=0.45, step=0)
    if name == "lphi4_static":
        p = lphi4(N, precision=64, expansion=0)
        st = random_state(N, 3, 64, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-3), pi_mean=(0.5, 0.0), pi_amp=(1e-3, 1e-3))
        return p, st, dict(t=0.0, a=1.0, ad=0.0, step=0)
    if name == "m2phi2_expanding":
        p = m2phi2(N, precision=64)
        st = random_state(N, 4, 64, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-4), pi_mean=(0.3, 0.0), pi_amp=(1e-3, 1e-2))
        return p, st, dict(t=0.0, a=1.0, ad=0.3, step=0)
    raise KeyError(name)


def _final_chi2(p, st, scal, nsteps, g2=None):
    o = Oracle(p)
    o.set_state(*st, **scal)
    if g2 is not None:
        o.set_g2(g2)
    o.step(nsteps)
    return o.chi2_mean()


CASES = ["lphi4_expanding", "lphi4_static", "m2phi2_expanding"]


@pytest.mark.parametrize("name", CASES)
def test_g2_gradient_matches_central_difference(name):
    p, st, scal = _case(name)
    o = Oracle(p)
    o.set_state(*st, **scal)
    J, _, _, dg2 = o.chi2_gradient(40)
    assert J == pytest.approx(_final_chi2(p, st, scal, 40), rel=1e-15)
    e = 1e-6 * p["g2"]
    fd = (_final_chi2(p, st, scal, 40, p["g2"] + e) - _final_chi2(p, st, scal, 40, p["g2"] - e)) / (2 * e)
    assert abs(dg2 - fd) <= 1e-8 * abs(fd)


@pytest.mark.parametrize("name", CASES)
def test_state_gradient_matches_central_difference(name):
    """Directional derivative along a random direction of all four arrays."""
    p, st, scal = _case(name)
    o = Oracle(p)
    o.set_state(*st, **scal)
    _, fb, pb, _ = o.chi2_gradient(40)
    rng = np.random.default_rng(11)
    u = [1e-6 * rng.standard_normal((N, N, N)) for _ in range(4)]
    plus = [s + d for s, d in zip(st, u)]
    minus = [s - d for s, d in zip(st, u)]
    fd = (_final_chi2(p, plus, scal, 40) - _final_chi2(p, minus, scal, 40)) / 2
    ad = sum(float(np.sum(g * d)) for g, d in zip(list(fb) + list(pb), u))
    assert abs(ad - fd) <= 1e-6 * abs(fd)


def _step_map(p, st, scal, nsteps=1):
    o = Oracle(p)
    o.set_state(*st, **scal)
    o.step(nsteps)
    s = o.scalars()
    return list(o.get_state()), s["a"], s["ad"]


@pytest.mark.parametrize("name", CASES)
def test_single_step_dot_product(name):
    """<v, J u> (central difference of one step) = <J^T v, u> (adjoint), with a, a'
    part of both the input and the output of the step."""
    p, st, scal = _case(name)
    rng = np.random.default_rng(21)
    v = [rng.standard_normal((N, N, N)) for _ in range(4)]
    va, vad = rng.standard_normal(2)
    eps = 1e-6
    u = [eps * rng.standard_normal((N, N, N)) for _ in range(4)]
    ua, uad = eps * rng.standard_normal(2) * (1.0 if p["expansion"] else 0.0)

    def side(sign):
        s2 = [x + sign * d for x, d in zip(st, u)]
        sc = dict(scal, a=scal["a"] + sign * ua, ad=scal["ad"] + sign * uad)
        arrs, a, ad = _step_map(p, s2, sc)
        return sum(float(np.sum(x * w)) for x, w in zip(arrs, v)) + (va * a + vad * ad if p["expansion"] else 0.0)

    jvp = (side(+1) - side(-1)) / 2
    o = Oracle(p)
    o.set_state(*st, **scal)
    fb, pb, ba, bad, _, _ = o.vjp(1, v[0:2], v[2:4], va if p["expansion"] else 0.0, vad if p["expansion"] else 0.0)
    vjp = sum(float(np.sum(g * d)) for g, d in zip(list(fb) + list(pb), u)) + ba * ua + bad * uad
    assert abs(vjp - jvp) <= 1e-7 * max(abs(jvp), 1e-300)


def test_linear_case_is_exact():
    """m^2 phi^2 with g^2 = 0 and no expansion: the step map is linear, J = <chi^2> is
    quadratic, so a central difference with a large step is exact up to rounding."""
    p = m2phi2(N, precision=64, expansion=0, g2=0.0)
    st = random_state(N, 9, 64, f_mean=(1.0, 0.0), f_amp=(1e-2, 1e-2), pi_mean=(0.3, 0.0), pi_amp=(1e-2, 1e-2))
    scal = dict(t=0.0, a=1.0, ad=0.0, step=0)
    o = Oracle(p)
    o.set_state(*st, **scal)
    _, fb, pb, _ = o.chi2_gradient(30)
    rng = np.random.default_rng(2)
    u = [0.1 * rng.standard_normal((N, N, N)) for _ in range(4)]
    plus = [s + d for s, d in zip(st, u)]
    minus = [s - d for s, d in zip(st, u)]
    fd = (_final_chi2(p, plus, scal, 30) - _final_chi2(p, minus, scal, 30)) / 2
    ad = sum(float(np.sum(g * d)) for g, d in zip(list(fb) + list(pb), u))
    assert abs(ad - fd) <= 1e-11 * abs(fd)
    # chi evolves on its own here: the gradient with respect to phi vanishes
    assert np.max(np.abs(fb[0])) == 0.0 and np.max(np.abs(pb[0])) == 0.0


def test_vjp_leaves_lattice_advanced():
    p, st, scal = _case("lphi4_expanding")
    o = Oracle(p)
    o.set_state(*st, **scal)
    z = np.zeros((N, N, N))
    o.vjp(7, [z, z], [z, z])
    ref = Oracle(p)
    ref.set_state(*st, **scal)
    ref.step(7)
    for x, y in zip(o.get_state(), ref.get_state()):
        assert np.array_equal(x, y)
    assert o.scalars() == ref.scalars()
