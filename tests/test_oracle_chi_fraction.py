"""Pins for the oracle's second observable of the derivative: the fraction of
the energy density in chi (orc_chi_fraction), and its gradient.

The observable takes eq. rho-pres's kinetic, gradient and potential terms at
the momentum time of the stored state (fields and a taken back half a step)
and divides chi's own kinetic and gradient energy by the total. Pinned by:
- its limits: 0 when chi and its momentum vanish, 1 when phi and its
  momentum vanish (the potential then vanishes too);
- the energies' chi share (energies(), taken at the field time with the
  momenta there): the two agree as dt -> 0, the gap falling linearly in dt,
  which fixes every factor of 1/2, the a^(-2s-2) of the gradient energy and
  the r h f of the kinetic one (a slip in any gives an O(1) gap);
- its gradient with respect to the stored f, pi, a and a', and its direct
  derivative with respect to g^2 (the interaction energy in the total), against
  central differences of the value itself;
- the gradient after 40 steps with respect to g^2 and the starting state
  against central differences of the forward map (FP64, 16^3), as for <chi^2>.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_0911_5692_gb300.workloads import lphi4, m2phi2, random_state


def _state(n, seed, chi_amp=1e-2):
    return random_state(n, seed, precision=64, f_mean=(1.0, 0.0), f_amp=(1e-2, chi_amp), pi_mean=(0.3, 0.0),
                        pi_amp=(1e-2, chi_amp))


def test_limits():
    n = 6
    p = lphi4(n, precision=64)
    f0, f1, p0, p1 = _state(n, 1)
    z = np.zeros_like(f0)
    o = Oracle(p)
    o.set_state(f0, z, p0, z, t=0.0, a=1.1, ad=0.4)
    assert o.chi_fraction() == 0.0
    o.set_state(z, f1, z, p1, t=0.0, a=1.1, ad=0.4)
    assert o.chi_fraction() == pytest.approx(1.0, rel=1e-15)


def _smooth(arrs, keep=1):
    """Keep the Fourier modes with every |n_d| <= keep (a long-wavelength state,
    whose half-step kick is small)."""
    out = []
    for a in arrs:
        F = np.fft.fftn(a)
        k = np.fft.fftfreq(a.shape[0]) * a.shape[0]
        mask = (np.abs(k)[:, None, None] <= keep) & (np.abs(k)[None, :, None] <= keep) & (np.abs(k)[None, None, :] <= keep)
        out.append(np.ascontiguousarray(np.real(np.fft.ifftn(F * mask))))
    return out


@pytest.mark.parametrize("mk,coupling", [(lphi4, dict(G=1.0)), (m2phi2, dict(g2=1e-12))])
def test_approaches_the_energies_chi_share(mk, coupling):
    """The same stored arrays and scalars read with a smaller dt: both the
    observable (momentum time) and energies()' (kin1 + grad1) / rho (field time)
    tend to the same instant's value, their gap falling linearly in dt. Smooth
    fields and a weak coupling keep the half-step kick, hence the gap, small."""
    n = 8
    st = _smooth(_state(n, 2, chi_amp=0.1))
    gaps = []
    for dt in (0.02, 0.01, 0.005):
        p = dict(mk(n, precision=64, **coupling), dt=dt)
        o = Oracle(p)
        o.set_state(*st, t=0.0, a=1.2, ad=0.5)
        e = o.energies()
        share = (e["kin1"] + e["grad1"]) / e["rho"]
        J = o.chi_fraction()
        assert 1e-4 < J < 0.9
        gaps.append(abs(J - share))
    assert gaps[0] < 1e-2
    assert 1.6 < gaps[0] / gaps[1] < 2.4 and 1.6 < gaps[1] / gaps[2] < 2.4


@pytest.mark.parametrize("expansion", [0, 1])
def test_seed_matches_central_differences_of_the_value(expansion):
    n = 4
    p = lphi4(n, precision=64, expansion=expansion)
    st = _state(n, 3, chi_amp=0.1)
    sc = dict(t=0.0, a=1.2 if expansion else 1.0, ad=0.5 if expansion else 0.0, step=0)
    o = Oracle(p)
    o.set_state(*st, **sc)
    J, fb, pb, ab, adb, dg2 = o.chi_fraction(with_gradient=True)
    grads = list(fb) + list(pb)
    rng = np.random.default_rng(5)
    for _ in range(6):
        q, idx = int(rng.integers(4)), tuple(int(i) for i in rng.integers(n, size=3))
        e = 1e-6
        vals = []
        for sgn in (1, -1):
            arr = [a.copy() for a in st]
            arr[q][idx] += sgn * e
            o.set_state(*arr, **sc)
            vals.append(o.chi_fraction())
        fd = (vals[0] - vals[1]) / (2 * e)
        assert grads[q][idx] == pytest.approx(fd, rel=1e-6, abs=1e-12 * abs(J))
    if expansion:
        for k, g in (("a", ab), ("ad", adb)):
            e = 1e-6
            vals = []
            for sgn in (1, -1):
                s2 = dict(sc)
                s2[k] += sgn * e
                o.set_state(*st, **s2)
                vals.append(o.chi_fraction())
            fd = (vals[0] - vals[1]) / (2 * e)
            assert g == pytest.approx(fd, rel=1e-6)
    else:
        assert ab == 0.0 and adb == 0.0
    # the direct dependence on g^2 (through the interaction energy in the total)
    vals = []
    for sgn in (1, -1):
        o.set_g2(p["g2"] * (1 + sgn * 1e-6))
        o.set_state(*st, **sc)
        vals.append(o.chi_fraction())
    o.set_g2(p["g2"])
    assert dg2 == pytest.approx((vals[0] - vals[1]) / (2e-6 * p["g2"]), rel=1e-6)


def _final_fraction(p, st, scal, nsteps, g2=None):
    o = Oracle(p)
    o.set_state(*st, **scal)
    if g2 is not None:
        o.set_g2(g2)
    o.step(nsteps)
    return o.chi_fraction()


@pytest.mark.parametrize("expansion", [0, 1])
def test_gradient_after_steps_matches_central_differences(expansion):
    N = 16
    p = lphi4(N, precision=64, expansion=expansion)
    st = random_state(N, 3, 64, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-3), pi_mean=(0.5, 0.0), pi_amp=(1e-3, 1e-3))
    scal = dict(t=0.0, a=1.1 if expansion else 1.0, ad=0.45 if expansion else 0.0, step=0)
    o = Oracle(p)
    o.set_state(*st, **scal)
    J, fb, pb, dg2 = o.chi_fraction_gradient(40)
    assert J == pytest.approx(_final_fraction(p, st, scal, 40), rel=1e-14)
    e = 1e-6 * p["g2"]
    fd = (_final_fraction(p, st, scal, 40, p["g2"] + e) - _final_fraction(p, st, scal, 40, p["g2"] - e)) / (2 * e)
    assert abs(dg2 - fd) <= 1e-7 * abs(fd)
    rng = np.random.default_rng(11)
    u = [1e-6 * rng.standard_normal((N, N, N)) for _ in range(4)]
    plus = [s + d for s, d in zip(st, u)]
    minus = [s - d for s, d in zip(st, u)]
    fd = (_final_fraction(p, plus, scal, 40) - _final_fraction(p, minus, scal, 40)) / 2
    ad = sum(float(np.sum(g * d)) for g, d in zip(list(fb) + list(pb), u))
    assert abs(ad - fd) <= 1e-6 * abs(fd)
