"""Pins for the oracle's per-site energy density and pressure (Sec. II.B, eq.
rho-pres evaluated at every site; the paper's second kernel, Sec. II.C).

- a homogeneous state gives the physical rho = sum phidot^2/2 + V(phi, chi) and
  p = sum phidot^2/2 - V at every site (the program-unit conversions undone by
  hand from the rescaling of Sec. II.B);
- a single Fourier mode gives, per site, the 7-point gradient energy of its
  closed form (trigonometry of cos(theta +- kappa) - cos(theta));
- the volume means equal the averages of energies() (summation by parts: each
  neighbour pair's squared difference is split evenly between its two sites);
- translating or mirroring the state translates or mirrors the fields (a
  one-sided split of the gradient energy would break the mirror symmetry).
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_0911_5692_gb300.workloads import lphi4, m2phi2, random_state


def _state(n, seed):
    return random_state(n, seed, precision=64, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-3), pi_mean=(0.5, 0.0),
                        pi_amp=(1e-3, 1e-3))


@pytest.mark.parametrize("stencil", [7, 27])
@pytest.mark.parametrize("expansion", [0, 1])
def test_means_are_the_volume_averages(stencil, expansion):
    n = 8
    p = dict(lphi4(n, precision=64, expansion=expansion), stencil=stencil)
    o = Oracle(p)
    o.set_state(*_state(n, 3), t=0.0, a=1.15 if expansion else 1.0, ad=0.3 if expansion else 0.0)
    rho, pres = o.energy_field()
    e = o.energies()
    assert rho.mean() == pytest.approx(e["rho"], rel=1e-12)
    assert pres.mean() == pytest.approx(e["p"], rel=1e-12)


@pytest.mark.parametrize("stencil", [7, 27])
def test_homogeneous_state_closed_form(stencil):
    """Static space, lambda phi^4 + g^2/2 phi^2 chi^2, homogeneous phi, chi and
    velocities: f = A phi, f' = (A/B) phidot (a = 1, r h = 0), dt negligible."""
    n = 6
    lam, g2 = 9e-14, 1.8e-11
    phi, chi, phid, chid = 0.342, 0.05, 3e-8, -2e-8
    p = dict(lphi4(n, precision=64, expansion=0), stencil=stencil, lam=lam, g2=g2, phi0=(phi, 0.0), dt=1e-9)
    o = Oracle(p)
    d = o.derived()
    A, B = d["A"], d["B"]
    one = np.ones((n, n, n))
    o.set_state(A * phi * one, A * chi * one, A / B * phid * one, A / B * chid * one, t=0.0, a=1.0, ad=0.0)
    rho, pres = o.energy_field()
    V = lam / 4 * phi ** 4 + 0.5 * g2 * phi ** 2 * chi ** 2
    K = 0.5 * phid ** 2 + 0.5 * chid ** 2
    np.testing.assert_allclose(rho, K + V, rtol=1e-7)
    np.testing.assert_allclose(pres, K - V, rtol=1e-7)


def test_single_mode_gradient_energy_closed_form_7():
    """f_phi = 1 + eps cos(theta), theta = 2 pi k.x / n, f_chi = 0, f' = 0, static
    space, m^2 phi^2 model: per site, rho - V = (B^2/A^2) (1/2) g(x) with
    g = (eps/dx)^2 sum_d [(1 - cos kappa_d)^2 cos^2 theta + sin^2 kappa_d sin^2 theta],
    kappa_d = 2 pi k_d / n (half of the squared differences to both neighbours
    along each axis)."""
    n, eps = 12, 1e-3
    kv = (1, 2, 3)
    p = dict(m2phi2(n, precision=64, expansion=0), dt=1e-9, g2=0.0)
    o = Oracle(p)
    d = o.derived()
    A, B, dx = d["A"], d["B"], d["dx"]
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    theta = 2 * np.pi * (kv[0] * x + kv[1] * y + kv[2] * z) / n
    f0 = 1.0 + eps * np.cos(theta)
    zero = np.zeros_like(f0)
    o.set_state(f0, zero, zero, zero, t=0.0, a=1.0, ad=0.0)
    rho, pres = o.energy_field()
    m = p["m"]
    V = 0.5 * m ** 2 * (f0 / A) ** 2                        # physical 1/2 m^2 phi^2
    g = sum((1 - math.cos(2 * np.pi * k / n)) ** 2 * np.cos(theta) ** 2
            + math.sin(2 * np.pi * k / n) ** 2 * np.sin(theta) ** 2 for k in kv) * (eps / dx) ** 2
    expect_grad = B ** 2 / A ** 2 * 0.5 * g
    np.testing.assert_allclose(rho - V, expect_grad, rtol=1e-6, atol=1e-9 * expect_grad.max())
    np.testing.assert_allclose(-pres - V, expect_grad / 3, rtol=1e-6, atol=1e-9 * expect_grad.max())


@pytest.mark.parametrize("stencil", [7, 27])
def test_translation_covariance(stencil):
    n = 8
    p = dict(lphi4(n, precision=64), stencil=stencil)
    st = _state(n, 4)
    o = Oracle(p)
    o.set_state(*st, t=0.0, a=1.1, ad=0.3)
    rho, pres = o.energy_field()
    sh = (1, 2, 3)
    o2 = Oracle(p)
    o2.set_state(*[np.roll(a, sh, axis=(0, 1, 2)) for a in st], t=0.0, a=1.1, ad=0.3)
    rho2, pres2 = o2.energy_field()
    np.testing.assert_allclose(rho2, np.roll(rho, sh, axis=(0, 1, 2)), rtol=1e-14)
    np.testing.assert_allclose(pres2, np.roll(pres, sh, axis=(0, 1, 2)), rtol=1e-14)


@pytest.mark.parametrize("stencil", [7, 27])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_mirror_symmetry(stencil, axis):
    """x -> -x (mod n) along one axis maps the fields into themselves mirrored."""
    n = 8
    p = dict(lphi4(n, precision=64, expansion=0), stencil=stencil)
    st = _state(n, 6)

    def mirror(a):
        return np.roll(np.flip(a, axis=axis), 1, axis=axis)

    o = Oracle(p)
    o.set_state(*st, t=0.0, a=1.0, ad=0.0)
    rho, pres = o.energy_field()
    o2 = Oracle(p)
    o2.set_state(*[mirror(a) for a in st], t=0.0, a=1.0, ad=0.0)
    rho2, pres2 = o2.energy_field()
    # the gradient part is ~1e-6 of rho; compare it after removing the site-local terms
    np.testing.assert_allclose(rho2, mirror(rho), rtol=1e-13)
    np.testing.assert_allclose(pres2, mirror(pres), rtol=1e-13)
    grad = rho - pres
    assert np.max(np.abs((rho2 - pres2) - mirror(grad))) <= 1e-9 * np.max(np.abs(grad - grad.mean()))
