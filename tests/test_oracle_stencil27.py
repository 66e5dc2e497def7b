"""Pins for the oracle's 27-point Laplacian (Sec. II.C: the Patra-Karttunen
stencil over the 3x3x3 cube, second-order accurate and fourth-order isotropic)
and for the evolution, gradient average and initial spectrum built on it.

The stencil is pinned by the properties the paper states, not by its weights:
a constant field gives zero; plane waves give -|k|^2 up to a relative error
falling as (k dx)^2; plane waves of equal |k| in different lattice directions
agree to O(k^6) (the 7-point stencil, checked alongside, differs at O(k^4)); a
dense 4^3 matrix assembled from the neighbour classes reproduces it; the
gradient average -<f L f> equals the bond sum over the 26 neighbour pairs; and
the leapfrog with this stencil follows its exact discrete dispersion.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle, grad2_mean27, laplacian, laplacian27
from paper_0911_5692_gb300.workloads import lphi4

# neighbour weights by class (face, edge, corner), in units of 1/dx^2: the
# Patra-Karttunen / DEFROST member of the family the conditions leave
FACE, EDGE, CORNER = 14 / 30, 3 / 30, 1 / 30


def _mode(n, kv):
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return np.cos(2 * np.pi * (kv[0] * x + kv[1] * y + kv[2] * z) / n)


def _eigen(lap, n, kv, dx):
    """Eigenvalue of a Laplacian on the mode cos(k.x) (the mode is an eigenvector
    of any symmetric periodic stencil)."""
    m = _mode(n, kv)
    lm = lap(m, dx)
    i = np.unravel_index(np.argmax(np.abs(m)), m.shape)
    assert np.max(np.abs(lm - lm[i] / m[i] * m)) <= 1e-10 * np.max(np.abs(lm))
    return lm[i] / m[i]


def test_constant_field_gives_zero():
    f = np.full((6, 6, 6), 3.25)
    assert np.max(np.abs(laplacian27(f, 0.7))) <= 1e-12


def test_second_order_accuracy():
    """(L + k^2)/k^2 -> 0 as (k dx)^2: halving dx at fixed k quarters it."""
    errs = []
    for n in (32, 64):
        dx = 1.0 / n
        kv = (1, 2, 0)
        k2 = sum((2 * np.pi * kk) ** 2 for kk in kv)
        lam = _eigen(laplacian27, n, kv, dx)
        errs.append(abs(lam + k2) / k2)
    assert 3.6 < errs[0] / errs[1] < 4.4


def test_fourth_order_isotropy():
    """Equal |k| along different lattice directions: (3,0,0), (2,2,1), (0,3,0)
    have |n|^2 = 9. The 27-point eigenvalues agree to O(k^6); the 7-point ones
    differ at O(k^4)."""
    n = 48
    dx = 1.0 / n
    k2 = (2 * np.pi * 3) ** 2
    kdx4 = (math.sqrt(k2) * dx) ** 4
    l27 = [_eigen(laplacian27, n, kv, dx) for kv in ((3, 0, 0), (2, 2, 1), (0, 3, 0))]
    l7 = [_eigen(laplacian, n, kv, dx) for kv in ((3, 0, 0), (2, 2, 1), (0, 3, 0))]
    spread27 = (max(l27) - min(l27)) / k2
    spread7 = (max(l7) - min(l7)) / k2
    assert spread7 > 0.01 * kdx4          # the 7-point stencil's k^4 term is anisotropic
    assert spread27 < 0.05 * spread7       # the 27-point stencil's is not
    assert abs(l27[0] - l27[2]) <= 1e-12 * k2   # symmetric under axis exchange


def test_brute_force_dense_matrix_4():
    """Assemble the 64 x 64 matrix of the stencil from its neighbour classes on a
    periodic 4^3 lattice and apply it to random fields; it is symmetric with zero
    row sums."""
    n, dx = 4, 0.37
    N = n ** 3
    A = np.zeros((N, N))
    w = {1: FACE, 2: EDGE, 3: CORNER}
    for z in range(n):
        for y in range(n):
            for x in range(n):
                i = (z * n + y) * n + x
                A[i, i] += -128 / 30
                for dz in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for ddx in (-1, 0, 1):
                            c = abs(dz) + abs(dy) + abs(ddx)
                            if c == 0:
                                continue
                            j = (((z + dz) % n) * n + (y + dy) % n) * n + (x + ddx) % n
                            A[i, j] += w[c]
    A /= dx * dx
    assert np.allclose(A, A.T, atol=0) and np.max(np.abs(A.sum(axis=1))) < 1e-12 / (dx * dx)
    rng = np.random.default_rng(3)
    f = rng.standard_normal((n, n, n))
    ref = (A @ f.ravel()).reshape(n, n, n)
    assert np.max(np.abs(laplacian27(f, dx) - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_gradient_average_is_bond_sum():
    """-<f L f> = (1/2) < sum over the 26 neighbours b of w_b (f(x+b) - f(x))^2 >
    (summation by parts for a symmetric stencil with zero row sums)."""
    rng = np.random.default_rng(5)
    n, dx = 8, 0.3
    f = 1.0 + 1e-3 * rng.standard_normal((n, n, n))
    acc = np.zeros_like(f)
    w = {1: FACE, 2: EDGE, 3: CORNER}
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for ddx in (-1, 0, 1):
                c = abs(dz) + abs(dy) + abs(ddx)
                if c:
                    acc += w[c] * (np.roll(f, (-dz, -dy, -ddx), axis=(0, 1, 2)) - f) ** 2
    ref = 0.5 * acc.mean() / (dx * dx)
    assert abs(grad2_mean27(f, dx) - ref) <= 1e-9 * ref


@pytest.mark.parametrize("nsteps", [1, 9, 150])
def test_leapfrog_dispersion_exact_27(nsteps):
    """Free massive field in static space with the 27-point stencil: a single mode
    evolves exactly as cos(k.x) cos(w_d (n+1/2) dt), cos(w_d dt) = 1 - w^2 dt^2/2,
    w^2 = m^2 - lambda_27(k) (lambda_27 the stencil's eigenvalue on the mode)."""
    n, dt = 8, 0.1
    p = dict(n=n, model=1, expansion=0, L=n * 0.5, dt=dt, lam=0.0, m=1e-6, g2=0.0, phi0=(1.0, 0.0),
             dphi0=(0.0, 0.0), eight_pi_G=1.0, fluct=0.0, seed=0, stencil=27)
    dx = p["L"] / n
    kf, kc = (1, 2, 0), (3, 1, 1)
    def wd(kv, m2):
        w2 = m2 - _eigen(laplacian27, n, kv, dx)
        return math.acos(1 - w2 * dt * dt / 2) / dt
    wf, wc = wd(kf, 1.0), wd(kc, 0.0)
    amp = 1e-3
    o = Oracle(p)
    z = np.zeros((n, n, n))
    o.set_state(amp * _mode(n, kf) * math.cos(wf * dt / 2), amp * _mode(n, kc) * math.cos(wc * dt / 2), z, z)
    o.step(nsteps)
    f0, f1, _, _ = o.get_state()
    np.testing.assert_allclose(f0, amp * _mode(n, kf) * math.cos(wf * (nsteps + 0.5) * dt), rtol=0, atol=1e-12 * amp)
    np.testing.assert_allclose(f1, amp * _mode(n, kc) * math.cos(wc * (nsteps + 0.5) * dt), rtol=0, atol=1e-12 * amp)


def test_sums_use_the_stencils_gradient_average():
    n = 8
    p = lphi4(n, precision=64)
    p["stencil"] = 27
    rng = np.random.default_rng(7)
    st = [1.0 + 1e-3 * rng.standard_normal((n, n, n)), 1e-3 * rng.standard_normal((n, n, n)),
          0.5 + 1e-3 * rng.standard_normal((n, n, n)), 1e-3 * rng.standard_normal((n, n, n))]
    o = Oracle(p)
    o.set_state(*st, t=0.0, a=1.0, ad=0.3)
    S = o.scalars()["S"]
    dx = p["L"] / n
    assert S[0] == pytest.approx(grad2_mean27(st[0], dx), rel=1e-14)
    assert S[1] == pytest.approx(grad2_mean27(st[1], dx), rel=1e-14)


def test_initial_spectrum_uses_the_stencils_dispersion():
    """With the 27-point stencil the vacuum spectrum follows 1/(2 w_k) with
    w_k^2 = -lambda_27(k) + m_eff^2, within the chi^2 sampling error."""
    n = 24
    p = lphi4(n, expansion=0, fluct=1.0)
    p["dt"] = 1e-12
    p["stencil"] = 27
    o = Oracle(p)
    o.init_fields()
    d = o.derived()
    dx = d["dx"]
    amp2 = (d["A"] * d["B"]) ** 2 * dx ** -3
    k = np.fft.fftfreq(n) * n
    KX, KY, KZ = np.meshgrid(k, k, k, indexing="ij")
    nmag = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    # the stencil's eigenvalues from its real-space action on a delta function
    delta = np.zeros((n, n, n))
    delta[0, 0, 0] = 1.0
    lam = np.real(np.fft.fftn(laplacian27(delta, dx)))
    fh = d["A"] * p["phi0"][0]
    meff2 = [3 * d["cdom0"] * fh ** 2, d["kappa0"] * fh ** 2]
    for field in (0, 1):
        f = o.array(field, 0)
        P = np.abs(np.fft.fftn(f - f.mean())) ** 2 / n ** 3
        expect = amp2 / (2 * np.sqrt(-lam + meff2[field]))
        for b in range(2, n // 4 + 1):
            inside = (np.rint(nmag) == b) & (nmag <= n / 4)
            if inside.sum() < 50:
                continue
            ratio = P[inside].mean() / expect[inside].mean()
            assert abs(ratio - 1) < 5 / math.sqrt(inside.sum() / 2), (field, b, ratio)
