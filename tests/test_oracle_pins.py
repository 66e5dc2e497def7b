"""Pins for the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed-form lattice solutions, exact identities and
invariants of the scheme, an independent ODE integration in physical time, a
library FFT, and the statistics of the generated fluctuations. A plausible
mistake in the oracle (a dropped term, a wrong sign or index, a transposed
operand) fails at least one of them; the comment on each test says which.
"""
import math
import os

import numpy as np
import pytest

from oracle.oracle import Oracle, fft1, fft3, grad2_mean, laplacian, normal, philox4x32_10
from paper_0911_5692_gb300.workloads import lphi4, m2phi2, random_state

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ random numbers

def test_philox_known_answers():
    """Philox-4x32-10 against the published known-answer vectors (Salmon et al., SC'11)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert philox4x32_10(v[0:4], v[4:6]) == v[6:10]


def test_normals_are_standard():
    """Box-Muller output: mean 0, variance 1, kurtosis 3 within sampling error."""
    z = np.array([normal(7, 1, 0, i) for i in range(40000)])
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / z.size)
    k = ((z - z.mean()) ** 4).mean() / z.var() ** 2
    assert abs(k - 3) < 5 * math.sqrt(24 / z.size)
    # distinct streams for distinct (field, quantity) are uncorrelated
    w = np.array([normal(7, 1, 1, i) for i in range(40000)])
    assert abs(np.corrcoef(z, w)[0, 1]) < 5 / math.sqrt(z.size)


# ------------------------------------------------------------------ FFT

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 12, 48, 96, 128])
def test_fft1_matches_library(n):
    """The oracle's mixed-radix DFT against numpy.fft (forward and inverse sign)."""
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    np.testing.assert_allclose(fft1(x, -1), np.fft.fft(x), rtol=0, atol=1e-12 * n)
    np.testing.assert_allclose(fft1(x, +1), np.fft.ifft(x) * n, rtol=0, atol=1e-12 * n)


@pytest.mark.parametrize("n", [4, 6, 12])
def test_fft3_matches_library(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    np.testing.assert_allclose(fft3(x, -1), np.fft.fftn(x), rtol=0, atol=1e-11 * n ** 3)


# ------------------------------------------------------------------ Laplacian and gradient

@pytest.mark.parametrize("n", [4, 6, 16])
def test_laplacian_plane_wave_symbol(n):
    """A lattice plane wave is an eigenvector of the 7-point Laplacian with eigenvalue
    -sum_d (2/dx sin(k_d dx/2))^2 (closed form). Catches wrong sign, dx scaling,
    missing neighbour or a wrong periodic wrap."""
    dx = 0.37
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    for kv in [(1, 0, 0), (0, 2 % n, 1), (1, 1, n // 2), (n // 2, n // 2, n // 2)]:
        ph = 2 * np.pi * (kv[0] * x + kv[1] * y + kv[2] * z) / n
        f = np.cos(ph + 0.3)
        lam = sum((2 / dx * math.sin(math.pi * k / n)) ** 2 for k in kv)
        np.testing.assert_allclose(laplacian(f, dx), -lam * f, rtol=0, atol=1e-12 * max(lam, 1))


def test_summation_by_parts_identity():
    """Sec. II.B, divergence-theorem identity: on a periodic lattice the average of
    |grad f|^2 equals -<f Lap f>, exactly for the 7-point stencil with forward
    differences. Pins the gradient average against the Laplacian."""
    rng = np.random.default_rng(3)
    for n in (4, 6, 10):
        f = rng.standard_normal((n, n, n))
        dx = 0.2
        lhs = grad2_mean(f, dx)
        rhs = -(f * laplacian(f, dx)).mean()
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_brute_force_laplacian_matrix_4():
    """Brute force on 4^3: the Laplacian as a dense 64x64 matrix built from the
    periodic neighbour graph (each site linked to its 6 neighbours)."""
    n, dx = 4, 0.5
    N = n ** 3
    M = np.zeros((N, N))
    for z in range(n):
        for y in range(n):
            for x in range(n):
                i = (z * n + y) * n + x
                M[i, i] -= 6
                for dz, dy, dxx in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]:
                    j = (((z + dz) % n) * n + (y + dy) % n) * n + (x + dxx) % n
                    M[i, j] += 1
    M /= dx * dx
    f = np.random.default_rng(1).standard_normal((n, n, n))
    np.testing.assert_allclose(laplacian(f, dx).ravel(), M @ f.ravel(), rtol=0, atol=1e-13)
    # eigenvalues of the dense matrix are the closed-form symbol
    ev = np.sort(np.linalg.eigvalsh(M))
    sym = np.sort([-sum((2 / dx * math.sin(math.pi * k / n)) ** 2 for k in (a, b, c))
                   for a in range(n) for b in range(n) for c in range(n)])
    np.testing.assert_allclose(ev, sym, atol=1e-10)


# ------------------------------------------------------------------ rescaling

def _golden(name):
    d = {}
    for l in open(os.path.join(GOLDEN, name)):
        if l.strip() and l[0] != "#":
            k, v = l.split()
            d[k] = float(v)
    return d


def test_rescaling_matches_paper():
    """Sec. III prints r = 3/2, s = 0, A = 1/phi0 for the m^2 phi^2 model; Sec. II.B's
    rule gives r = 1, s = -1 for lambda phi^4. Both satisfy s - 2r + 3 = 0, and the
    choice makes the dominant potential term exactly f^beta/beta (coefficient 1)."""
    g = _golden("rescaling_sec3.txt")
    p = m2phi2(8)
    d = Oracle(p).derived()
    assert d["r"] == g["r"] and d["s"] == g["s"]
    assert abs(d["A"] * p["phi0"][0] - g["A_times_phi0"]) < 1e-15
    assert abs(d["B"] / p["m"] - g["B_over_m"]) < 1e-12
    assert abs(d["cdom0"] - 1) < 1e-12 and d["pdom"] == 0
    # interaction g^2 phi^2 chi^2/2 -> (g^2 phi0^2 / m^2) a^-3 f^2 chi^2 / 2
    assert abs(d["kappa0"] / (p["g2"] * p["phi0"][0] ** 2 / p["m"] ** 2) - 1) < 1e-12 and d["pint"] == -3
    q = lphi4(8)
    e = Oracle(q).derived()
    assert e["r"] == g["lambda_r"] and e["s"] == g["lambda_s"]
    assert abs(e["cdom0"] - 1) < 1e-12 and e["pdom"] == 0
    assert abs(e["kappa0"] / 200 - 1) < 1e-12 and e["pint"] == 0


# ------------------------------------------------------------------ leapfrog dispersion (P1)

def _free_params(n, dt, model=1, g2=0.0):
    # m^2 phi^2 model in static space: f'' = Lap f - f (program units, B = m), chi massless
    return dict(n=n, model=model, expansion=0, L=n * 0.5, dt=dt, lam=0.0, m=1e-6, g2=g2,
                phi0=(1.0, 0.0), dphi0=(0.0, 0.0), eight_pi_G=1.0, fluct=0.0, seed=0)


@pytest.mark.parametrize("nsteps", [1, 7, 200])
def test_leapfrog_dispersion_exact(nsteps):
    """Free massive field, static space: a single lattice mode evolves as
    f_{n+1/2} = cos(k.x) cos(w_d (n+1/2) dt) with cos(w_d dt) = 1 - w^2 dt^2/2 and
    w^2 = m^2 + sum_d (2/dx sin(k_d dx/2))^2, for any number of steps. Pins the
    kick/drift order, the Laplacian symbol and the sign of the mass term."""
    n, dt = 8, 0.1
    p = _free_params(n, dt)
    o = Oracle(p)
    dx = p["L"] / n
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    kf = (1, 2, 0)   # phi mode, massive (program mass 1)
    kc = (3, 0, 1)   # chi mode, massless
    def mode(kv):
        return np.cos(2 * np.pi * (kv[0] * x + kv[1] * y + kv[2] * z) / n)
    def wd(kv, m2):
        w2 = m2 + sum((2 / dx * math.sin(math.pi * k / n)) ** 2 for k in kv)
        return math.acos(1 - w2 * dt * dt / 2) / dt
    wf, wc = wd(kf, 1.0), wd(kc, 0.0)
    amp = 1e-3
    o.set_state(1.0 + 0 * x, amp * mode(kc) * math.cos(wc * dt / 2), np.zeros((n, n, n)), np.zeros((n, n, n)))
    # phi: homogeneous value 0 plus the mode (V = f^2/2 is linear in its derivative)
    o.array(0, 0)[...] = amp * mode(kf) * math.cos(wf * dt / 2)
    o.set_state(*o.get_state())
    o.step(nsteps)
    f0, f1, p0, p1 = o.get_state()
    np.testing.assert_allclose(f0, amp * mode(kf) * math.cos(wf * (nsteps + 0.5) * dt), rtol=0, atol=1e-12 * amp)
    np.testing.assert_allclose(f1, amp * mode(kc) * math.cos(wc * (nsteps + 0.5) * dt), rtol=0, atol=1e-12 * amp)
    # momenta at integer times: (f_{n+1/2} - f_{n-1/2}) / dt
    pf = -amp * mode(kf) * 2 * math.sin(wf * nsteps * dt) * math.sin(wf * dt / 2) / dt
    np.testing.assert_allclose(p0, pf, rtol=0, atol=1e-11 * amp)


# ------------------------------------------------------------------ reversibility (P2)

def _reverse_run(p, state, nsteps, expansion):
    o = Oracle(p)
    o.set_state(*state, t=0.0, a=1.0 if not expansion else 1.1, ad=0.0 if not expansion else 0.3)
    start = o.get_state()
    s0 = o.scalars()
    o.step(nsteps)
    f0, f1, p0, p1 = o.get_state()
    sc = o.scalars()
    dt = p["dt"]
    # negate momenta (and a'), drift by dt
    p0, p1 = -p0, -p1
    ad = -sc["ad"]
    f0 = f0 + dt * p0; f1 = f1 + dt * p1
    a = sc["a"] + dt * ad
    o.set_state(f0, f1, p0, p1, t=0.0, a=a, ad=ad)
    o.step(nsteps - 1)
    # final kick alone: one full step, then undo its drift
    o.step(1)
    f0, f1, p0, p1 = o.get_state()
    sc = o.scalars()
    f0 = f0 - dt * p0; f1 = f1 - dt * p1
    a = sc["a"] - dt * sc["ad"]
    return start, s0, (f0, f1, -p0, -p1), a, -sc["ad"]


@pytest.mark.parametrize("expansion", [0, 1])
def test_time_reversibility(expansion):
    """Staggered leapfrog is time-reversible: n steps forward, momenta (and a')
    negated, n steps back returns the initial state. Holds for the nonlinear,
    coupled system and, with the time-centred a' of eq. scale, with expansion on.
    Catches any asymmetric term (e.g. a kick using a lagged a'' or a field order
    dependence)."""
    n = 6
    p = lphi4(n, expansion=expansion)
    p["dt"] = 0.05
    st = random_state(n, 11, precision=64, f_mean=(1.0, 0.0), f_amp=(0.05, 0.05), pi_mean=(0.1, 0.0),
                      pi_amp=(0.05, 0.05))
    start, s0, back, a_back, ad_back = _reverse_run(p, st, 40, expansion)
    for x, y in zip(start, back):
        np.testing.assert_allclose(y, x, rtol=0, atol=1e-12)
    if expansion:
        assert abs(a_back - s0["a"]) < 1e-12
        assert abs(ad_back - s0["ad"]) < 1e-12


# ------------------------------------------------------------------ energy (P3) and homogeneous limit (P6)

def _energy_drift(dt_over_dx):
    n = 8
    p = lphi4(n, expansion=0, dt_over_dx=dt_over_dx, fluct=0.0, G=2.0)
    o = Oracle(p)
    st = random_state(n, 5, precision=64, f_mean=(1.0, 0.0), f_amp=(0.05, 0.05), pi_mean=(0.0, 0.0),
                      pi_amp=(0.0, 0.0))
    # smooth initial fields: keep only long wavelengths so the dt^2 regime is clean
    sm = []
    for a in st[:2]:
        F = np.fft.fftn(a)
        k = np.fft.fftfreq(n) * n
        kk = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
        F[kk > 1.5] = 0
        F[0, 0, 0] = a.sum()
        sm.append(np.real(np.fft.ifftn(F)))
    o.set_state(sm[0], sm[1], np.zeros((n, n, n)), np.zeros((n, n, n)))
    T = 6.0
    nsteps = int(round(T / p["dt"]))
    E0 = o.energies()["rho"]
    drift = 0.0
    chunk = max(1, nsteps // 60)
    for _ in range(nsteps // chunk):
        o.step(chunk)
        drift = max(drift, abs(o.energies()["rho"] / E0 - 1))
    return drift


def test_energy_conservation_second_order():
    """Static space: the total energy of the leapfrog is conserved to O(dt^2);
    halving dt reduces the maximum relative drift by 4 (within 20%)."""
    d1 = _energy_drift(0.1)
    d2 = _energy_drift(0.05)
    assert d1 < 1e-2
    assert 4 * 0.8 < d1 / d2 < 4 * 1.2, (d1, d2)


def _ode_reference(p, tau_end):
    """Homogeneous FRW + scalar fields in PHYSICAL variables (Sec. II.B eq. fe with
    Delta = 0 and the constraint H^2 = 8 pi G rho / 3), integrated with the program
    time tau as independent variable (dt_pr = B a^s dt)."""
    from scipy.integrate import solve_ivp
    o = Oracle(p)
    d = o.derived()
    A, B, r, s, beta = d["A"], d["B"], d["r"], d["s"], d["beta"]
    cpl = p["lam"] if p["model"] == 0 else p["m"] ** 2
    g2, G8 = p["g2"], p["eight_pi_G"]

    def rhs(tau, Y):
        a, ph, phd, ch, chd = Y
        V = cpl / beta * ph ** beta + 0.5 * g2 * ph * ph * ch * ch
        rho = 0.5 * (phd ** 2 + chd ** 2) + V
        H = math.sqrt(G8 * rho / 3)
        dV0 = cpl * ph ** (beta - 1) + g2 * ph * ch * ch
        dV1 = g2 * ph * ph * ch
        J = 1.0 / (B * a ** s)
        return [J * a * H, J * phd, J * (-3 * H * phd - dV0), J * chd, J * (-3 * H * chd - dV1)]

    Y0 = [1.0, p["phi0"][0], p["dphi0"][0], p["phi0"][1], p["dphi0"][1]]
    sol = solve_ivp(rhs, (0, tau_end), Y0, method="DOP853", rtol=1e-13, atol=1e-16, dense_output=True)
    def program(tau):
        a, ph, phd, ch, chd = sol.sol(tau)
        return a, A * a ** r * ph, A * a ** r * ch
    return program


def _homog_error(p, tau_end):
    ref = _ode_reference(p, tau_end + p["dt"])
    o = Oracle(p)
    o.init_fields()
    nsteps = int(round(tau_end / p["dt"]))
    errs = []
    for _ in range(4):
        o.step(nsteps // 4)
        sc = o.scalars()
        tau = sc["t"] + p["dt"] / 2
        a_ref, f_ref, _ = ref(tau)
        f = o.array(0, 0)
        assert np.ptp(f) == 0.0  # stays homogeneous
        errs.append(max(abs(sc["a"] / a_ref - 1), abs(f.flat[0] - f_ref)))
    return max(errs)


@pytest.mark.parametrize("model", ["lphi4", "m2phi2"])
def test_homogeneous_limit_matches_physical_ode(model):
    """With no fluctuations the lattice reduces to the homogeneous Friedmann +
    Klein-Gordon system. Integrated independently in physical variables (ODE
    solver at 1e-13), mapped with f = A a^r phi, the leapfrog's f and a must agree
    with error O(dt^2). Pins the rescaling (A, B, r, s), the sign of the f term of
    eq. scalar-evo (r(s-r+2), not the printed r(s-r-2)), eq. scale and the
    time-centred a' (a lagged a'' would give O(dt))."""
    if model == "lphi4":
        mk = lambda k: dict(lphi4(4, fluct=0.0), dt=0.04 / k)
        T = 6.0
    else:
        mk = lambda k: m2phi2(4, fluct=0.0, dt=0.02 / k)
        T = 8.0
    e1 = _homog_error(mk(1), T)
    e2 = _homog_error(mk(2), T)
    assert e1 < 3e-3
    assert 4 * 0.8 < e1 / e2 < 4 * 1.2, (e1, e2)


def test_friedmann_constraint_second_order():
    """Sec. III: the residual curvature K/(a^2H^2) = 8piG<rho>/(3H^2) - 1 is zero in
    the continuum; eq. scale only conserves it up to the O(dt^2) scheme error."""
    def run(k):
        p = m2phi2(4, fluct=0.0, dt=0.02 / k)
        o = Oracle(p)
        o.init_fields()
        worst = 0.0
        for _ in range(8):
            o.step(int(round(1.0 / p["dt"])))
            worst = max(worst, abs(o.energies()["curv_resid"]))
        return worst
    c1, c2 = run(1), run(2)
    assert c1 < 1e-3
    assert 4 * 0.75 < c1 / c2 < 4 * 1.25, (c1, c2)


def test_scale_update_solves_implicit_equation():
    """The a' update is the exact root of a'_{n+1} = a'_n + dt a''(a'_{n+1/2}) with
    a'' from eq. scale; residual at rounding level, and it reduces to the explicit
    update when s = -2 (no a'^2 term)."""
    p = lphi4(6)
    o = Oracle(p)
    o.init_fields()
    d = o.derived()
    a1, ah, add = o.scale_update()
    sc = o.scalars()
    assert abs(ah - 0.5 * (sc["ad"] + a1)) < 1e-15
    assert abs(a1 - (sc["ad"] + p["dt"] * add)) < 1e-15
    q = -(d["s"] + 2) / sc["a"]
    S = sc["S"]
    c = p["eight_pi_G"] / d["A"] ** 2 * sc["a"] ** (-2 * d["s"] - 2 * d["r"] - 1) * (
        (S[0] + S[1]) / 3 + sc["a"] ** (2 * d["s"] + 2) * (d["cdom0"] * S[2] + d["kappa0"] * S[3]))
    assert abs(add - (q * ah * ah + c)) < 1e-14 * abs(add)


# ------------------------------------------------------------------ initial conditions (P8)

def test_initial_spectrum_statistics():
    """DEFROST-style vacuum: the fluctuation of field i has shell-mean |F_k|^2 / n^3
    equal to the shell mean of (fluct A B)^2 dx^-3 / (2 w_k), w_k^2 = k_lat^2 + m_eff^2,
    within the chi^2 sampling error; k = 0 and |n| > kcut are empty; the mean is the
    homogeneous value."""
    n = 24
    p = lphi4(n, expansion=0, fluct=1.0)
    p["dt"] = 1e-12      # makes the half-step desync negligible
    o = Oracle(p)
    o.init_fields()
    d = o.derived()
    dx = d["dx"]
    amp2 = (d["A"] * d["B"]) ** 2 * dx ** -3
    k = np.fft.fftfreq(n) * n
    KX, KY, KZ = np.meshgrid(k, k, k, indexing="ij")
    nmag = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    klat2 = sum((2 / dx * np.sin(np.pi * K / n)) ** 2 for K in (KX, KY, KZ))
    fh = d["A"] * p["phi0"][0]
    meff2 = [3 * d["cdom0"] * fh ** 2, d["kappa0"] * fh ** 2]
    nb = n // 4 + 1
    for field in (0, 1):
        f = o.array(field, 0)
        assert abs(f.mean() - (fh if field == 0 else 0.0)) < 1e-12 * (abs(fh) if field == 0 else f.std())
        kk, pp, cc = o.spectrum(field, nb + 3)
        P = np.abs(np.fft.fftn(f - f.mean())) ** 2 / n ** 3
        expect = amp2 / (2 * np.sqrt(klat2 + meff2[field]))
        for b in range(1, nb + 3):
            sel = np.rint(nmag) == b
            # the oracle's spectrum against shell means of a library FFT; the field's
            # mean (1 against fluctuations of 1e-7) sets the FFT rounding floor
            assert cc[b] == sel.sum()
            assert abs(pp[b] - P[sel].mean()) <= 1e-6 * P[sel].mean() + 1e-12 * P.max()
            assert abs(kk[b] - (2 * np.pi / p["L"]) * nmag[sel].mean()) < 1e-12 * kk[b]
            inside = sel & (nmag <= n / 4)
            if b > n / 4 + 1:
                assert pp[b] <= 1e-12 * P.max()   # empty shell: FFT rounding floor only
                continue
            if inside.sum() < 50:
                continue
            ratio = P[inside].mean() / expect[inside].mean()
            sigma = 1 / math.sqrt(inside.sum() / 2)
            assert abs(ratio - 1) < 5 * sigma, (field, b, ratio, sigma)


def test_initial_state_is_desynchronised():
    """After init the fields are advanced by dt/2 with the initial momenta (and a by
    dt/2 with a'), Sec. II.B last paragraph."""
    n = 8
    p = lphi4(n)
    a = Oracle(dict(p, dt=1e-30)); a.init_fields()
    b = Oracle(p); b.init_fields()
    f0a, f1a, p0a, p1a = a.get_state()
    f0b, f1b, p0b, p1b = b.get_state()
    np.testing.assert_allclose(p0b, p0a, rtol=1e-15)
    np.testing.assert_allclose(f0b, f0a + 0.5 * p["dt"] * p0a, rtol=1e-14)
    np.testing.assert_allclose(f1b, f1a + 0.5 * p["dt"] * p1a, rtol=1e-14, atol=1e-30)
    assert abs(b.scalars()["a"] - (1 + 0.5 * p["dt"] * b.scalars()["ad"])) < 1e-15
    # H0 from the homogeneous energy: a'_0 = H0 / B with H0^2 = 8piG V(phi0)/3
    d = b.derived()
    H0 = math.sqrt(p["eight_pi_G"] * p["lam"] / 4 * p["phi0"][0] ** 4 / 3)
    assert abs(b.scalars()["ad"] - H0 / d["B"]) < 1e-12 * H0 / d["B"]


def test_results_do_not_depend_on_the_thread_count():
    """Every oracle sum is taken per z-plane and the planes are added in index
    order, so one thread and all threads give bit-identical steps, sums and
    energies (the CPU baseline is timed both ways)."""
    from oracle.oracle import set_threads
    n = 12
    p = lphi4(n, precision=64)
    st = random_state(n, 21, 64, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-3), pi_mean=(0.5, 0.0), pi_amp=(1e-3, 1e-3))
    out = []
    before = set_threads(0)
    try:
        for threads in (1, max(2, os.cpu_count() or 2)):
            set_threads(threads)
            o = Oracle(p)
            o.set_state(*st, t=0.0, a=1.1, ad=0.45)
            o.step(7)
            out.append((o.get_state(), o.scalars(), o.energies()))
    finally:
        set_threads(before)
    (s1, c1, e1), (s2, c2, e2) = out
    for x, y in zip(s1, s2):
        assert np.array_equal(x, y)
    assert c1 == c2
    assert e1 == e2
