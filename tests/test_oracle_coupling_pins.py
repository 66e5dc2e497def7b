"""Pins for the oracle's interaction term and its dependence on the scale factor.

The coupling g^2 phi^2 chi^2 / 2 enters the program-unit potential as
kappa0 a^pint f0^2 f1^2 / 2 (Sec. II.B: V_pr = (A^2/B^2) a^(2r-2s) V(f / (A a^r));
pint = -3 for the m^2 phi^2 model of Sec. III, 0 for lambda phi^4). These tests
reach it with both fields non-zero and, where it matters, with the universe
expanding, against references that share nothing with the oracle:

* the homogeneous Friedmann + Klein-Gordon system for BOTH fields, integrated in
  physical variables by an adaptive ODE solver (Sec. II.B eq. fe, eq. frw);
* static-space energy conservation of the coupled m^2 phi^2 model, which holds
  only if the force on each field is the derivative of the same potential;
* a brute-force restatement of whole steps on a 4^3 lattice: a dense 64 x 64
  Laplacian matrix, the program-unit potential built from the PHYSICAL potential
  and the rescaling definition, its derivatives by complex-step differentiation,
  the per-site sums by explicit loops and the implicit a' update solved by a
  bracketing root finder instead of the closed-form root.

A wrong power of a in the coupling (pint = -2 for m^2 phi^2), a dropped kappa term
in either force, or a coupling evaluated at the wrong time fails at least one of
them (checked by planting each in a scratch copy of the oracle).
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_0911_5692_gb300.workloads import lphi4, m2phi2, random_state


# ------------------------------------------------------------------ homogeneous limit, both fields (P6)

def _ode_two_fields(p, tau_end):
    """Homogeneous FRW with both scalar fields in physical variables, program time
    as the independent variable (dt_pr = B a^s dt); the Friedmann constraint
    H^2 = 8 pi G rho / 3 gives H (Sec. II.B). Returns tau -> (a, f0, f1) in
    program units, f_i = A a^r phi_i with the paper's rescaling rule."""
    from scipy.integrate import solve_ivp
    beta = 4.0 if p["model"] == 0 else 2.0
    cpl = p["lam"] if p["model"] == 0 else p["m"] ** 2
    phi0 = p["phi0"][0]
    A = 1.0 / phi0
    B = math.sqrt(cpl) * abs(phi0) ** (beta / 2 - 1)
    r = 6.0 / (2.0 + beta)
    s = 3.0 * (2.0 - beta) / (2.0 + beta)
    g2, G8 = p["g2"], p["eight_pi_G"]

    def rhs(tau, Y):
        a, ph, phd, ch, chd = Y
        V = cpl / beta * ph ** beta + 0.5 * g2 * ph * ph * ch * ch
        H = math.sqrt(G8 * (0.5 * (phd ** 2 + chd ** 2) + V) / 3)
        J = 1.0 / (B * a ** s)
        return [J * a * H, J * phd, J * (-3 * H * phd - cpl * ph ** (beta - 1) - g2 * ph * ch * ch),
                J * chd, J * (-3 * H * chd - g2 * ph * ph * ch)]

    Y0 = [1.0, p["phi0"][0], p["dphi0"][0], p["phi0"][1], p["dphi0"][1]]
    sol = solve_ivp(rhs, (0, tau_end), Y0, method="DOP853", rtol=1e-13, atol=1e-16, dense_output=True)

    def program(tau):
        a, ph, _, ch, _ = sol.sol(tau)
        return a, A * a ** r * ph, A * a ** r * ch
    return program


def _coupled_params(model, k):
    """Both fields homogeneous and non-zero, expansion on, a coupling that moves
    chi on the time scale of phi (program mass of chi about sqrt(2) at the start)."""
    if model == "lphi4":
        p = dict(lphi4(4, fluct=0.0, G=2.0), dt=0.04 / k)
        p["phi0"] = (0.342, 0.06)
        return p, 6.0
    # m^2 phi^2: G_m = g^2 phi0^2 / m^2 = 2, chi0 = 0.15 (reduced Planck units)
    p = m2phi2(4, fluct=0.0, dt=0.02 / k, g2=2.0e-12 / 1.009343 ** 2)
    p["phi0"] = (1.009343, 0.15)
    return p, 8.0


def _coupled_error(p, T):
    ref = _ode_two_fields(p, T + p["dt"])
    o = Oracle(p)
    o.init_fields()
    nsteps = int(round(T / p["dt"]))
    ea = ef0 = ef1 = 0.0
    a_end = None
    chi_scale = 0.0
    for _ in range(8):
        o.step(nsteps // 8)
        sc = o.scalars()
        tau = sc["t"] + p["dt"] / 2
        a_ref, f0_ref, f1_ref = ref(tau)
        f0, f1 = o.array(0, 0), o.array(1, 0)
        assert np.ptp(f0) == 0.0 and np.ptp(f1) == 0.0   # stays homogeneous
        chi_scale = max(chi_scale, abs(f1_ref))
        ea = max(ea, abs(sc["a"] / a_ref - 1))
        ef0 = max(ef0, abs(f0.flat[0] - f0_ref))
        ef1 = max(ef1, abs(f1.flat[0] - f1_ref))
        a_end = sc["a"]
    return ea, ef0, ef1 / chi_scale, a_end


@pytest.mark.parametrize("model", ["lphi4", "m2phi2"])
def test_homogeneous_limit_with_coupling(model):
    """Both fields homogeneous and non-zero under expansion: the leapfrog's a, f_phi
    and f_chi follow the independent physical ODE with error O(dt^2) (halving dt
    divides every error by 4 within 20 %). The interaction acts on both fields and,
    for m^2 phi^2, carries a^-3: with a growing several-fold over the run a wrong
    power of a, a missing kappa term in either force or a coupling taken at the
    wrong time shows as an O(1) error or as first-order convergence."""
    p1, T = _coupled_params(model, 1)
    p2, _ = _coupled_params(model, 2)
    e1 = _coupled_error(p1, T)
    e2 = _coupled_error(p2, T)
    assert e1[3] > 2.0, "the run must expand enough for the a-dependence to matter"
    for k, what in enumerate(("a", "f_phi", "f_chi")):
        assert e1[k] < 5e-3, (what, e1[k])
        assert 4 * 0.8 < e1[k] / e2[k] < 4 * 1.2, (what, e1[k], e2[k])


# ------------------------------------------------------------------ energy, coupled m^2 phi^2 (P3)

def _energy_drift_m2(dt):
    n = 8
    # static space, G_m = g^2 phi0^2 / m^2 = 2: program-unit potential f0^2/2 + f0^2 f1^2
    p = m2phi2(n, fluct=0.0, expansion=0, dt=dt, g2=2.0e-12 / 1.009343 ** 2)
    p["L"] = 8.0
    o = Oracle(p)
    st = random_state(n, 9, precision=64, f_mean=(1.0, 0.3), f_amp=(0.05, 0.05), pi_mean=(0.0, 0.0),
                      pi_amp=(0.0, 0.0))
    sm = []
    for a in st[:2]:
        F = np.fft.fftn(a)
        k = np.fft.fftfreq(n) * n
        kk = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
        F[kk > 1.5] = 0
        F[0, 0, 0] = a.sum()
        sm.append(np.real(np.fft.ifftn(F)))
    o.set_state(sm[0], sm[1], np.zeros((n, n, n)), np.zeros((n, n, n)))
    nsteps = int(round(6.0 / dt))
    E0 = o.energies()["rho"]
    drift = 0.0
    chunk = max(1, nsteps // 60)
    for _ in range(nsteps // chunk):
        o.step(chunk)
        drift = max(drift, abs(o.energies()["rho"] / E0 - 1))
    return drift


def test_energy_conservation_coupled_m2phi2():
    """Static space, m^2 phi^2 with the coupling switched on (both fields non-zero):
    the total energy (kinetic + gradient + m^2 phi^2/2 + g^2 phi^2 chi^2/2) drifts
    as O(dt^2). Energy is conserved only if each force is the derivative of the
    potential whose average the energy uses, so a kappa term dropped from or
    scaled differently in either force, or in the potential, gives a drift that
    does not fall with dt."""
    d1 = _energy_drift_m2(0.04)
    d2 = _energy_drift_m2(0.02)
    assert d1 < 1e-2
    assert 4 * 0.8 < d1 / d2 < 4 * 1.2, (d1, d2)


# ------------------------------------------------------------------ brute force, whole steps on 4^3 (P5)

def _dense_laplacian(n, dx):
    N = n ** 3
    M = np.zeros((N, N))
    for z in range(n):
        for y in range(n):
            for x in range(n):
                i = (z * n + y) * n + x
                for dz, dy, dxx in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]:
                    j = (((z + dz) % n) * n + (y + dy) % n) * n + (x + dxx) % n
                    M[i, j] += 1.0
                    M[i, i] -= 1.0
    return M / (dx * dx)


class _Restated:
    """One lattice stepped by a plain restatement of Sec. II.B, written without
    the oracle: program units from the rescaling definition, the potential from
    the physical one, eq. scalar-evo, eq. scale and the staggered leapfrog."""

    def __init__(self, p):
        self.n = p["n"]
        self.dx = p["L"] / self.n
        self.dt = p["dt"]
        self.expansion = p["expansion"]
        self.G8 = p["eight_pi_G"]
        self.beta = 4.0 if p["model"] == 0 else 2.0
        self.cpl = p["lam"] if p["model"] == 0 else p["m"] ** 2
        self.g2 = p["g2"]
        phi0 = p["phi0"][0]
        self.A = 1.0 / phi0
        self.B = math.sqrt(self.cpl) * abs(phi0) ** (self.beta / 2 - 1)
        self.r = 6.0 / (2.0 + self.beta)
        self.s = 3.0 * (2.0 - self.beta) / (2.0 + self.beta)
        self.M = _dense_laplacian(self.n, self.dx)

    def V_phys(self, phi, chi):
        return self.cpl / self.beta * phi ** self.beta + 0.5 * self.g2 * phi * phi * chi * chi

    def V_pr(self, f0, f1, a):
        """Sec. II.B: V_pr = (A^2/B^2) a^(2r-2s) V(f / (A a^r))."""
        sc = self.A * a ** self.r
        return (self.A / self.B) ** 2 * a ** (2 * self.r - 2 * self.s) * self.V_phys(f0 / sc, f1 / sc)

    def dV_pr(self, f0, f1, a):
        """Both field derivatives of V_pr by complex-step differentiation (exact to
        rounding for an analytic function: no difference of nearby values)."""
        h = 1e-30
        d0 = np.imag(self.V_pr(f0 + 1j * h, f1.astype(complex), a)) / h
        d1 = np.imag(self.V_pr(f0.astype(complex), f1 + 1j * h, a)) / h
        return d0, d1

    def grad2_mean(self, f):
        """<|grad f|^2> by forward differences, one site at a time."""
        n, acc = self.n, 0.0
        for z in range(n):
            for y in range(n):
                for x in range(n):
                    c = f[z, y, x]
                    acc += ((f[z, y, (x + 1) % n] - c) ** 2 + (f[z, (y + 1) % n, x] - c) ** 2
                            + (f[(z + 1) % n, y, x] - c) ** 2)
        return acc / (self.dx * self.dx) / n ** 3

    def step(self, f, pi, a, ad):
        """One step: f (two fields, t + dt/2), pi (t), a (t + dt/2), a' (t)."""
        dt, r, s = self.dt, self.r, self.s
        cL, cF, ad_next = 1.0, 0.0, 0.0
        if self.expansion:
            g2m = self.grad2_mean(f[0]) + self.grad2_mean(f[1])
            vm = float(np.mean(self.V_pr(f[0], f[1], a)))
            c = self.G8 / self.A ** 2 * a ** (-2 * s - 2 * r - 1) * (g2m / 3 + a ** (2 * s + 2) * vm)

            def resid(x):   # eq. scale with a'' at the field time from the mean momentum
                return x - ad - dt * (-(s + 2) / a * (0.5 * (ad + x)) ** 2 + c)
            from scipy.optimize import brentq
            w = 0.1 * abs(ad) + dt * abs(c) + 1e-12
            ad_next = brentq(resid, ad - 10 * w, ad + 10 * w, xtol=1e-300, rtol=1e-15, maxiter=500)
            ad_half = 0.5 * (ad + ad_next)
            add = -(s + 2) / a * ad_half ** 2 + c
            h = ad_half / a
            cL = a ** (-2 * s - 2)
            cF = r * (s - r + 2) * h * h + r * add / a
        d0, d1 = self.dV_pr(f[0], f[1], a)
        n3 = self.n ** 3
        lap = [(self.M @ f[i].reshape(n3)).reshape(f[i].shape) for i in (0, 1)]
        pi_new = [pi[0] + dt * (cL * lap[0] + cF * f[0] - d0), pi[1] + dt * (cL * lap[1] + cF * f[1] - d1)]
        f_new = [f[i] + dt * pi_new[i] for i in (0, 1)]
        a_new = a + dt * ad_next if self.expansion else a
        return f_new, pi_new, a_new, ad_next if self.expansion else 0.0

    def sums(self, f, a):
        """(<|grad f0|^2>, <|grad f1|^2>, <f0^beta/beta>, <f0^2 f1^2/2>, <V_pr>) by loops."""
        n, b = self.n, self.beta
        sd = si = 0.0
        for z in range(n):
            for y in range(n):
                for x in range(n):
                    u, v = f[0][z, y, x], f[1][z, y, x]
                    sd += u ** b / b
                    si += 0.5 * u * u * v * v
        return (self.grad2_mean(f[0]), self.grad2_mean(f[1]), sd / n ** 3, si / n ** 3,
                float(np.mean(self.V_pr(f[0], f[1], a))))


def _rel(x, ref):
    return float(np.max(np.abs(np.asarray(x) - np.asarray(ref))) / max(np.max(np.abs(ref)), 1e-300))


@pytest.mark.parametrize("model", ["lphi4", "m2phi2"])
@pytest.mark.parametrize("expansion", [0, 1])
def test_brute_force_full_steps_4(model, expansion):
    """P5 in full: three consecutive steps of a 4^3 lattice with both fields
    fluctuating, a = 1.3 and a' = 0.4 (expansion on) restated independently and
    compared with the oracle at 1e-14 normwise: fields, momenta, a, a', the four
    sums and <V_pr> rebuilt from the oracle's derived constants. The coupling is
    large enough that its terms move every field at 1e-3 or more per step."""
    n = 4
    if model == "lphi4":
        p = dict(lphi4(n, precision=64, expansion=expansion, G=3.0), dt=0.05)
    else:
        p = m2phi2(n, precision=64, expansion=expansion, dt=0.05, g2=3.0e-12 / 1.009343 ** 2)
    st = random_state(n, 77, precision=64, f_mean=(1.0, 0.2), f_amp=(0.05, 0.1), pi_mean=(0.3, 0.05),
                      pi_amp=(0.05, 0.1))
    a0, ad0 = (1.3, 0.4) if expansion else (1.0, 0.0)
    o = Oracle(p)
    o.set_state(*st, t=0.0, a=a0, ad=ad0)
    R = _Restated(p)
    f, pi, a, ad = [st[0], st[1]], [st[2], st[3]], a0, ad0
    d = o.derived()
    for k in range(3):
        f, pi, a, ad = R.step(f, pi, a, ad)
        o.step(1)
        of0, of1, op0, op1 = o.get_state()
        for x, ref in ((of0, f[0]), (of1, f[1]), (op0, pi[0]), (op1, pi[1])):
            assert _rel(x, ref) <= 1e-14, (k, _rel(x, ref))
        sc = o.scalars()
        assert abs(sc["a"] - a) <= 1e-14 * a
        assert abs(sc["ad"] - ad) <= 1e-14 * max(abs(ad), 1e-300) or ad == sc["ad"] == 0.0
        S = R.sums(f, a)
        for j in range(4):
            assert abs(sc["S"][j] - S[j]) <= 1e-14 * abs(S[j]), (k, j, sc["S"][j], S[j])
        vpr = d["cdom0"] * a ** d["pdom"] * sc["S"][2] + d["kappa0"] * a ** d["pint"] * sc["S"][3]
        assert abs(vpr - S[4]) <= 1e-14 * abs(S[4]), (k, vpr, S[4])
