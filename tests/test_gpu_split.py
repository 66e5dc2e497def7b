"""Split storage of the inflaton (lat_params.split = 1): phi held as an FP64
homogeneous mode plus fluctuation arrays, against the FP64 oracle, which holds
phi whole.

The scheme is the same leapfrog as for phi stored whole (Sec. II.B, eq. evo
with eq. scalar-evo and eq. scale); what changes is the precision with which
FP32 arrays hold the inflaton's fluctuations. So besides the whole-field bounds
of the other parity tests (2e-6 normwise FP32 per step, 1e-12 FP64) the
fluctuation parts are held to bounds relative to their OWN size,
    max |phi - phi_ref| / max |phi_ref - <phi_ref>|,
which FP32 arrays storing phi whole cannot meet (their rounding of phi ~ 1 is
6e-8, i.e. 6e-5 of fluctuations of 1e-3, and more than the fluctuations
themselves at the vacuum amplitude of the paper's runs).
"""
import math

import numpy as np
import pytest

from gpu_helpers import normwise
from oracle.oracle import Oracle
from paper_0911_5692_gb300 import Lattice, LatticeError
from paper_0911_5692_gb300.workloads import lphi4, m2phi2, random_state

pytestmark = pytest.mark.gpu

TOL = {32: 2e-6, 64: 1e-12}


def fluct_err(x, ref):
    """max |x - ref| / max |ref - mean(ref)|: an error relative to the
    fluctuation part of a field."""
    ref = np.asarray(ref)
    return float(np.max(np.abs(np.asarray(x) - ref)) / np.max(np.abs(ref - ref.mean())))


def _params(model, n, prec, expansion, stencil=7):
    if model == "lphi4":
        p = lphi4(n, precision=prec, expansion=expansion, split=1)
    else:
        p = m2phi2(n, precision=prec, expansion=expansion, split=1)
    return dict(p, stencil=stencil)


def _state(model, n, prec, seed):
    if model == "lphi4":
        return random_state(n, seed, precision=prec, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-3),
                            pi_mean=(0.5, 0.0), pi_amp=(1e-3, 1e-3))
    return random_state(n, seed, precision=prec, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-4),
                        pi_mean=(0.3, 0.0), pi_amp=(1e-3, 1e-2))


def _pair(p, st, sc):
    g = Lattice(p)
    g.set_state(*st, t=sc[0], a=sc[1], ad=sc[2], step=sc[3])
    o = Oracle(p)
    o.set_state(*st, t=sc[0], a=sc[1], ad=sc[2], step=sc[3])
    return g, o


def _check_step(g, o, prec, what, steps=1):
    gs, os_ = g.get_state_exact(), o.get_state()
    for name, x, r in zip(("f0", "f1", "p0", "p1"), gs, os_):
        assert normwise(x, r) <= steps * TOL[prec], (what, name, normwise(x, r))
    # the inflaton's fluctuation parts, relative to their own size
    for name, x, r in (("f0", gs[0], os_[0]), ("p0", gs[2], os_[2])):
        assert fluct_err(x, r) <= steps * TOL[prec], (what, name, fluct_err(x, r))


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("kernel", ["v2", "v4", "v5", "27"])
@pytest.mark.parametrize("model,expansion", [("lphi4", 1), ("m2phi2", 1), ("lphi4", 0)])
@pytest.mark.parametrize("n", [16, 36, 64])
def test_split_one_step_parity(n, model, expansion, kernel, prec):
    """One step of a split lattice from the oracle's state (whole fields, moved
    to zero-mean fluctuations by lat_recenter): whole fields within the per-step
    bound and the inflaton's fluctuations within the same bound relative to their
    own size; a, a' and the four sums of the new fields."""
    p = _params(model, n, prec, expansion, stencil=27 if kernel == "27" else 7)
    st = _state(model, n, prec, seed=n + prec)
    sc = (0.0, 1.2, 0.4, 0) if expansion else (0.0, 1.0, 0.0, 0)
    g, o = _pair(p, st, sc)
    if kernel in ("v4", "v5"):
        try:
            g.set_kernel(int(kernel[1]))
        except LatticeError:
            pytest.skip("x-tiled kernel does not serve this lattice")
    P, Pi = g.background()
    assert abs(P - st[0].mean()) <= 1e-15 and abs(Pi - st[2].mean()) <= 1e-15
    g.evolve(1)
    o.step(1)
    _check_step(g, o, prec, f"N={n} {model} exp={expansion} {kernel} fp{prec}")
    gs, os_ = g.scalars(), o.scalars()
    ta, tad = (1e-14, 1e-13) if prec == 64 else (1e-8, 1e-7)
    assert abs(gs["a"] - os_["a"]) <= ta * os_["a"]
    assert abs(gs["ad"] - os_["ad"]) <= tad * max(abs(os_["ad"]), 1.0)
    # the FP32 sums of the fluctuations keep FP32 precision of their own size
    stol = [1e-11, 1e-11, 1e-13, 1e-11] if prec == 64 else [1e-5, 1e-5, 1e-7, 1e-5]
    if kernel == "27" and prec == 64:
        stol[0] = stol[1] = 1e-9   # the oracle's -<f L27 f> cancels the mean of f
    for k in range(4):
        ref = os_["S"][k]
        assert abs(gs["S"][k] - ref) <= stol[k] * abs(ref) + 1e-300, (k, gs["S"][k], ref)


@pytest.mark.parametrize("prec", [32, 64])
def test_split_ten_steps(prec):
    """Ten steps of the 32^3 lambda phi^4 lattice: the homogeneous mode advances in
    the last block of every step from the same coefficients as the arrays."""
    n = 32
    p = lphi4(n, precision=prec, split=1)
    st = _state("lphi4", n, prec, seed=3)
    g, o = _pair(p, st, (0.0, 1.1, 0.45, 0))
    g.evolve(10)
    o.step(10)
    _check_step(g, o, prec, "10 steps", steps=10)
    assert abs(g.scalars()["a"] / o.scalars()["a"] - 1) <= (1e-13 if prec == 64 else 1e-7)


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("model", ["lphi4", "m2phi2"])
def test_split_init_parity(model, prec):
    """DEFROST-style initial conditions of a split lattice: the homogeneous values
    go to the FP64 mode, the vacuum fluctuations (1e-7 of phi for lambda phi^4 at
    32^3) to the arrays; against the oracle's own initialisation, the fluctuations
    of phi and its momentum agree to FP32 rounding of their own size."""
    p = _params(model, 32, prec, 1)
    p["seed"] = 12345
    g = Lattice(p)
    g.init_fields()
    o = Oracle(p)
    o.init_fields()
    gs, os_ = g.get_state_exact(), o.get_state()
    tol = 1e-13 if prec == 64 else 2e-7
    for name, x, r in zip(("f0", "f1", "p0", "p1"), gs, os_):
        assert normwise(x, r) <= tol, (name, normwise(x, r))
    for name, x, r in (("f0", gs[0], os_[0]), ("p0", gs[2], os_[2])):
        # the oracle holds phi whole in FP64: its own resolution of the
        # fluctuations is a few ulp of phi
        res = 8 * 2.0 ** -53 * np.max(np.abs(r)) / np.max(np.abs(r - r.mean()))
        assert fluct_err(x, r) <= max(tol, res), (name, fluct_err(x, r), res)
    P, Pi = g.background()
    d = o.derived()
    assert abs(P - (d["A"] * p["phi0"][0] + 0.5 * p["dt"] * Pi)) <= 1e-15 * abs(P)
    assert abs(g.scalars()["a"] - o.scalars()["a"]) <= 1e-15


@pytest.mark.parametrize("fluct", [1.0])
def test_split_run_statistics_vacuum(fluct):
    """The 32^3 lambda phi^4 run on the FP32 split path against the FP64 oracle from
    the same start (the lattice's own state in FP64), every 100 of 1000 steps:
    <phi>, var phi, var chi, the total energy and a within 1e-3, at the vacuum
    amplitude, where FP32 arrays holding phi whole cannot resolve var phi at all
    (fluctuations of 1.6e-7 about 1)."""
    p = lphi4(32, precision=32, fluct=fluct, split=1)
    g = Lattice(p)
    g.init_fields()
    st = g.get_state_exact()
    sc = g.scalars()
    o = Oracle(dict(p, precision=64))
    o.set_state(*st, t=sc["t"], a=sc["a"], ad=sc["ad"], step=sc["step"])
    for _ in range(10):
        g.evolve(100)
        o.step(100)
        eg, eo = g.energies(), o.energies()
        assert abs(eg["a"] / eo["a"] - 1) <= 1e-3
        assert abs(eg["rho"] / eo["rho"] - 1) <= 1e-3
        assert abs(eg["mean0"] - eo["mean0"]) <= 1e-3 * math.sqrt(eo["var0"])
        assert abs(eg["mean1"] - eo["mean1"]) <= 1e-3 * math.sqrt(eo["var1"])
        assert abs(eg["var0"] / eo["var0"] - 1) <= 1e-3, (eg["var0"], eo["var0"])
        assert abs(eg["var1"] / eo["var1"] - 1) <= 1e-3


def test_split_against_whole_fp32():
    """The point of split storage, measured: 200 steps of the 32^3 lambda phi^4
    vacuum state in FP32, whole and split, against FP64 from the same initial
    conditions. Split keeps the inflaton's fluctuations to 1e-4 of their size;
    stored whole they are lost (errors of order one or more)."""
    p = lphi4(32, precision=64)
    ref = Lattice(p)
    ref.init_fields()
    ref.evolve(200)
    r = ref.get_state()
    s = Lattice(dict(p, precision=32, split=1))
    s.init_fields()
    s.evolve(200)
    x = s.get_state_exact()
    w = Lattice(dict(p, precision=32, split=0))
    w.init_fields()
    w.evolve(200)
    y = w.get_state()
    for k in (0, 2):
        assert fluct_err(x[k], r[k]) <= 1e-4, fluct_err(x[k], r[k])
        assert fluct_err(y[k], r[k]) >= 1e-1, fluct_err(y[k], r[k])


def test_background_moves_keep_the_state():
    """lat_set_background re-expresses the stored arrays about another homogeneous
    mode (the fields do not change beyond one rounding of the fluctuations), and
    the evolution from either representation agrees to FP32 precision of the
    fluctuations; lat_recenter leaves fluctuations of zero mean."""
    n = 32
    p = lphi4(n, precision=32, split=1)
    st = _state("lphi4", n, 32, seed=8)
    a = Lattice(p)
    a.set_state(*st, t=0.0, a=1.1, ad=0.45)
    b = Lattice(p)
    b.set_state(*st, t=0.0, a=1.1, ad=0.45)
    P, Pi = b.background()
    b.set_background(P + 3e-4, Pi - 2e-4)
    assert b.background() == (P + 3e-4, Pi - 2e-4)
    # one FP32 rounding of the shifted fluctuations
    for x, y, s in zip(a.get_state_exact(), b.get_state_exact(), b.get_state_stored()):
        assert np.max(np.abs(x - y)) <= 2.0 ** -24 * np.max(np.abs(s))
    a.evolve(5)
    b.evolve(5)
    for k, (x, y) in enumerate(zip(a.get_state_exact(), b.get_state_exact())):
        assert fluct_err(y, x) <= 1e-5, (k, fluct_err(y, x))
    b.recenter()
    f0, _, p0, _ = b.get_state_stored()
    assert abs(f0.mean()) <= 1e-9 and abs(p0.mean()) <= 1e-9


def test_split_checkpoint_and_whole_exchange():
    """A checkpoint carries the homogeneous mode (bit-identical resume), and
    lat_get_state / lat_set_state exchange whole fields on a split lattice
    (stored + mode on the way out, minus the mode on the way in)."""
    n = 32
    p = lphi4(n, precision=32, split=1)
    g = Lattice(p)
    g.init_fields()
    g.evolve(7)
    blob = g.save_checkpoint()
    g.evolve(40)
    ref = g.get_state_stored()
    h = Lattice(p)
    h.load_checkpoint(blob)
    h.evolve(40)
    for x, y in zip(ref, h.get_state_stored()):
        assert np.array_equal(x, y)
    assert g.background() == h.background()
    whole = g.get_state()
    P, Pi = g.background()
    assert np.max(np.abs(whole[0] - (ref[0] + P))) <= 2 ** -24 * (abs(P) + 1)
    assert np.max(np.abs(whole[2] - (ref[2] + Pi))) <= 2 ** -24 * (abs(Pi) + 1)


@pytest.mark.parametrize("prec", [32, 64])
def test_split_diagnostics(prec):
    """Energies, the per-site energy density and the spectrum of a split lattice
    against the oracle on the same state: they see phi whole."""
    n = 32
    p = lphi4(n, precision=prec, split=1)
    st = _state("lphi4", n, prec, seed=17)
    g, o = _pair(p, st, (0.0, 1.1, 0.45, 0))
    g.evolve(3)
    o.step(3)
    eg, eo = g.energies(), o.energies()
    tol = 1e-10 if prec == 64 else 1e-5
    for k in ("rho", "p", "kin0", "kin1", "grad0", "grad1", "pot", "mean0", "var0", "var1"):
        assert abs(eg[k] - eo[k]) <= tol * abs(eo[k]), (k, eg[k], eo[k])
    rho, pres = g.energy_field()
    rho_o, pres_o = o.energy_field()
    assert normwise(rho.double().cpu().numpy(), rho_o) <= (1e-12 if prec == 64 else 2e-6)
    assert normwise(pres.double().cpu().numpy(), pres_o) <= (1e-12 if prec == 64 else 2e-6)
    k, pw, c = g.spectrum(0, 17)
    ko, pwo, co = o.spectrum(0, 17)
    assert np.array_equal(c, co)
    np.testing.assert_allclose(pw, pwo, rtol=1e-9 if prec == 64 else 1e-4)


def test_split_lform():
    """The L = 1/H form on a split lattice: its read-only pass sees phi whole."""
    n = 32
    p = lphi4(n, precision=32, expansion=2, split=1)
    st = _state("lphi4", n, 32, seed=5)
    g, o = _pair(p, st, (0.0, 1.1, 0.45, 0))
    g.evolve(2)
    o.step(2)
    _check_step(g, o, 32, "L form", steps=2)
    assert abs(g.hubble_length() / o.ell() - 1) <= 1e-7


def test_split_ensemble_members():
    """Ensemble members stored split evolve as single split lattices do."""
    from paper_0911_5692_gb300 import Ensemble
    ps = [lphi4(32, precision=32, split=1, seed=1), lphi4(48, precision=32, split=1, G=80.0, seed=2)]
    ens = Ensemble(ps)
    ens.init_fields()
    ens.evolve(20)
    ens.sync()
    for i, p in enumerate(ps):
        g = Lattice(p)
        g.init_fields()
        g.evolve(20)
        m = ens.member(i)
        x, y = g.get_state_exact(), m.get_state_exact()
        for k in range(4):
            assert normwise(y[k], x[k]) <= 1e-6
        assert fluct_err(y[0], x[0]) <= 1e-5 and fluct_err(y[2], x[2]) <= 1e-5
        assert abs(g.scalars()["a"] / m.scalars()["a"] - 1) <= 1e-12
        for u, v in zip(g.background(), m.background()):
            assert abs(u - v) <= 1e-12 * abs(u)


def test_split_derivative_is_refused():
    p = lphi4(16, precision=32, split=1)
    g = Lattice(p)
    g.init_fields()
    with pytest.raises(LatticeError) as e:
        g.adjoint(4)
    assert e.value.status == 7   # LAT_EUNSUPPORTED


def test_background_calls_on_a_whole_lattice():
    g = Lattice(lphi4(16, precision=32))
    g.init_fields()
    assert g.background() == (0.0, 0.0)
    with pytest.raises(LatticeError) as e:
        g.recenter()
    assert e.value.status == 8   # LAT_ESTATE
    with pytest.raises(LatticeError):
        g.set_background(1.0, 0.0)


def test_m2phi2_run_statistics_through_the_resonance():
    """The m^2 phi^2 model with the couplings of the paper's run (m = 1e-6,
    g^2 = 2.5e-7, dt = 2^-10, Sec. III) at 32^3 on the FP32 split path against the
    FP64 oracle from the same start, every 1000 steps through the linear stage of
    the resonance, in which var chi grows by more than nine orders of magnitude:
    a, rho, var phi and var chi within 1e-3 relative and <phi> within 1e-3 of its
    oscillation amplitude. The comparison ends at the first sample where the
    inflaton's fluctuations have grown to var phi > 1e-3 of its oscillation
    amplitude squared (backreaction; near step 68000 here): past that point the
    dynamics are chaotic, and two FP64 runs that differ only in the order of
    their sums (this library's FP64 path and the oracle) separate by a factor of
    about 30 per 4000 steps, from 1e-13 to 1e-3 by the end of the growth of chi
    (measured at this size), so no finite-precision run can be held to a fixed
    tolerance beyond it."""
    p = m2phi2(32, precision=32, split=1)
    g = Lattice(p)
    g.init_fields()
    st = g.get_state_exact()
    sc = g.scalars()
    o = Oracle(dict(p, precision=64))
    o.set_state(*st, t=sc["t"], a=sc["a"], ad=sc["ad"], step=sc["step"])
    chunk = 1000
    var1_start, amp, end = None, 0.0, None
    for k in range(1, 131):
        g.evolve(chunk)
        o.step(chunk)
        eg, eo = g.energies(), o.energies()
        var1_start = var1_start if var1_start is not None else eo["var1"]
        amp = max(amp, abs(eo["mean0"]))
        where = f"step {k * chunk}"
        assert abs(eg["a"] / eo["a"] - 1) <= 1e-3, where
        assert abs(eg["rho"] / eo["rho"] - 1) <= 1e-3, where
        assert abs(eg["mean0"] - eo["mean0"]) <= 1e-3 * amp, (where, eg["mean0"], eo["mean0"])
        assert abs(eg["var0"] / eo["var0"] - 1) <= 1e-3, (where, eg["var0"], eo["var0"])
        assert abs(eg["var1"] / eo["var1"] - 1) <= 1e-3, (where, eg["var1"], eo["var1"])
        if eo["var0"] > 1e-3 * amp * amp:
            end = k * chunk
            growth = eo["var1"] / var1_start
            break
    assert end is not None, "no backreaction within 130000 steps"
    assert growth > 1e9, growth   # the run went through the resonance


@pytest.mark.parametrize("expansion", [1, 2])
def test_benchmark_configuration_512(expansion):
    """The benchmark's workload as it runs: the 512^3 lambda phi^4 lattice in FP32
    with phi stored split, the default kernel (variant 5, two planes in flight)
    and eq. scale (expansion 1) or the L = 1/H form with its pass (expansion 2):
    one step against the oracle's full-lattice step, the inflaton's fluctuations
    to the per-step bound relative to their own size, a, a' and the sums."""
    from paper_0911_5692_gb300.workloads import WORKLOADS
    p = dict(WORKLOADS["lphi4_512_fp32"]["params"], expansion=expansion)
    assert p["split"] == 1 and p["n"] == 512 and p["precision"] == 32
    st = _state("lphi4", 512, 32, seed=512 + expansion)
    g, o = _pair(p, st, (0.0, 1.02, 0.5, 0))
    del st
    info = g.kernel_info()
    assert (info["variant"], info["depth"]) == (5, 2)
    g.evolve(1)
    o.step(1)
    _check_step(g, o, 32, f"benchmark configuration 512 expansion {expansion}")
    gs, os_ = g.scalars(), o.scalars()
    assert abs(gs["a"] - os_["a"]) <= 1e-8 * os_["a"]
    assert abs(gs["ad"] - os_["ad"]) <= 1e-7 * max(abs(os_["ad"]), 1.0)
    for k, tol in enumerate([1e-5, 1e-5, 1e-7, 1e-5]):
        ref = os_["S"][k]
        assert abs(gs["S"][k] - ref) <= tol * abs(ref) + 1e-300, (k, gs["S"][k], ref)
    o.close()
