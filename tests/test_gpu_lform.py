"""GPU parity of the L = 1/H form of the scale-factor update (expansion = 2): the
CUDA path (step kernel plus the read-only pass whose last block solves the
implicit midpoint equations for l and the f coefficient) against the FP64 oracle
on identical seeded inputs.

Tolerances as for eq. scale: FP32 path 2e-6 normwise per step, FP64 1e-12 (also
over 1000 steps of the 32^3 lambda phi^4 run), run statistics 1e-3. The scalars
a, a' and l are FP64 on both sides; an FP32 lattice forms the four sums of the
solve in FP32 (compensated per thread, ~1e-7 relative), which moves l by about
dt times that.
"""
import math

import numpy as np
import pytest

from gpu_helpers import compare_states, normwise, paired
from oracle.oracle import Oracle
from paper_0911_5692_gb300 import Ensemble, Lattice, LatticeError
from paper_0911_5692_gb300.workloads import lphi4, m2phi2, random_state

pytestmark = pytest.mark.gpu

TOL = {32: 2e-6, 64: 1e-12}
VARIANTS = [2, 4, 5]


def _params(model, n, prec, stencil=7):
    mk = lphi4 if model == "lphi4" else m2phi2
    return dict(mk(n, precision=prec, expansion=2), stencil=stencil)


def _state(model, n, prec, seed):
    if model == "lphi4":
        return random_state(n, seed, precision=prec, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-3),
                            pi_mean=(0.5, 0.0), pi_amp=(1e-3, 1e-3))
    return random_state(n, seed, precision=prec, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-4),
                        pi_mean=(0.3, 0.0), pi_amp=(1e-3, 1e-2))


def _variant_ok(g, variant):
    try:
        g.set_kernel(variant)
        return True
    except LatticeError:
        return False


def _check_scalars(g, o, prec, steps=1):
    gs, os_ = g.scalars(), o.scalars()
    assert gs["step"] == os_["step"]
    ta, tad, tl = (1e-13, 1e-12, 1e-13) if prec == 64 else (1e-8 * steps, 1e-7 * steps, 1e-8 * steps)
    assert abs(gs["a"] - os_["a"]) <= ta * os_["a"], (gs["a"], os_["a"])
    assert abs(gs["ad"] - os_["ad"]) <= tad * abs(os_["ad"]), (gs["ad"], os_["ad"])
    assert abs(g.hubble_length() - o.ell()) <= tl * abs(o.ell()), (g.hubble_length(), o.ell())


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("model", ["lphi4", "m2phi2"])
@pytest.mark.parametrize("n", [4, 16, 36, 64])
def test_one_step_parity(n, model, prec, variant):
    """One step from an identical stored state (several tiles, ragged N = 36,
    degenerate N = 4): f, f', a, a' and l."""
    p = _params(model, n, prec)
    st = _state(model, n, prec, seed=n + prec + 5)
    sc = (0.0, 1.2, 0.4, 0)
    g, o = paired(p, st, sc)
    if not _variant_ok(g, variant):
        pytest.skip(f"variant {variant} does not serve N={n} precision {prec}")
    g.set_state(*st, t=sc[0], a=sc[1], ad=sc[2], step=sc[3])
    assert g.hubble_length() == o.ell()          # both from a and a' by the same formula
    g.evolve(1)
    o.step(1)
    compare_states(g, o, TOL[prec], f"L form N={n} {model} fp{prec} v{variant}")
    _check_scalars(g, o, prec)


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("n", [16, 36])
def test_one_step_parity_27_point(n, prec):
    p = _params("lphi4", n, prec, stencil=27)
    st = _state("lphi4", n, prec, seed=n + 1)
    g, o = paired(p, st, (0.0, 1.1, 0.45, 0))
    g.evolve(1)
    o.step(1)
    compare_states(g, o, TOL[prec], f"L form 27-point N={n} fp{prec}")
    _check_scalars(g, o, prec)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("prec", [32, 64])
def test_ten_steps_parity(prec, variant):
    """Ten steps (32 would replay a captured graph: see the run below): every
    step's coefficients come from the pass that follows the step before."""
    n = 32
    p = _params("lphi4", n, prec)
    st = _state("lphi4", n, prec, seed=3)
    g, o = paired(p, st, (0.0, 1.1, 0.45, 0))
    if not _variant_ok(g, variant):
        pytest.skip("variant unavailable")
    g.set_state(*st, t=0.0, a=1.1, ad=0.45, step=0)
    g.evolve(10)
    o.step(10)
    compare_states(g, o, 10 * TOL[prec], f"L form 10 steps fp{prec} v{variant}")
    _check_scalars(g, o, prec, steps=10)


def test_fp64_full_run_lphi4_32():
    """The 32^3 FP64 lambda phi^4 run in the L form from seed 0 (each side its own
    initial conditions), 1000 steps (graph replay on the GPU): 1e-12 normwise."""
    p = _params("lphi4", 32, 64)
    g = Lattice(p)
    g.init_fields()
    o = Oracle(p)
    o.init_fields()
    compare_states(g, o, 1e-13, "after init")
    assert abs(g.hubble_length() / o.ell() - 1) < 1e-15
    g.evolve(1000)
    o.step(1000)
    compare_states(g, o, 1e-12, "after 1000 steps")
    assert abs(g.scalars()["a"] / o.scalars()["a"] - 1) < 1e-12
    assert abs(g.hubble_length() / o.ell() - 1) < 1e-12
    eg, eo = g.energies(), o.energies()
    for k in ("rho", "p", "H", "kin0", "pot", "curv_resid"):
        assert abs(eg[k] - eo[k]) <= 1e-10 * abs(eo[k]) + 1e-300, (k, eg[k], eo[k])


def test_fp32_run_statistics():
    """Statistics over 1000 steps of the 32^3 lambda phi^4 run (fluctuations scaled
    up by 1e4 so that FP32 resolves var phi): <f>, var f, rho, a and l every 100
    steps within 1e-3 of the FP64 oracle."""
    p = _params("lphi4", 32, 32)
    p["fluct"] = 1e4
    g = Lattice(p)
    g.init_fields()
    st = g.get_state()
    sc = g.scalars()
    o = Oracle(dict(p, precision=64))
    o.set_state(*st, t=sc["t"], a=sc["a"], ad=sc["ad"], step=sc["step"])
    for _ in range(10):
        g.evolve(100)
        o.step(100)
        eg, eo = g.energies(), o.energies()
        assert abs(eg["a"] / eo["a"] - 1) <= 1e-3
        assert abs(g.hubble_length() / o.ell() - 1) <= 1e-3
        assert abs(eg["rho"] / eo["rho"] - 1) <= 1e-3
        assert abs(eg["mean0"] - eo["mean0"]) <= 1e-3 * abs(eo["mean0"]) + 1e-3 * math.sqrt(eo["var0"])
        assert abs(eg["var0"] / eo["var0"] - 1) <= 1e-3
        assert abs(eg["var1"] / eo["var1"] - 1) <= 1e-3


@pytest.mark.parametrize("prec", [32, 64])
def test_energies_parity(prec):
    """Energies at the field time use the L form's a' there (a / Lambda) and its
    f coefficient for the momenta at the field time."""
    n = 32
    p = _params("m2phi2", n, prec)
    st = _state("m2phi2", n, prec, seed=9)
    g, o = paired(p, st, (0.5, 1.05, 0.6, 0))
    eg, eo = g.energies(), o.energies()
    tol = 1e-11 if prec == 64 else 1e-6
    for k in ("t", "a", "ad", "H", "rho", "p", "w", "kin0", "kin1", "pot"):
        assert abs(eg[k] - eo[k]) <= tol * abs(eo[k]) + 1e-300, (k, eg[k], eo[k])


def test_set_hubble_length():
    """l set by hand (here a time-reversed run's -l) is what the next step uses."""
    n = 16
    p = _params("lphi4", n, 64)
    st = _state("lphi4", n, 64, seed=4)
    g, o = paired(p, st, (0.0, 1.1, 0.45, 0))
    g.set_hubble_length(2.5)
    o.set_ell(2.5)
    assert g.hubble_length() == 2.5
    g.evolve(3)
    o.step(3)
    compare_states(g, o, 1e-12, "after setting l")
    _check_scalars(g, o, 64)
    with pytest.raises(LatticeError):
        g.set_hubble_length(0.0)
    e = Lattice(lphi4(16, precision=64))
    with pytest.raises(LatticeError) as ei:
        e.hubble_length()
    assert ei.value.status == 8


@pytest.mark.parametrize("variant", VARIANTS)
def test_checkpoint_resume_and_graph_replay_bit_identical(variant):
    """70 steps in one call (two graph replays of 32 and 6 single launches) equal
    33 steps, a checkpoint (which carries l), a new lattice and 37 more steps."""
    n = 32
    p = _params("lphi4", n, 32)
    a = Lattice(p)
    if not _variant_ok(a, variant):
        pytest.skip("variant unavailable")
    a.init_fields()
    a.evolve(70)
    b = Lattice(p); b.set_kernel(variant); b.init_fields()
    for _ in range(33):
        b.evolve(1)
    blob = b.save_checkpoint()
    c = Lattice(p); c.set_kernel(variant)
    c.load_checkpoint(blob)
    c.evolve(37)
    for x, y in zip(a.get_state(), c.get_state()):
        assert np.array_equal(x, y)
    assert a.scalars() == c.scalars()
    assert a.hubble_length() == c.hubble_length()


def test_recollapse_is_reported_not_faulted():
    """A closed universe recollapses: l = 1/h grows without bound toward H = 0,
    where the solve cannot converge; the device raises LAT_ENONFINITE (sticky)
    and the context stays usable (the oracle stops at the same point)."""
    n = 8
    p = dict(_params("lphi4", n, 64), dt=0.02)
    st = random_state(n, 3, precision=64, f_mean=(1.0, 0.0), f_amp=(0.05, 0.05), pi_mean=(0.0, 0.0),
                      pi_amp=(0.05, 0.05))
    g, o = paired(p, st, (0.0, 1.0, 0.6, 0))
    with pytest.raises(LatticeError) as ei:
        g.evolve(100)
        g.sync()
    assert ei.value.status == 5
    g2 = Lattice(_params("lphi4", 16, 32))   # the GPU context is still usable
    g2.init_fields()
    g2.evolve(2)
    g2.sync()


def test_static_and_unsupported():
    n = 16
    p = _params("lphi4", n, 32)
    g = Lattice(p)
    with pytest.raises(LatticeError) as ei:       # a' = 0: l undefined
        g.set_scalars(t=0.0, a=1.0, ad=0.0, step=0)
    assert ei.value.status == 1
    g.init_fields()
    with pytest.raises(LatticeError) as ei:        # the derivative follows eq. scale only
        g.adjoint(2)
    assert ei.value.status == 7
    with pytest.raises(LatticeError) as ei:
        Ensemble([p, p])
    assert ei.value.status == 7


def test_full_size_step_parity_256():
    """The 256^3 m^2 phi^2 lattice in the launch configuration the benchmark times
    (automatic kernel choice, then the L-form pass): one step against the
    oracle's full-lattice step."""
    n = 256
    p = _params("m2phi2", n, 32)
    st = _state("m2phi2", n, 32, seed=77)
    g = Lattice(p)
    g.set_state(*st, t=0.0, a=1.02, ad=0.5)
    o = Oracle(p)
    o.set_state(*st, t=0.0, a=1.02, ad=0.5)
    del st
    g.evolve(1)
    o.step(1)
    compare_states(g, o, TOL[32], "L form full size 256")
    _check_scalars(g, o, 32)
