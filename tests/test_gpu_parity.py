"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on
identical seeded inputs, element by element.

Tolerances (normwise per field and quantity, max|gpu - oracle| / max|oracle|):
FP32 path 2e-6 per step, FP64 path 1e-12 (also over the 1000 steps of the
32^3 lambda phi^4 run); run statistics 1e-3.
"""
import math

import numpy as np
import pytest

from gpu_helpers import compare_states, normwise, paired
from oracle.oracle import Oracle
from paper_0911_5692_gb300 import Lattice, LatticeError
from paper_0911_5692_gb300.workloads import lphi4, m2phi2, random_state

pytestmark = pytest.mark.gpu

TOL = {32: 2e-6, 64: 1e-12}
VARIANTS = [2, 4, 5]


def _params(model, n, prec, expansion):
    if model == "lphi4":
        return lphi4(n, precision=prec, expansion=expansion)
    return m2phi2(n, precision=prec, expansion=expansion)


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


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("model,expansion", [("lphi4", 1), ("m2phi2", 1), ("lphi4", 0)])
@pytest.mark.parametrize("n", [4, 16, 36, 64])
def test_one_step_parity(n, model, expansion, prec, variant):
    """One fused step from an identical stored state (several tiles, ragged N=36,
    degenerate N=4): f, f', a, a' and the sums of the new fields."""
    p = _params(model, n, prec, expansion)
    st = _state(model, n, prec, seed=n + prec)
    sc = (0.0, 1.2, 0.4, 0) if expansion else (0.0, 1.0, 0.0, 0)
    g, o = paired(p, st, sc)
    if not _variant_ok(g, variant):
        pytest.skip(f"variant {variant} does not serve N={n} precision {prec}")
    g.set_state(*st, t=sc[0], a=sc[1], ad=sc[2], step=sc[3])
    g.evolve(1)
    o.step(1)
    compare_states(g, o, TOL[prec], f"N={n} {model} exp={expansion} fp{prec} v{variant}")
    gs, os_ = g.scalars(), o.scalars()
    assert gs["step"] == os_["step"] == 1
    # a and a' are FP64 on both sides; an FP32 lattice forms the sums that set a''
    # in FP32 (compensated per thread, relative error ~1e-7), which moves a' by
    # about dt dc and a by about dt^2 dc (dt <= 0.125 here)
    ta, tad = (1e-14, 1e-13) if prec == 64 else (1e-8, 1e-7)
    assert abs(gs["a"] - os_["a"]) <= ta * os_["a"]
    assert abs(gs["ad"] - os_["ad"]) <= tad * max(abs(os_["ad"]), 1.0)
    # sums of the new fields. FP64: the oracle's, to rounding. FP32: the GPU sums
    # the fields it writes, so they are compared with the oracle's FP64 sums of
    # those same FP32 fields; what is left is the FP32 arithmetic of the sums
    # (differences exact by Sterbenz, squares rounded to 6e-8, per-thread FP32
    # accumulation over at most 2 x 64 terms before the FP64 block sums:
    # a few 1e-7 in practice, 2e-6 at most for these lattices)
    if prec == 64:
        ref_s = os_["S"]
        stol = [1e-11, 1e-11, 1e-13, 1e-11]
    else:
        own = Oracle(p)
        own.set_state(*g.get_state(), t=gs["t"], a=gs["a"], ad=gs["ad"], step=gs["step"])
        ref_s = own.scalars()["S"]
        stol = [2e-6, 2e-6, 1e-6, 2e-6]
    for k in range(4):
        ref = ref_s[k]
        assert abs(gs["S"][k] - ref) <= stol[k] * abs(ref) + 1e-300, (k, gs["S"][k], ref)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("prec", [32, 64])
def test_ten_steps_parity(prec, variant):
    """Ten steps: the coefficients come from the device-side a(t) update in the
    kernels' last block (no host round trip)."""
    n = 32
    p = lphi4(n, precision=prec)
    st = _state("lphi4", n, prec, seed=3)
    g, o = paired(p, st, (0.0, 1.1, 0.45, 0))
    if not _variant_ok(g, variant):
        pytest.skip("variant unavailable")
    g.set_state(*st, t=0.0, a=1.1, ad=0.45, step=0)
    g.evolve(10)
    o.step(10)
    compare_states(g, o, 10 * TOL[prec], f"10 steps fp{prec} v{variant}")
    assert abs(g.scalars()["a"] / o.scalars()["a"] - 1) <= (1e-13 if prec == 64 else 1e-7)


def test_fp64_full_run_lphi4_32():
    """The 32^3 FP64 lambda phi^4 run: both sides initialise from seed 0 with their
    own Philox / FFT pipelines and evolve 1000 steps; fields, momenta and a agree
    to 1e-12 normwise."""
    p = lphi4(32, precision=64)
    g = Lattice(p)
    g.init_fields()
    o = Oracle(p)
    o.init_fields()
    compare_states(g, o, 1e-13, "after init")
    g.evolve(1000)
    o.step(1000)
    compare_states(g, o, 1e-12, "after 1000 steps")
    assert abs(g.scalars()["a"] / o.scalars()["a"] - 1) < 1e-12
    eg, eo = g.energies(), o.energies()
    for k in ("rho", "p", "H", "kin0", "pot", "mean0"):
        assert abs(eg[k] - eo[k]) <= 1e-10 * abs(eo[k]) + 1e-300, (k, eg[k], eo[k])
    # a variance moves by at most 2 sigma |delta f| when the fields move by delta f
    for i in (0, 1):
        k = f"var{i}"
        bound = 2 * math.sqrt(eo[k]) * 1e-12 * np.max(np.abs(o.get_state()[i]))
        assert abs(eg[k] - eo[k]) <= bound, (k, eg[k], eo[k], bound)


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("model", ["lphi4", "m2phi2"])
def test_init_parity(model, prec):
    """DEFROST-style initial state (Philox white noise, Fourier filtering, program
    units, half-step drift): GPU against oracle, same seed."""
    p = _params(model, 32, prec, 1)
    p["seed"] = 12345
    g = Lattice(p)
    g.init_fields()
    o = Oracle(p)
    o.init_fields()
    tol = 1e-13 if prec == 64 else 1e-6
    errs = compare_states(g, o, tol, f"init {model} fp{prec}")
    assert abs(g.scalars()["a"] - o.scalars()["a"]) < 1e-15
    # fluctuation fields themselves (subtract the homogeneous part), FP64 only
    if prec == 64:
        gs, os_ = g.get_state(), o.get_state()
        d_g, d_o = gs[1], os_[1]
        assert normwise(d_g, d_o) < 1e-12


@pytest.mark.parametrize("prec", [32, 64])
def test_energies_parity(prec):
    """Energy density, pressure, w, H, residual curvature, means and variances
    (eq. rho-pres with momenta at the field time)."""
    n = 32
    p = m2phi2(n, precision=prec)
    st = _state("m2phi2", n, prec, seed=9)
    g, o = paired(p, st, (0.5, 1.05, 0.6, 0))
    eg, eo = g.energies(), o.energies()
    tol = 1e-11 if prec == 64 else 1e-6
    for k in ("t", "a", "ad", "H", "rho", "p", "w", "kin0", "kin1", "pot", "mean0", "mean1"):
        assert abs(eg[k] - eo[k]) <= tol * abs(eo[k]) + 1e-300, (k, eg[k], eo[k])
    for k in ("grad0", "grad1", "var0", "var1", "curv_resid"):
        assert abs(eg[k] - eo[k]) <= (1e-10 if prec == 64 else 1e-3) * abs(eo[k]) + 1e-300, (k, eg[k], eo[k])


def test_spectrum_parity():
    n = 32
    p = lphi4(n, precision=64)
    g = Lattice(p)
    g.init_fields()
    o = Oracle(p)
    o.init_fields()
    for field in (0, 1):
        kg, pg, cg = g.spectrum(field, 30)
        ko, po, co = o.spectrum(field, 30)
        assert (cg == co).all()
        np.testing.assert_allclose(kg, ko, rtol=1e-12)
        scale = po[1:].max()
        np.testing.assert_allclose(pg[1:], po[1:], rtol=1e-9, atol=1e-9 * scale)


def test_dispersion_exact_on_gpu():
    """The GPU path itself against the closed-form leapfrog solution of a free
    massive lattice mode (static space, FP64): f_{n+1/2} = cos(k.x) cos(w_d (n+1/2) dt)."""
    n, dt = 16, 0.1
    p = dict(n=n, precision=64, model=1, expansion=0, L=n * 0.5, dt=dt, lam=0.0, m=1e-6, g2=0.0,
             phi0=(1.0, 0.0), dphi0=(0.0, 0.0), eight_pi_G=1.0, fluct=0.0, seed=0)
    dx = p["L"] / n
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    kv = (1, 3, 2)
    mode = np.cos(2 * np.pi * (kv[0] * x + kv[1] * y + kv[2] * z) / n)
    w2 = 1.0 + sum((2 / dx * math.sin(math.pi * k / n)) ** 2 for k in kv)
    wd = math.acos(1 - w2 * dt * dt / 2) / dt
    for variant in VARIANTS:
        g = Lattice(p)
        if not _variant_ok(g, variant):
            continue
        zero = np.zeros((n, n, n))
        g.set_state(1e-3 * mode * math.cos(wd * dt / 2), zero, zero, zero)
        g.evolve(100)
        f0 = g.get_state()[0]
        np.testing.assert_allclose(f0, 1e-3 * mode * math.cos(wd * 100.5 * dt), rtol=0, atol=1e-15)


@pytest.mark.parametrize("variant", VARIANTS)
def test_graph_replay_bit_identical_to_single_launches(variant):
    """lat_evolve(64) replays a captured graph of 32-step chunks; 64 single-step
    calls launch directly. Same kernels, same order: bit-identical; and two runs
    are bit-identical (fixed-order reductions)."""
    n = 32
    p = lphi4(n, precision=32)
    st = _state("lphi4", n, 32, seed=4)
    outs = []
    for mode in ("graph", "single", "graph"):
        g = Lattice(p)
        if not _variant_ok(g, variant):
            pytest.skip("variant unavailable")
        g.set_state(*st, t=0.0, a=1.1, ad=0.45)
        if mode == "graph":
            g.evolve(64)
        else:
            for _ in range(64):
                g.evolve(1)
        outs.append((g.get_state(), g.scalars()))
    for k in (1, 2):
        for a, b in zip(outs[0][0], outs[k][0]):
            assert np.array_equal(a, b)
        assert outs[0][1] == outs[k][1]


@pytest.mark.parametrize("variant", VARIANTS)
def test_checkpoint_resume_bit_identical(variant):
    """n steps == k steps, checkpoint (parameters, FP64 scalar block, arrays),
    load into a new lattice, n - k steps: bit-identical."""
    n = 32
    p = lphi4(n, precision=32)
    a = Lattice(p)
    if not _variant_ok(a, variant):
        pytest.skip("variant unavailable")
    a.init_fields(); a.evolve(70)
    b = Lattice(p); b.set_kernel(variant); b.init_fields(); b.evolve(33)
    blob = b.save_checkpoint()
    c = Lattice(p); c.set_kernel(variant)
    c.load_checkpoint(blob)
    c.evolve(37)
    for x, y in zip(a.get_state(), c.get_state()):
        assert np.array_equal(x, y)
    sa, sc_ = a.scalars(), c.scalars()
    assert sa == sc_ and sa["step"] == 70
    # a blob from other parameters is refused
    d = Lattice(dict(p, seed=1))
    with pytest.raises(LatticeError):
        d.load_checkpoint(blob)


def test_resume_from_state_and_scalars():
    """Resuming from the arrays and (t, a, a', step) alone recomputes the sums in
    FP64, so it continues within rounding of the uninterrupted run."""
    n = 32
    p = lphi4(n, precision=32)
    a = Lattice(p); a.init_fields(); a.evolve(70)
    b = Lattice(p); b.init_fields(); b.evolve(33)
    sc = b.scalars()
    c = Lattice(p)
    c.set_state(*b.get_state(), t=sc["t"], a=sc["a"], ad=sc["ad"], step=sc["step"])
    c.evolve(37)
    for x, y in zip(a.get_state(), c.get_state()):
        assert normwise(y, x) < 1e-5
    assert abs(a.scalars()["a"] / c.scalars()["a"] - 1) < 1e-7


def test_nonfinite_is_sticky_and_stops_the_steps():
    """A NaN planted in the host-side input makes the sums non-finite; the device
    raises LAT_ENONFINITE, later steps are no-ops, and the next synchronising call
    returns the error."""
    n = 16
    p = lphi4(n, precision=32)
    st = list(_state("lphi4", n, 32, seed=1))
    st[1] = st[1].copy()
    st[1][3, 4, 5] = np.nan
    g = Lattice(p)
    g.set_state(*st, t=0.0, a=1.0, ad=0.4)
    with pytest.raises(LatticeError) as ei:
        g.evolve(5)
        g.sync()
    assert ei.value.status == 5


def test_evolve_zero_steps_is_noop():
    n = 16
    p = lphi4(n, precision=64)
    st = _state("lphi4", n, 64, seed=2)
    g, _ = paired(p, st, (0.0, 1.0, 0.4, 0))
    before = g.get_state()
    g.evolve(0)
    for x, y in zip(before, g.get_state()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("n,model", [(256, "m2phi2"), (512, "lphi4")])
def test_full_size_step_parity(n, model):
    """Full-size lattices in the launch configuration the benchmark times (the
    automatic kernel choice): one step against the oracle's full-lattice step."""
    p = _params(model, n, 32, 1)
    st = _state(model, n, 32, seed=77)
    g = Lattice(p)
    g.set_state(*st, t=0.0, a=1.02, ad=0.5)
    o = Oracle(p)
    o.set_state(*st, t=0.0, a=1.02, ad=0.5)
    del st
    g.evolve(1)
    o.step(1)
    compare_states(g, o, TOL[32], f"full size {n}")


@pytest.mark.parametrize("depth", [1, 2, 3, 4])
@pytest.mark.parametrize("ty,zr", [(1, 5), (2, 7), (4, 16)])
@pytest.mark.parametrize("prec", [32, 64])
def test_march_geometries(prec, ty, zr, depth):
    """The plane-ring z-march at every prefetch depth and with ragged z-chunks:
    ten steps against the oracle."""
    n = 36 if ty != 4 else 32
    p = lphi4(n, precision=prec)
    st = _state("lphi4", n, prec, seed=ty * 10 + depth)
    g, o = paired(p, st, (0.0, 1.1, 0.45, 0))
    try:
        g.set_kernel(2, ty, zr, depth)
    except LatticeError:
        pytest.skip("geometry does not fit")
    assert g.kernel_info()["depth"] == depth
    g.set_state(*st, t=0.0, a=1.1, ad=0.45, step=0)
    g.evolve(10)
    o.step(10)
    compare_states(g, o, 10 * TOL[prec], f"march ty={ty} zr={zr} depth={depth} fp{prec}")


@pytest.mark.parametrize("prec,n,ty,depth,zr", [(32, 128, 4, 1, 23), (32, 128, 8, 1, 23), (32, 256, 4, 1, 23),
                                                (32, 256, 8, 1, 23), (32, 512, 2, 1, 23), (32, 512, 4, 1, 23),
                                                (32, 128, 8, 2, 23), (32, 256, 4, 2, 23), (32, 256, 8, 2, 23),
                                                (32, 512, 2, 2, 23), (32, 128, 8, 2, 1), (32, 128, 8, 2, 2),
                                                (32, 128, 8, 1, 1), (64, 256, 4, 1, 23), (64, 512, 1, 1, 23)])
def test_specialised_instances(prec, n, ty, depth, zr):
    """The compile-time-geometry instances of the z-march (one per (N, ty, depth)
    the automatic choice can pick), against the oracle; z chunks that do not
    divide N exercise the unrolled plane loop's early exits, chunks of one or two
    planes the prologue of the deeper ring."""
    p = lphi4(n, precision=prec)
    st = _state("lphi4", n, prec, seed=n + ty)
    g, o = paired(p, st, (0.0, 1.05, 0.5, 0))
    g.set_kernel(2, ty, zr, depth)
    info = g.kernel_info()
    assert (info["ty"], info["depth"]) == (ty, depth)
    steps = 2 if n >= 512 else 3
    g.set_state(*st, t=0.0, a=1.05, ad=0.5, step=0)
    g.evolve(steps)
    o.step(steps)
    compare_states(g, o, steps * TOL[prec], f"fast N={n} ty={ty} depth={depth} zr={zr} fp{prec}")
    gs, os_ = g.scalars(), o.scalars()
    assert abs(gs["a"] / os_["a"] - 1) <= (1e-13 if prec == 64 else 1e-7)


@pytest.mark.parametrize("fluct", [1.0, 1e4])
def test_fp32_run_statistics(fluct):
    """Statistics over a run (<f>, var f, total energy, a(t)) of the 32^3 lambda phi^4
    configuration on the FP32 path against the FP64 oracle from the same start, every
    100 of 1000 steps, within 1e-3 (parametric resonance does not saturate this early).
    At the vacuum amplitude (fluct = 1) the inflaton's fluctuations (1.6e-7 about 1)
    are below FP32 resolution, so var phi is compared only with fluctuations scaled
    up by 1e4, where FP32 resolves them."""
    p = lphi4(32, precision=32, fluct=fluct)
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
        assert abs(eg["rho"] / eo["rho"] - 1) <= 1e-3
        assert abs(eg["mean0"] - eo["mean0"]) <= 1e-3 * abs(eo["mean0"]) + 1e-3 * math.sqrt(eo["var0"])
        assert abs(eg["mean1"] - eo["mean1"]) <= 1e-3 * math.sqrt(eo["var1"])
        assert abs(eg["var1"] / eo["var1"] - 1) <= 1e-3
        if fluct > 1.0:
            assert abs(eg["var0"] / eo["var0"] - 1) <= 1e-3


@pytest.mark.parametrize("src", ["host", "device"])
def test_upload_state_is_set_state(src):
    """lat_upload_state (all four arrays queued on the stream at once, from pinned
    host or device memory) leaves the lattice exactly as four lat_set_state calls
    do: same arrays, same scalars, and bit-identical steps after it."""
    import torch
    n = 32
    p = lphi4(n, precision=32)
    st = _state("lphi4", n, 32, seed=41)
    a = Lattice(p)
    a.set_state(*st, t=0.0, a=1.1, ad=0.4)
    b = Lattice(p)
    b.set_scalars(0.0, 1.1, 0.4, 0)
    ts = [torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32).reshape(-1)) for x in st]
    ts = [t.pin_memory() for t in ts] if src == "host" else [t.cuda() for t in ts]
    b.upload_state(*ts)
    b.sync()
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    assert a.scalars() == b.scalars()
    a.evolve(3)
    b.evolve(3)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    assert a.scalars() == b.scalars()


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("n,ty", [(4, 0), (16, 0), (36, 4), (64, 8), (64, 16), (128, 32), (136, 8), (264, 8),
                                  (200, 8)])
def test_xtile_kernel_geometries(n, ty, prec):
    """Variant 4 (x tiles of at most 32 or 16 vectors, taller y tiles) over tile
    heights and sides whose rows split into ragged x tiles, against the oracle:
    five FP64 steps (an indexing mistake shows far above 1e-12), one FP32 step
    (the per-step FP32 bound; FP32 rounding of the degenerate N = 4 lattice,
    dt = 0.125, grows past five times it over five steps)."""
    p = lphi4(n, precision=prec)
    st = _state("lphi4", n, prec, seed=n + ty)
    g, o = paired(p, st, (0.0, 1.1, 0.45, 0))
    try:
        g.set_kernel(4, ty, 0, 0)
    except LatticeError:
        pytest.skip("geometry does not fit")
    info = g.kernel_info()
    assert info["variant"] == 4 and (ty == 0 or info["ty"] == ty)
    g.set_state(*st, t=0.0, a=1.1, ad=0.45, step=0)
    steps = 5 if prec == 64 else 1
    g.evolve(steps)
    o.step(steps)
    compare_states(g, o, steps * TOL[prec], f"x tiles N={n} ty={ty} fp{prec}")


@pytest.mark.parametrize("variant", [4, 5])
def test_xtile_kernel_full_size_512(variant):
    """The x-tiled kernels (variant 4; variant 5, one warp wide with an edge warp)
    on the 512^3 lambda phi^4 lattice (FP32): one step against the oracle's
    full-lattice step."""
    n = 512
    p = _params("lphi4", n, 32, 1)
    st = _state("lphi4", n, 32, seed=79)
    g = Lattice(p)
    g.set_kernel(variant)
    g.set_state(*st, t=0.0, a=1.02, ad=0.5)
    o = Oracle(p)
    o.set_state(*st, t=0.0, a=1.02, ad=0.5)
    del st
    g.evolve(1)
    o.step(1)
    compare_states(g, o, TOL[32], f"x tiles full size 512 v{variant}")


def test_fp64_full_size_default_kernel():
    """FP64 rows of 128 vectors take the x-tiled kernel by default: one 256^3
    FP64 step against the oracle at the FP64 bound."""
    n = 256
    p = _params("m2phi2", n, 64, 1)
    st = _state("m2phi2", n, 64, seed=80)
    g = Lattice(p)
    assert g.kernel_info()["variant"] == 4
    g.set_state(*st, t=0.0, a=1.02, ad=0.5)
    o = Oracle(p)
    o.set_state(*st, t=0.0, a=1.02, ad=0.5)
    del st
    g.evolve(1)
    o.step(1)
    compare_states(g, o, TOL[64], "FP64 full size 256, default kernel")


def test_fp64_full_size_512_two_steps():
    """The FP64 variant that the 512^3 FP32 run's error is measured against (the
    bench's fp32_vs_fp64_512, every 16th site per axis): two 512^3 FP64 steps of
    the lambda phi^4 model against the oracle's full-lattice steps at the FP64
    bound."""
    n = 512
    p = _params("lphi4", n, 64, 1)
    st = _state("lphi4", n, 64, seed=81)
    g = Lattice(p)
    g.set_state(*st, t=0.0, a=1.05, ad=0.45)
    o = Oracle(p)
    o.set_state(*st, t=0.0, a=1.05, ad=0.45)
    del st
    g.evolve(2)
    o.step(2)
    compare_states(g, o, 2 * TOL[64], "FP64 full size 512, two steps")
    assert abs(g.scalars()["a"] / o.scalars()["a"] - 1) < 1e-13



@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("n,depth", [(256, 1), (256, 2), (512, 1), (512, 2)])
def test_warp_tile_kernel(n, depth, prec):
    """Variant 5 (x tiles one warp wide, compiled N, ty and depth, an edge warp
    for the tile's x neighbours and its boundary column) on its compiled sides:
    three steps against the oracle, and the sums of the new fields (whose x
    differences at the tile edges come from the edge warp) against the oracle's
    sums of the same fields."""
    p = _params("lphi4", n, prec, 1)
    st = _state("lphi4", n, prec, seed=n + depth)
    g = Lattice(p)
    try:
        g.set_kernel(5, 16, 0, depth)
    except LatticeError:
        pytest.skip(f"no compiled instance for N={n} depth={depth} fp{prec}")
    assert g.kernel_info()["variant"] == 5
    g.set_state(*st, t=0.0, a=1.05, ad=0.5)
    o = Oracle(p)
    o.set_state(*st, t=0.0, a=1.05, ad=0.5)
    del st
    g.evolve(3)
    o.step(3)
    compare_states(g, o, 3 * TOL[prec], f"warp tiles N={n} depth={depth} fp{prec}")
    gs = g.scalars()
    own = Oracle(p)
    own.set_state(*g.get_state(), t=gs["t"], a=gs["a"], ad=gs["ad"], step=gs["step"])
    tol = [1e-11, 1e-11, 1e-13, 1e-11] if prec == 64 else [2e-6, 2e-6, 1e-6, 2e-6]
    for k in range(4):
        ref = own.scalars()["S"][k]
        assert abs(gs["S"][k] - ref) <= tol[k] * abs(ref), (k, gs["S"][k], ref)
