"""GPU parity of the 27-point Laplacian path (Sec. II.C: the Patra-Karttunen
stencil) against the FP64 CPU oracle, through the C ABI.

Fields and momenta: normwise (max|gpu - oracle| / max|oracle| per quantity)
2e-6 per FP32 step and 1e-12 per FP64 step, as for the 7-point path.

Gradient averages: the oracle evaluates -<f L f> literally, which cancels the
mean of f against the zero-sum stencil: its relative rounding error grows as
eps |f|^2 / <(delta f)^2>, about 4e-11 for the fluctuations of 1e-3 used here
(measured against an exactly summed bond form). The CUDA path sums the
equivalent weighted squared differences over each site's 13 neighbour pairs,
which does not cancel, so the FP64 tolerance on those two sums is 1e-9.
"""
import math

import numpy as np
import pytest

from gpu_helpers import compare_states, normwise, paired
from oracle.oracle import Oracle, laplacian27
from paper_0911_5692_gb300 import Ensemble, Lattice, LatticeError
from paper_0911_5692_gb300.workloads import lphi4, m2phi2, random_state

pytestmark = pytest.mark.gpu

TOL = {32: 2e-6, 64: 1e-12}
STOL = {64: [1e-9, 1e-9, 1e-13, 1e-11], 32: [3e-3, 3e-3, 1e-6, 1e-5]}


def _params(model, n, prec, expansion=1):
    p = (lphi4 if model == "lphi4" else m2phi2)(n, precision=prec, expansion=expansion)
    p["stencil"] = 27
    return p


def _state(model, n, prec, seed):
    if model == "lphi4":
        return random_state(n, seed, precision=prec, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-3),
                            pi_mean=(0.5, 0.0), pi_amp=(1e-3, 1e-3))
    return random_state(n, seed, precision=prec, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-4),
                        pi_mean=(0.3, 0.0), pi_amp=(1e-3, 1e-2))


def _check_scalars(g, o, prec, steps):
    """a and a' are FP64 on both sides, but on the FP32 path they are driven by
    sums of FP32 fields (relative errors up to STOL[32]), which moves a'' by
    about 1e-6 relative and a by about dt^2 steps^2 of that: 1e-10 per step
    bounds it; FP64 keeps rounding level."""
    gs, os_ = g.scalars(), o.scalars()
    assert gs["step"] == os_["step"] == steps
    ta, tad = (1e-14, 1e-13) if prec == 64 else (1e-10, 1e-9)
    assert abs(gs["a"] - os_["a"]) <= ta * steps * os_["a"]
    assert abs(gs["ad"] - os_["ad"]) <= tad * steps * max(abs(os_["ad"]), 1.0)
    for k in range(4):
        ref = os_["S"][k]
        tol = STOL[prec][k] * (1 if prec == 64 else steps)
        assert abs(gs["S"][k] - ref) <= tol * abs(ref) + 1e-300, (k, gs["S"][k], ref)


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("model,expansion", [("lphi4", 1), ("m2phi2", 1), ("lphi4", 0)])
@pytest.mark.parametrize("n", [4, 8, 20, 36, 64])
def test_one_step_parity_27(n, model, expansion, prec):
    """One fused step from an identical stored state: several tiles, ragged
    N = 20 and 36, the degenerate N = 4 (every neighbour wraps)."""
    p = _params(model, n, prec, expansion)
    st = _state(model, n, prec, seed=3 * n + prec)
    sc = (0.0, 1.2, 0.4, 0) if expansion else (0.0, 1.0, 0.0, 0)
    g, o = paired(p, st, sc)
    assert g.kernel_info()["variant"] == 2
    g.evolve(1)
    o.step(1)
    compare_states(g, o, TOL[prec], f"27-point N={n} {model} exp={expansion} fp{prec}")
    _check_scalars(g, o, prec, 1)


def test_sums_after_upload_27():
    """The sums of an uploaded state (the no-step pass that follows set_state)."""
    n = 24
    p = _params("lphi4", n, 64)
    st = _state("lphi4", n, 64, seed=5)
    g, o = paired(p, st, (0.0, 1.1, 0.3, 0))
    gs, os_ = g.scalars(), o.scalars()
    for k in range(4):
        assert abs(gs["S"][k] - os_["S"][k]) <= STOL[64][k] * abs(os_["S"][k]), k


@pytest.mark.parametrize("depth", [1, 2, 3])
@pytest.mark.parametrize("ty,zr", [(1, 5), (2, 7), (4, 16), (8, 0), (3, 11)])
@pytest.mark.parametrize("prec", [32, 64])
def test_geometries_27(prec, ty, zr, depth):
    """Every tile height, prefetch depth and ragged z-chunking (zr = 0: one
    resident wave with uneven runs): ten steps against the oracle."""
    n = 36 if ty in (1, 2) else 24 if ty == 3 else 32
    p = _params("lphi4", n, prec)
    st = _state("lphi4", n, prec, seed=ty * 10 + depth)
    g, o = paired(p, st, (0.0, 1.1, 0.45, 0))
    try:
        g.set_kernel(2, ty, zr, depth)
    except LatticeError:
        pytest.skip("geometry does not fit")
    info = g.kernel_info()
    assert (info["variant"], info["ty"], info["depth"]) == (2, ty, depth)
    g.set_state(*st, t=0.0, a=1.1, ad=0.45, step=0)
    g.evolve(10)
    o.step(10)
    compare_states(g, o, 10 * TOL[prec], f"27-point ty={ty} zr={zr} depth={depth} fp{prec}")
    _check_scalars(g, o, prec, 10)


@pytest.mark.parametrize("prec,n", [(64, 136), (64, 200), (32, 260), (32, 264)])
def test_x_tiles_27(prec, n):
    """Rows are split into x tiles of at most 16 vectors with a halo vector on
    either side; these sides give odd tile counts and widths (FP64: 17 tiles
    of 8 columns, 10 of 20; FP32: 5 tiles of 52 columns, 6 of 44): three steps
    against the oracle."""
    p = _params("lphi4", n, prec)
    st = _state("lphi4", n, prec, seed=n)
    g, o = paired(p, st, (0.0, 1.1, 0.45, 0))
    g.evolve(3)
    o.step(3)
    compare_states(g, o, 3 * TOL[prec], f"27-point x tiles N={n} fp{prec}")
    _check_scalars(g, o, prec, 3)


def test_fp64_run_from_init_27():
    """Both sides initialise from seed 7 with their own Philox / FFT pipelines and
    the 27-point dispersion, then evolve 300 steps (FP64)."""
    p = _params("lphi4", 32, 64)
    p["seed"] = 7
    g = Lattice(p)
    g.init_fields()
    o = Oracle(p)
    o.init_fields()
    compare_states(g, o, 1e-13, "after init")
    g.evolve(300)
    o.step(300)
    compare_states(g, o, 1e-12, "after 300 steps")
    assert abs(g.scalars()["a"] / o.scalars()["a"] - 1) < 1e-12


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("model", ["lphi4", "m2phi2"])
def test_init_parity_27(model, prec):
    """Initial fluctuations filtered with the 27-point k_lat^2 (the GPU evaluates
    the stencil's symbol in sin^2 form, the oracle in cosines)."""
    p = _params(model, 32, prec)
    p["seed"] = 4242
    g = Lattice(p)
    g.init_fields()
    o = Oracle(p)
    o.init_fields()
    compare_states(g, o, 1e-13 if prec == 64 else 1e-6, f"init 27 {model} fp{prec}")
    if prec == 64:
        assert normwise(g.get_state()[1], o.get_state()[1]) < 1e-12


@pytest.mark.parametrize("prec", [32, 64])
def test_energies_parity_27(prec):
    n = 32
    p = _params("m2phi2", n, prec)
    st = _state("m2phi2", n, prec, seed=9)
    g, o = paired(p, st, (0.5, 1.05, 0.6, 0))
    eg, eo = g.energies(), o.energies()
    tol = 1e-11 if prec == 64 else 1e-6
    for k in ("t", "a", "ad", "H", "rho", "p", "w", "kin0", "kin1", "pot", "mean0", "mean1"):
        assert abs(eg[k] - eo[k]) <= tol * abs(eo[k]) + 1e-300, (k, eg[k], eo[k])
    for k in ("grad0", "grad1", "var0", "var1", "curv_resid"):
        assert abs(eg[k] - eo[k]) <= (1e-9 if prec == 64 else 1e-3) * abs(eo[k]) + 1e-300, (k, eg[k], eo[k])


def test_dispersion_exact_on_gpu_27():
    """The GPU path against the closed-form leapfrog solution of a free massive
    mode with the 27-point stencil (static space, FP64): the mode's eigenvalue is
    taken from the oracle's stencil applied to it."""
    n, dt = 16, 0.1
    p = dict(n=n, precision=64, model=1, expansion=0, L=n * 0.5, dt=dt, lam=0.0, m=1e-6, g2=0.0,
             phi0=(1.0, 0.0), dphi0=(0.0, 0.0), eight_pi_G=1.0, fluct=0.0, seed=0, stencil=27)
    dx = p["L"] / n
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    kv = (1, 3, 2)
    mode = np.cos(2 * np.pi * (kv[0] * x + kv[1] * y + kv[2] * z) / n)
    lm = laplacian27(mode, dx)
    lam = lm[0, 0, 0] / mode[0, 0, 0]
    assert np.max(np.abs(lm - lam * mode)) < 1e-10 * np.max(np.abs(lm))
    w2 = 1.0 - lam
    wd = math.acos(1 - w2 * dt * dt / 2) / dt
    g = Lattice(p)
    zero = np.zeros((n, n, n))
    g.set_state(1e-3 * mode * math.cos(wd * dt / 2), zero, zero, zero)
    g.evolve(100)
    np.testing.assert_allclose(g.get_state()[0], 1e-3 * mode * math.cos(wd * 100.5 * dt), rtol=0, atol=1e-15)


def test_graph_replay_bit_identical_27():
    n = 32
    p = _params("lphi4", n, 32)
    st = _state("lphi4", n, 32, seed=4)
    a = Lattice(p)
    a.set_state(*st, t=0.0, a=1.0, ad=0.3)
    a.evolve(64)
    b = Lattice(p)
    b.set_state(*st, t=0.0, a=1.0, ad=0.3)
    for _ in range(64):
        b.evolve(1)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    assert a.scalars() == b.scalars()


@pytest.mark.parametrize("n,model", [(256, "m2phi2"), (512, "lphi4")])
def test_full_size_step_parity_27(n, model):
    """Full-size lattices in the automatic launch configuration: one step against
    the oracle's full-lattice step."""
    p = _params(model, n, 32)
    st = _state(model, n, 32, seed=78)
    g = Lattice(p)
    g.set_state(*st, t=0.0, a=1.02, ad=0.5)
    o = Oracle(p)
    o.set_state(*st, t=0.0, a=1.02, ad=0.5)
    del st
    g.evolve(1)
    o.step(1)
    compare_states(g, o, TOL[32], f"27-point full size {n}")


def test_paths_without_27_point_form_refuse():
    """Kernels and paths written for the 7-point stencil refuse a 27-point
    lattice instead of computing the wrong operator."""
    n = 16
    p = _params("lphi4", n, 64)
    g = Lattice(p)
    with pytest.raises(LatticeError, match="UNSUPPORTED"):
        g.set_kernel(4)       # the x-tiled ring is written for 7 points
    with pytest.raises(LatticeError, match="UNSUPPORTED"):
        g.set_kernel(5)       # warp-wide tiles: compiled sides only (256, 512)
    for variant in (1, 3):    # no such kernels
        with pytest.raises(LatticeError, match="EINVAL"):
            g.set_kernel(variant)
    g.set_kernel(2)
    assert g.kernel_info()["variant"] == 2
    import torch
    fb = torch.zeros(2 * n ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(LatticeError, match="UNSUPPORTED"):
        g.vjp(1, fb, fb.clone())
    with pytest.raises(LatticeError, match="UNSUPPORTED"):
        Ensemble([p, p])
    from paper_0911_5692_gb300.slab import SlabGPU
    with pytest.raises(LatticeError, match="UNSUPPORTED"):
        SlabGPU(p, 0, n)


def test_checkpoint_resume_bit_identical_27():
    """n steps == k steps, checkpoint, load into a new lattice, n - k steps:
    bit-identical with the 27-point kernel (the stencil is part of the
    parameters the blob must match)."""
    n = 32
    p = _params("lphi4", n, 32)
    a = Lattice(p)
    a.init_fields()
    a.evolve(70)
    b = Lattice(p)
    b.init_fields()
    b.evolve(33)
    blob = b.save_checkpoint()
    c = Lattice(p)
    c.load_checkpoint(blob)
    c.evolve(37)
    for x, y in zip(a.get_state(), c.get_state()):
        assert np.array_equal(x, y)
    assert a.scalars() == c.scalars()
    d = Lattice(dict(p, stencil=7))
    with pytest.raises(LatticeError):
        d.load_checkpoint(blob)


def test_nonfinite_is_sticky_27():
    """A NaN in the uploaded fields makes the 27-point sums non-finite; the device
    raises LAT_ENONFINITE and the next synchronising call returns it."""
    n = 16
    p = _params("lphi4", n, 32)
    st = list(_state("lphi4", n, 32, seed=1))
    st[0] = st[0].copy()
    st[0][2, 3, 4] = np.nan
    g = Lattice(p)
    g.set_state(*st, t=0.0, a=1.0, ad=0.4)
    with pytest.raises(LatticeError) as ei:
        g.evolve(3)
        g.sync()
    assert ei.value.status == 5


def _own_sums_check(g, p, prec):
    """The lattice's sums of its new fields against the oracle's sums of the
    same fields (FP64 on the oracle side): per-thread FP32 accumulation of the
    bond sums bounds the FP32 error at about 2e-6."""
    gs = g.scalars()
    own = Oracle(p)
    own.set_state(*g.get_state(), t=gs["t"], a=gs["a"], ad=gs["ad"], step=gs["step"])
    tol = [1e-9, 1e-9, 1e-13, 1e-11] if prec == 64 else [2e-6, 2e-6, 1e-6, 2e-6]
    ref = own.scalars()["S"]
    own.close()
    for k in range(4):
        assert abs(gs["S"][k] - ref[k]) <= tol[k] * abs(ref[k]), (k, gs["S"][k], ref[k])


@pytest.mark.parametrize("zr", [0, 1, 7])
@pytest.mark.parametrize("prec", [32, 64])
def test_warp_tiles_27(prec, zr):
    """Variant 5 of the 27-point stencil: x tiles one warp wide with N = 256 and
    ty = 16 compiled in, the Laplacian from per-plane aggregates carried along
    z, an edge warp that computes each tile's boundary column, and the bond sums
    counted at the left end of each bond. Two steps against the oracle with z
    runs of every length (zr = 1: runs of one plane, each with its own prologue
    and final bond pass; zr = 7: runs crossing y tiles), then the sums of the new
    fields against the oracle's sums of the same fields."""
    n = 256
    p = _params("m2phi2", n, prec)
    st = _state("m2phi2", n, prec, seed=40 + zr)
    g = Lattice(p)
    g.set_kernel(5, 16, zr, 1)
    info = g.kernel_info()
    assert (info["variant"], info["ty"], info["depth"]) == (5, 16, 1)
    g.set_state(*st, t=0.0, a=1.05, ad=0.5)
    o = Oracle(p)
    o.set_state(*st, t=0.0, a=1.05, ad=0.5)
    del st
    g.evolve(2)
    o.step(2)
    compare_states(g, o, 2 * TOL[prec], f"27-point warp tiles zr={zr} fp{prec}")
    _check_scalars(g, o, prec, 2)
    o.close()
    _own_sums_check(g, p, prec)


def test_warp_tiles_27_fp64_512():
    """Variant 5 of the 27-point stencil in FP64 at N = 512 (four x tiles per row):
    one step against the oracle, and the sums of the new fields."""
    n = 512
    p = _params("lphi4", n, 64)
    st = _state("lphi4", n, 64, seed=91)
    g = Lattice(p)
    g.set_kernel(5)
    assert g.kernel_info()["variant"] == 5
    g.set_state(*st, t=0.0, a=1.02, ad=0.5)
    o = Oracle(p)
    o.set_state(*st, t=0.0, a=1.02, ad=0.5)
    del st
    g.evolve(1)
    o.step(1)
    compare_states(g, o, TOL[64], "27-point warp tiles FP64 512")
    o.close()
    _own_sums_check(g, p, 64)


def test_warp_tiles_27_match_plane_ring_kernel():
    """The two 27-point kernels (variant 2: full-row plane ring; variant 5: warp-wide
    tiles) from the same state: ten FP32 steps agree to FP32 rounding."""
    n = 256
    p = _params("lphi4", n, 32)
    st = _state("lphi4", n, 32, seed=17)
    a = Lattice(p)
    a.set_kernel(5)
    b = Lattice(p)
    b.set_kernel(2)
    for g in (a, b):
        g.set_state(*st, t=0.0, a=1.0, ad=0.4)
        g.evolve(10)
    for x, y in zip(a.get_state(), b.get_state()):
        assert normwise(x, y) <= 10 * 2e-6
