"""GPU parity of the reverse-mode derivative (lat_vjp / lat_adjoint and the
torch.autograd binding) against the FP64 oracle's adjoint and against central
finite differences of the GPU's own forward map.

Tolerances: FP64 lattices agree with the oracle to 1e-10 normwise (the two
sum the volume reductions in different orders). FP32 lattices (phi stored
whole: the derivative does not take split lattices): every step of the forward
recomputation and of the reverse sweep rounds each field value once or a few
times to u = 2^-24 relative; the leapfrog's propagator neither grows nor damps
these perturbations outside a resonance band, so after n steps they add up to
about n times a few u. On top of that, phi ~ 1 held in FP32 is rounded to
about 6e-8, which is 6e-5 of the 1e-3 fluctuations of the test states, and the
gradient, which depends on those fluctuations, carries that relative error. The
bound used is fp32_tol(n) = 6e-5 + 16 n u (1.1e-4 at 50 steps, 2.5e-4 at 200),
normwise against an FP64 reference. The central-difference check
on 16^3 FP64 is the contract's rel <= 1e-5, asserted at 1e-7. Results do not
depend on the checkpoint interval, bit for bit.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import normwise
from oracle.oracle import Oracle
from paper_0911_5692_gb300 import Lattice, LatticeError
from paper_0911_5692_gb300.autograd import LatticeEvolve
from paper_0911_5692_gb300.workloads import lphi4, m2phi2, random_state

pytestmark = pytest.mark.gpu


def fp32_tol(steps):
    """Normwise bound of an FP32 gradient against an FP64 one after `steps`
    steps (module docstring): 6e-5 + 16 n u, u = 2^-24."""
    return 6e-5 + 16 * steps * 2.0 ** -24


def _case(model, n, prec, expansion=1):
    if model == "lphi4":
        p = lphi4(n, precision=prec, expansion=expansion)
        st = random_state(n, 3, prec, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-3), pi_mean=(0.5, 0.0), pi_amp=(1e-3, 1e-3))
        sc = dict(t=0.0, a=1.1 if expansion else 1.0, ad=0.45 if expansion else 0.0, step=0)
    else:
        p = m2phi2(n, precision=prec, expansion=expansion)
        st = random_state(n, 4, prec, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-4), pi_mean=(0.3, 0.0), pi_amp=(1e-3, 1e-2))
        sc = dict(t=0.0, a=1.0, ad=0.3 if expansion else 0.0, step=0)
    return p, st, sc


def _gpu(p, st, sc):
    g = Lattice(p)
    g.set_state(*st, **sc)
    return g


def _oracle_grad(p, st, sc, nsteps):
    o = Oracle(p)
    o.set_state(*st, **sc)
    return o.chi2_gradient(nsteps)


@pytest.mark.parametrize("model,expansion", [("lphi4", 1), ("lphi4", 0), ("m2phi2", 1)])
def test_adjoint_fp64_matches_oracle(model, expansion):
    n, steps = 16, 40
    p, st, sc = _case(model, n, 64, expansion)
    g = _gpu(p, st, sc)
    J, df, dp, dg2 = g.adjoint(steps)
    Jo, dfo, dpo, dg2o = _oracle_grad(p, st, sc, steps)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    assert abs(dg2 - dg2o) <= 1e-10 * abs(dg2o)
    df, dp = df.cpu().numpy(), dp.cpu().numpy()
    for i in (0, 1):
        assert normwise(df[i], dfo[i]) <= 1e-10, ("df", i)
        assert normwise(dp[i], dpo[i]) <= 1e-10, ("dp", i)


@pytest.mark.parametrize("n,steps", [(32, 9), (64, 6), (96, 3)])
def test_adjoint_march_kernel_fp64(n, steps):
    """N a multiple of 32 takes the z-march reverse kernel (several z chunks)."""
    p, st, sc = _case("lphi4", n, 64)
    g = _gpu(p, st, sc)
    J, df, dp, dg2 = g.adjoint(steps)
    Jo, dfo, dpo, dg2o = _oracle_grad(p, st, sc, steps)
    assert abs(dg2 - dg2o) <= 1e-10 * abs(dg2o)
    df, dp = df.cpu().numpy(), dp.cpu().numpy()
    for i in (0, 1):
        assert normwise(df[i], dfo[i]) <= 1e-10, ("df", i)
        assert normwise(dp[i], dpo[i]) <= 1e-10, ("dp", i)


def test_adjoint_ends_at_final_state():
    n, steps = 16, 25
    p, st, sc = _case("lphi4", n, 64)
    g = _gpu(p, st, sc)
    g.adjoint(steps)
    ref = _gpu(p, st, sc)
    ref.evolve(steps)
    for x, y in zip(g.get_state(), ref.get_state()):
        assert np.array_equal(x, y)
    assert g.scalars() == ref.scalars()
    # and continues exactly like the reference
    g.evolve(5)
    ref.evolve(5)
    for x, y in zip(g.get_state(), ref.get_state()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("prec", [32, 64])
def test_checkpoint_interval_does_not_change_result(prec):
    n, steps = 32, 37
    p, st, sc = _case("lphi4", n, prec)
    outs = []
    for k in (1, 5, 0, 37, 100):
        g = _gpu(p, st, sc)
        J, df, dp, dg2 = g.adjoint(steps, ckpt_every=k)
        outs.append((J, df.cpu().numpy(), dp.cpu().numpy(), dg2))
    for o in outs[1:]:
        assert o[0] == outs[0][0] and o[3] == outs[0][3]
        assert np.array_equal(o[1], outs[0][1]) and np.array_equal(o[2], outs[0][2])


def test_central_difference_on_gpu_fp64():
    """P9: the GPU adjoint against central differences of the GPU forward map."""
    n, steps = 16, 60
    p, st, sc = _case("lphi4", n, 64)
    g = _gpu(p, st, sc)
    _, df, dp, dg2 = g.adjoint(steps)

    def J_of(state, g2=None):
        h = Lattice(p)
        if g2 is not None:
            h.set_g2(g2)
        h.set_state(*state, **sc)
        return _final_J(h, steps)

    e = 1e-6 * p["g2"]
    fd = (J_of(st, p["g2"] + e) - J_of(st, p["g2"] - e)) / (2 * e)
    assert abs(dg2 - fd) <= 1e-7 * abs(fd)
    rng = np.random.default_rng(8)
    u = [1e-6 * rng.standard_normal((n, n, n)) for _ in range(4)]
    fdd = (J_of([s + d for s, d in zip(st, u)]) - J_of([s - d for s, d in zip(st, u)])) / 2
    grads = [df[0], df[1], dp[0], dp[1]]
    ad = sum(float(np.sum(gr.cpu().numpy() * d)) for gr, d in zip(grads, u))
    assert abs(ad - fdd) <= 1e-7 * abs(fdd)


def _final_J(h, steps):
    h.evolve(steps)
    return h.adjoint(0)[0]


def test_zero_steps_is_observable_and_its_gradient():
    n = 16
    p, st, sc = _case("lphi4", n, 64)
    g = _gpu(p, st, sc)
    J, df, dp, dg2 = g.adjoint(0)
    f1 = st[1]
    assert J == pytest.approx(float(np.mean(f1 * f1)), rel=1e-13)
    assert np.allclose(df[1].cpu().numpy(), 2 * f1 / n ** 3, rtol=1e-15, atol=0)
    assert np.max(np.abs(df[0].cpu().numpy())) == 0 and np.max(np.abs(dp.cpu().numpy())) == 0
    assert dg2 == 0.0


def test_general_vjp_matches_oracle():
    """lat_vjp with an arbitrary adjoint of the final state, a and a' included."""
    n, steps = 16, 20
    p, st, sc = _case("lphi4", n, 64)
    rng = np.random.default_rng(4)
    v = [rng.standard_normal((n, n, n)) for _ in range(4)]
    va, vad = 0.7, -1.3
    g = _gpu(p, st, sc)
    fb = torch.tensor(np.concatenate([v[0].ravel(), v[1].ravel()]), device="cuda")
    pb = torch.tensor(np.concatenate([v[2].ravel(), v[3].ravel()]), device="cuda")
    ba, bad, bk0, bg2 = g.vjp(steps, fb, pb, va, vad)
    o = Oracle(p)
    o.set_state(*st, **sc)
    fbo, pbo, bao, bado, bk0o, bg2o = o.vjp(steps, v[0:2], v[2:4], va, vad)
    assert abs(ba - bao) <= 1e-10 * abs(bao)
    assert abs(bad - bado) <= 1e-10 * abs(bado)
    assert abs(bk0 - bk0o) <= 1e-10 * abs(bk0o)
    fb, pb = fb.cpu().numpy().reshape(2, n, n, n), pb.cpu().numpy().reshape(2, n, n, n)
    for i in (0, 1):
        assert normwise(fb[i], fbo[i]) <= 1e-10
        assert normwise(pb[i], pbo[i]) <= 1e-10


@pytest.mark.parametrize("variant", [2, 4])
def test_other_step_kernels(variant):
    """Handles configured for either plane-ring step kernel (full rows or x
    tiles) give the same derivative."""
    n, steps = 32, 12
    p, st, sc = _case("lphi4", n, 64)
    g = _gpu(p, st, sc)
    try:
        g.set_kernel(variant)
    except LatticeError:
        pytest.skip("variant unavailable")
    J, df, dp, dg2 = g.adjoint(steps)
    Jo, dfo, dpo, dg2o = _oracle_grad(p, st, sc, steps)
    assert abs(dg2 - dg2o) <= 1e-10 * abs(dg2o)
    for i in (0, 1):
        assert normwise(df[i].cpu().numpy(), dfo[i]) <= 1e-10


@pytest.mark.parametrize("model", ["lphi4", "m2phi2"])
def test_adjoint_fp32_matches_oracle(model):
    n, steps = 32, 50
    p, st, sc = _case(model, n, 32)
    g = _gpu(p, st, sc)
    J, df, dp, dg2 = g.adjoint(steps)
    Jo, dfo, dpo, dg2o = _oracle_grad(dict(p, precision=64), st, sc, steps)
    assert abs(J - Jo) <= fp32_tol(steps) * abs(Jo)
    assert abs(dg2 - dg2o) <= fp32_tol(steps) * abs(dg2o), (dg2, dg2o)
    df, dp = df.cpu().numpy(), dp.cpu().numpy()
    for i in (0, 1):
        assert normwise(df[i], dfo[i]) <= fp32_tol(steps), ("df", i, normwise(df[i], dfo[i]))
        assert normwise(dp[i], dpo[i]) <= fp32_tol(steps), ("dp", i, normwise(dp[i], dpo[i]))


@pytest.mark.parametrize("model,n,steps", [("lphi4", 64, 12), ("m2phi2", 64, 12), ("lphi4", 128, 4)])
def test_adjoint_pair_kernel_fp32(model, n, steps):
    """FP32 lattices with N a multiple of 64 take the two-site reverse kernel."""
    p, st, sc = _case(model, n, 32)
    g = _gpu(p, st, sc)
    J, df, dp, dg2 = g.adjoint(steps)
    Jo, dfo, dpo, dg2o = _oracle_grad(dict(p, precision=64), st, sc, steps)
    assert abs(J - Jo) <= fp32_tol(steps) * abs(Jo)
    assert abs(dg2 - dg2o) <= fp32_tol(steps) * abs(dg2o), (dg2, dg2o)
    df, dp = df.cpu().numpy(), dp.cpu().numpy()
    for i in (0, 1):
        assert normwise(df[i], dfo[i]) <= fp32_tol(steps), ("df", i, normwise(df[i], dfo[i]))
        assert normwise(dp[i], dpo[i]) <= fp32_tol(steps), ("dp", i, normwise(dp[i], dpo[i]))


def test_autograd_function():
    n, steps = 16, 15
    p, st, sc = _case("lphi4", n, 64)
    g = Lattice(p)
    f = torch.tensor(np.stack(st[0:2]), device="cuda", requires_grad=True)
    pi = torch.tensor(np.stack(st[2:4]), device="cuda", requires_grad=True)
    g2 = torch.tensor(p["g2"], dtype=torch.float64, requires_grad=True)
    J = LatticeEvolve.apply(f, pi, g2, g, steps, sc)
    (J * 3.0).backward()
    Jo, dfo, dpo, dg2o = _oracle_grad(p, st, sc, steps)
    assert float(J) == pytest.approx(Jo, rel=1e-12)
    assert abs(float(g2.grad) - 3 * dg2o) <= 1e-10 * abs(3 * dg2o)
    for i in (0, 1):
        assert normwise(f.grad[i].cpu().numpy(), 3 * dfo[i]) <= 1e-10
        assert normwise(pi.grad[i].cpu().numpy(), 3 * dpo[i]) <= 1e-10
    # without gradients the same J comes from the plain evolution
    J2 = LatticeEvolve.apply(f.detach(), pi.detach(), g2.detach(), g, steps, sc)
    assert float(J2) == float(J)


def test_set_g2_matches_fresh_handle():
    n = 32
    p, st, sc = _case("lphi4", n, 32)
    a = _gpu(p, st, sc)
    a.set_g2(2.5 * p["g2"])
    a.set_state(*st, **sc)
    b = _gpu(dict(p, g2=2.5 * p["g2"]), st, sc)
    a.evolve(40)
    b.evolve(40)
    for x, y in zip(a.get_state(), b.get_state()):
        assert np.array_equal(x, y)
    with pytest.raises(LatticeError):
        a.set_g2(-1.0)


# ------------------------------------------------------------------ observable 1: energy fraction in chi

def _oracle_frac(p, st, sc, nsteps):
    o = Oracle(p)
    o.set_state(*st, **sc)
    return o.chi_fraction_gradient(nsteps)


@pytest.mark.parametrize("model,expansion", [("lphi4", 1), ("lphi4", 0), ("m2phi2", 1)])
def test_energy_fraction_fp64_matches_oracle(model, expansion):
    n, steps = 16, 40
    p, st, sc = _case(model, n, 64, expansion)
    g = _gpu(p, st, sc)
    J, df, dp, dg2 = g.adjoint(steps, observable=1)
    Jo, dfo, dpo, dg2o = _oracle_frac(p, st, sc, steps)
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    assert abs(dg2 - dg2o) <= 1e-10 * abs(dg2o)
    df, dp = df.cpu().numpy(), dp.cpu().numpy()
    for i in (0, 1):
        assert normwise(df[i], dfo[i]) <= 1e-10, ("df", i)
        assert normwise(dp[i], dpo[i]) <= 1e-10, ("dp", i)


def test_energy_fraction_zero_steps_is_the_oracle_seed():
    n = 16
    p, st, sc = _case("lphi4", n, 64)
    g = _gpu(p, st, sc)
    J, df, dp, dg2 = g.adjoint(0, observable=1)
    o = Oracle(p)
    o.set_state(*st, **sc)
    Jo, fbo, pbo, _, _, dg2o = o.chi_fraction(with_gradient=True)
    assert J == pytest.approx(Jo, rel=1e-13)
    assert dg2 == pytest.approx(dg2o, rel=1e-12)
    df, dp = df.cpu().numpy(), dp.cpu().numpy()
    for i in (0, 1):
        assert normwise(df[i], fbo[i]) <= 1e-12
        assert normwise(dp[i], pbo[i]) <= 1e-12


def test_energy_fraction_central_difference_on_gpu_fp64():
    """dJ/dg2 of the GPU's own forward map by central differences (16^3 FP64)."""
    n, steps = 16, 30
    p, st, sc = _case("lphi4", n, 64)

    def final(g2):
        g = Lattice(dict(p, g2=g2))
        g.set_state(*st, **sc)
        return g.adjoint(steps, observable=1)[0]

    g = _gpu(p, st, sc)
    _, _, _, dg2 = g.adjoint(steps, observable=1)
    e = 1e-6 * p["g2"]
    fd = (final(p["g2"] + e) - final(p["g2"] - e)) / (2 * e)
    assert abs(dg2 - fd) <= 1e-7 * abs(fd)


@pytest.mark.parametrize("n,steps", [(32, 50), (64, 12)])
def test_energy_fraction_fp32_matches_oracle(n, steps):
    p, st, sc = _case("lphi4", n, 32)
    g = _gpu(p, st, sc)
    J, df, dp, dg2 = g.adjoint(steps, observable=1)
    Jo, dfo, dpo, dg2o = _oracle_frac(dict(p, precision=64), st, sc, steps)
    assert abs(J - Jo) <= fp32_tol(steps) * abs(Jo)
    assert abs(dg2 - dg2o) <= fp32_tol(steps) * abs(dg2o), (dg2, dg2o)
    df, dp = df.cpu().numpy(), dp.cpu().numpy()
    for i in (0, 1):
        assert normwise(df[i], dfo[i]) <= fp32_tol(steps), ("df", i, normwise(df[i], dfo[i]))
        assert normwise(dp[i], dpo[i]) <= fp32_tol(steps), ("dp", i, normwise(dp[i], dpo[i]))


def test_autograd_energy_fraction():
    n, steps = 16, 15
    p, st, sc = _case("lphi4", n, 64)
    g = Lattice(p)
    f = torch.tensor(np.stack(st[0:2]), device="cuda", requires_grad=True)
    pi = torch.tensor(np.stack(st[2:4]), device="cuda", requires_grad=True)
    g2 = torch.tensor(p["g2"], dtype=torch.float64, requires_grad=True)
    J = LatticeEvolve.apply(f, pi, g2, g, steps, sc, 0, 1)
    J.backward()
    Jo, dfo, dpo, dg2o = _oracle_frac(p, st, sc, steps)
    assert float(J) == pytest.approx(Jo, rel=1e-12)
    assert abs(float(g2.grad) - dg2o) <= 1e-10 * abs(dg2o)
    for i in (0, 1):
        assert normwise(f.grad[i].cpu().numpy(), dfo[i]) <= 1e-10
        assert normwise(pi.grad[i].cpu().numpy(), dpo[i]) <= 1e-10



@pytest.mark.parametrize("observable", [0, 1])
def test_adjoint_fp32_against_fp64_c5_shape(observable):
    """The derivative configuration's shape (lambda phi^4, 128^3, vacuum
    initial conditions, J = <chi^2> or the energy fraction in chi) over 200
    steps: the FP32 gradient against the FP64 gradient of the same start on the
    GPU (the FP64 path is pinned to the oracle above), within fp32_tol(200) =
    2.5e-4 normwise for dJ/df and dJ/dpi and relative for dJ/dg^2."""
    n, steps = 128, 200
    p = lphi4(n, precision=64)
    g64 = Lattice(p)
    g64.init_fields()
    st = g64.get_state()
    sc = g64.scalars()
    g32 = Lattice(dict(p, precision=32))
    g32.set_state(*st, t=sc["t"], a=sc["a"], ad=sc["ad"], step=sc["step"])
    # both from the FP32-representable start
    g64.set_state(*g32.get_state(), t=sc["t"], a=sc["a"], ad=sc["ad"], step=sc["step"])
    J32, df32, dp32, dg32 = g32.adjoint(steps, observable=observable)
    J64, df64, dp64, dg64 = g64.adjoint(steps, observable=observable)
    tol = fp32_tol(steps)
    errs = {"J": abs(J32 / J64 - 1), "dg2": abs(dg32 / dg64 - 1)}
    for i in (0, 1):
        errs[f"df{i}"] = normwise(df32[i].double().cpu().numpy(), df64[i].cpu().numpy())
        errs[f"dp{i}"] = normwise(dp32[i].double().cpu().numpy(), dp64[i].cpu().numpy())
    assert max(errs.values()) <= tol, errs
