"""GPU parity of the per-site energy density and pressure (lat_energy_field;
Sec. II.B, eq. rho-pres per site, the paper's second kernel) against the FP64
oracle, through the C ABI.

Tolerances (normwise, max|gpu - oracle| / max|oracle|): FP64 1e-12; FP32 2e-6
(each site's terms are formed in the lattice precision from exact neighbour
differences). States with zero field means make the kinetic, gradient and
potential parts of comparable size, so the gradient part is tested at the same
tolerance as the whole.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import normwise, paired
from paper_0911_5692_gb300 import Lattice
from paper_0911_5692_gb300.workloads import lphi4, m2phi2, random_state

pytestmark = pytest.mark.gpu

TOL = {32: 2e-6, 64: 1e-12}


def _case(model, n, prec, stencil, expansion, centred):
    p = (lphi4 if model == "lphi4" else m2phi2)(n, precision=prec, expansion=expansion)
    p["stencil"] = stencil
    mean = (0.0, 0.0) if centred else (1.0, 0.0)
    st = random_state(n, 11 * n + stencil, precision=prec, f_mean=mean, f_amp=(1e-3, 1e-3),
                      pi_mean=(0.0, 0.0) if centred else (0.5, 0.0), pi_amp=(1e-3, 1e-3))
    return p, st


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("stencil", [7, 27])
@pytest.mark.parametrize("model,expansion,centred", [("lphi4", 1, False), ("m2phi2", 1, True), ("m2phi2", 0, True),
                                                     ("lphi4", 0, False)])
@pytest.mark.parametrize("n", [4, 20, 32])
def test_energy_field_parity(n, model, expansion, centred, stencil, prec):
    p, st = _case(model, n, prec, stencil, expansion, centred)
    sc = (0.0, 1.1, 0.4, 0) if expansion else (0.0, 1.0, 0.0, 0)
    g, o = paired(p, st, sc)
    rho, pres = g.energy_field()
    torch.cuda.synchronize()
    ro, po = o.energy_field()
    assert normwise(rho.double().cpu().numpy(), ro) <= TOL[prec]
    assert normwise(pres.double().cpu().numpy(), po) <= TOL[prec]


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("stencil", [7, 27])
def test_energy_field_means_are_lat_energies(prec, stencil):
    """The volume means of the fields are the averages lat_energies reports (FP64
    sums of the two FP64 diagnostics; FP32 fields summed in FP64)."""
    n = 32
    p, st = _case("lphi4", n, prec, stencil, 1, False)
    g, _ = paired(p, st, (0.0, 1.2, 0.3, 0))
    rho, pres = g.energy_field()
    e = g.energies()
    tol = 1e-12 if prec == 64 else 2e-6
    assert rho.double().mean().item() == pytest.approx(e["rho"], rel=tol)
    assert pres.double().mean().item() == pytest.approx(e["p"], rel=tol)


def test_energy_field_after_evolution_and_into_given_buffers():
    """After steps (the ping-pong parity and the device coefficients of the
    current step) and into caller-supplied tensors, against the oracle."""
    n = 24
    p, st = _case("m2phi2", n, 64, 27, 1, True)
    g, o = paired(p, st, (0.0, 1.05, 0.5, 0))
    g.evolve(7)
    o.step(7)
    rho = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
    pres = torch.empty_like(rho)
    r2, p2 = g.energy_field(rho, pres)
    assert r2 is rho and p2 is pres
    torch.cuda.synchronize()
    ro, po = o.energy_field()
    assert normwise(rho.cpu().numpy(), ro) <= 1e-11
    assert normwise(pres.cpu().numpy(), po) <= 1e-11


def test_energy_field_rejects_bad_buffers():
    n = 8
    g = Lattice(dict(lphi4(n, precision=32)))
    with pytest.raises(ValueError):
        g.energy_field(torch.empty((n, n, n), dtype=torch.float64, device="cuda"))


def test_energy_field_and_upload_on_a_slab():
    """The per-site fields are a whole-lattice diagnostic: a slab handle refuses
    them (LAT_ESTATE); its state can still be uploaded in one call."""
    from paper_0911_5692_gb300.slab import SlabGPU
    n = 16
    p = lphi4(n, precision=32)
    s = SlabGPU(p, 0, 8)
    rho = torch.empty((s.nzl + 3) * n * n, dtype=torch.float32, device="cuda")
    pres = torch.empty_like(rho)
    import ctypes as C
    st = s._L.lat_energy_field(s._h, C.c_void_p(rho.data_ptr()), C.c_void_p(pres.data_ptr()))
    assert st == 8
    src = [torch.full(((s.nzl + 3) * n * n,), float(k + 1), dtype=torch.float32, device="cuda") for k in range(4)]
    ptrs = (C.c_void_p * 4)(*[t.data_ptr() for t in src])
    assert s._L.lat_upload_state(s._h, ptrs, 1) == 0
    s.sync()
    for k in range(4):
        assert torch.equal(s.buffers[k], src[k].view_as(s.buffers[k]))
    s.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_energy_field_into_buffers_not_16_byte_aligned(prec):
    """Buffers aligned to their element but not to 16 bytes take the per-site
    kernel instead of the vector one; same results against the oracle."""
    n = 20
    p, st = _case("lphi4", n, prec, 7, 1, False)
    g, o = paired(p, st, (0.0, 1.1, 0.4, 0))
    dt = torch.float32 if prec == 32 else torch.float64
    base = torch.empty(2 * n ** 3 + 2, dtype=dt, device="cuda")
    rho, pres = base[1:1 + n ** 3], base[2 + n ** 3 - 1:2 * n ** 3 + 1]
    assert rho.data_ptr() % 16 != 0 and pres.data_ptr() % 16 != 0
    g.energy_field(rho, pres)
    torch.cuda.synchronize()
    ro, po = o.energy_field()
    assert normwise(rho.double().cpu().numpy().reshape(n, n, n), ro) <= TOL[prec]
    assert normwise(pres.double().cpu().numpy().reshape(n, n, n), po) <= TOL[prec]
    # the vector kernel gives the same fields
    r2, p2 = g.energy_field()
    torch.cuda.synchronize()
    assert normwise(r2.double().cpu().numpy(), ro) <= TOL[prec]
