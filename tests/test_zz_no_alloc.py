"""lat_field_sums_static: the volume sums without any device allocation.

It exists for callers that cannot call cudaMalloc (memory already reserved by
another allocator, a fixed budget, or no room for cudaMalloc's implicit
synchronisation). Its scratch is a static device array shared by all calls, so
this test checks two calls in a row against the sums the handle path reports
(lat_get_scalars out[4..7]) for the same fields: to FP64 rounding for FP64
fields, to the FP32 rounding of the handle's sums (1e-6) for FP32 fields. This file is collected last so
that a run stopping at the first failure has already run every other test; it
passes alone in a fresh process and after the others.
"""
import numpy as np
import pytest

from paper_0911_5692_gb300 import Lattice
from paper_0911_5692_gb300.lattice import LatticeError, field_sums_static
from paper_0911_5692_gb300.workloads import lphi4, m2phi2, random_state

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("model", ["lphi4", "m2phi2"])
@pytest.mark.parametrize("n", [16, 36])
def test_static_sums_match_handle_sums(n, model, prec):
    import torch
    p = lphi4(n, precision=prec) if model == "lphi4" else m2phi2(n, precision=prec)
    st = random_state(n, 31 + n, precision=prec, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-3), pi_mean=(0.5, 0.0),
                      pi_amp=(1e-3, 1e-3))
    g = Lattice(p)
    g.set_state(*st, t=0.0, a=1.1, ad=0.4, step=0)
    ref = np.array(g.scalars()["S"])            # sums of the current fields, handle path
    f_phi = g.get_state_device(0, 0)
    f_chi = g.get_state_device(1, 0)
    out = torch.full((4,), float("nan"), dtype=torch.float64, device=g.device)
    for call in range(2):                        # the scratch is reused by the second call
        out.fill_(float("nan"))
        field_sums_static(f_phi, f_chi, n, prec, p["model"], p["L"], out, stream=g.stream)
        g.stream.synchronize()
        got = out.cpu().numpy()
        # FP64 on both sides for FP64 fields; a handle with FP32 fields forms
        # the sums in FP32 (exact differences, compensated per-thread sums)
        np.testing.assert_allclose(got, ref, rtol=1e-12 if prec == 64 else 1e-6, atol=0, err_msg=f"call {call}")


def test_static_sums_reject_bad_sizes():
    import torch
    x = torch.zeros(64, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(LatticeError) as e:
        field_sums_static(x, x, 6, 32, 0, 10.0, out)          # not a multiple of 4
    assert e.value.status == 1
    with pytest.raises(LatticeError) as e:
        field_sums_static(x, x, 2048, 32, 0, 10.0, out)       # beyond the largest lattice served
    assert e.value.status == 7
