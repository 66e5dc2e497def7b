"""lat_field_sums_static: the volume sums without any device allocation.

It exists for callers that cannot call cudaMalloc (memory already reserved by
another allocator, a fixed budget, or no room for cudaMalloc's implicit
synchronisation). Its scratch is a static device array shared by all calls, so
these tests check two calls in a row against the FP64 oracle's sums of the same
fields (orc_sums; FP64 arithmetic on both sides, so agreement to rounding) and
against the sums the handle path reports (lat_get_scalars out[4..7]; to FP64
rounding for FP64 fields, to the FP32 rounding of the handle's sums, 1e-6, for
FP32 fields), at small sides and at one side past 512, where the grid-stride
loop over columns and the full partial array are in use. This file is collected
last so that a run stopping at the first failure has already run every other
test; it passes alone in a fresh process and after the others.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_0911_5692_gb300 import Lattice
from paper_0911_5692_gb300.lattice import LatticeError, field_sums_static
from paper_0911_5692_gb300.workloads import lphi4, m2phi2, random_state

pytestmark = pytest.mark.gpu


def _static_twice(g, n, prec, p, f_phi, f_chi):
    """Two calls in a row on the lattice's stream; the output buffer is filled
    with NaN on that stream before each, so a call that wrote nothing fails."""
    import torch
    out = torch.empty(4, dtype=torch.float64, device=g.device)
    got = []
    for _ in range(2):                           # the scratch is reused by the second call
        with torch.cuda.stream(g.stream):
            out.fill_(float("nan"))
        field_sums_static(f_phi, f_chi, n, prec, p["model"], p["L"], out, stream=g.stream)
        g.stream.synchronize()
        got.append(out.cpu().numpy().copy())
    return got


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("model", ["lphi4", "m2phi2"])
@pytest.mark.parametrize("n", [16, 36])
def test_static_sums_match_oracle_and_handle(n, model, prec):
    p = lphi4(n, precision=prec) if model == "lphi4" else m2phi2(n, precision=prec)
    st = random_state(n, 31 + n, precision=prec, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-3), pi_mean=(0.5, 0.0),
                      pi_amp=(1e-3, 1e-3))
    g = Lattice(p)
    g.set_state(*st, t=0.0, a=1.1, ad=0.4, step=0)
    handle = np.array(g.scalars()["S"])          # sums of the current fields, handle path
    o = Oracle(p)
    o.set_state(*st, t=0.0, a=1.1, ad=0.4)
    oracle = np.array(o.scalars()["S"])
    for call, got in enumerate(_static_twice(g, n, prec, p, g.get_state_device(0, 0), g.get_state_device(1, 0))):
        np.testing.assert_allclose(got, oracle, rtol=1e-12, atol=0, err_msg=f"call {call} vs oracle")
        # a handle with FP32 fields forms the sums in FP32 (exact differences,
        # compensated per-thread sums)
        np.testing.assert_allclose(got, handle, rtol=1e-12 if prec == 64 else 1e-6, atol=0,
                                   err_msg=f"call {call} vs handle")


def test_static_sums_large_lattice():
    """FP32 n = 516: 516^2 columns exceed the 1024 blocks x 256 threads of one
    pass, so every thread strides over a second column and all 1024 partial
    slots of the scratch are written; against the oracle's sums."""
    import torch
    n = 516
    p = lphi4(n, precision=32)
    st = random_state(n, 5, precision=32, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-3), pi_mean=(0.0, 0.0),
                      pi_amp=(0.0, 0.0))
    o = Oracle(p)
    o.set_state(st[0], st[1], st[2], st[3], t=0.0, a=1.0, ad=0.0)
    oracle = np.array(o.scalars()["S"])
    o.close()
    g = Lattice(dict(p, n=16))                   # supplies the stream only
    f_phi = torch.from_numpy(st[0].astype(np.float32).reshape(-1)).to(g.device)
    f_chi = torch.from_numpy(st[1].astype(np.float32).reshape(-1)).to(g.device)
    del st
    torch.cuda.synchronize()
    for call, got in enumerate(_static_twice(g, n, 32, p, f_phi, f_chi)):
        np.testing.assert_allclose(got, oracle, rtol=1e-12, atol=0, err_msg=f"call {call}")


def test_static_sums_reject_bad_sizes():
    import torch
    x = torch.zeros(64, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(LatticeError) as e:
        field_sums_static(x, x, 2, 32, 0, 10.0, out)          # below the smallest side
    assert e.value.status == 1
    with pytest.raises(LatticeError) as e:
        field_sums_static(x, x, 2048, 32, 0, 10.0, out)       # beyond the sides the library serves
    assert e.value.status == 7
