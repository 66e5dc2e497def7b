"""lat_evolve_host: a state held in page-locked host memory evolved step by
step through the GPU (upload, the sums of the uploaded fields, the fused step,
download; the copies in z-chunks on one stream per direction) against the
same steps taken call by call (lat_upload_state, lat_evolve, lat_download_state,
lat_get_scalars) and against the FP64 oracle."""
import numpy as np
import pytest
import torch

from gpu_helpers import normwise
from oracle.oracle import Oracle
from paper_0911_5692_gb300 import Lattice, LatticeError
from paper_0911_5692_gb300.workloads import lphi4, m2phi2, random_state

pytestmark = pytest.mark.gpu

SCAL = dict(t=0.0, a=1.05, ad=0.4, step=0)


def _host(lat, st, pinned=True):
    dt = torch.float32 if lat.precision == 32 else torch.float64
    ts = [torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).to(dt) for x in st]
    return [t.pin_memory() for t in ts] if pinned else ts


def _stored(lat):
    """The four stored arrays of the lattice's current state (host, pinned)."""
    ts = [torch.empty(lat.n ** 3, dtype=lat.dtype).pin_memory() for _ in range(4)]
    lat.download_state(*ts)
    return ts


@pytest.mark.parametrize("prec,n,chunks,split", [(32, 64, 0, 0), (32, 48, 5, 1), (64, 48, 1, 0), (32, 36, 64, 0),
                                                 (64, 64, 3, 1)])
def test_matches_call_by_call_loop(prec, n, chunks, split):
    """Bit-identical arrays and scalars after every step, whatever the chunking
    (ragged chunks of a 48-plane lattice, more chunks than planes)."""
    p = dict(m2phi2(n, precision=prec), split=split) if n == 48 else dict(lphi4(n, precision=prec), split=split)
    st = random_state(n, 3 + n, prec, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-3), pi_mean=(0.4, 0.0),
                      pi_amp=(1e-3, 1e-3))
    a, b = Lattice(p), Lattice(p)
    for g in (a, b):
        g.set_state(*st, **SCAL)
    ha, hb = _stored(a), _stored(b)
    steps = 4
    rows = a.evolve_host(*ha, n_steps=steps, chunks=chunks)
    assert rows.shape == (steps, 8)
    for k in range(steps):
        b.upload_state(*hb)
        b.evolve(1)
        b.download_state(*hb)
        sc = b.scalars()
        assert rows[k, 3] == sc["step"] == k + 1
        assert (rows[k, 0], rows[k, 1], rows[k, 2]) == (sc["t"], sc["a"], sc["ad"])
        assert list(rows[k, 4:]) == list(sc["S"])
    for x, y in zip(ha, hb):
        assert torch.equal(x, y)
    assert a.scalars() == b.scalars()


def test_against_oracle():
    n, steps = 32, 5
    p = lphi4(n, precision=64)
    st = random_state(n, 9, 64, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-3), pi_mean=(0.5, 0.0), pi_amp=(1e-3, 1e-3))
    g = Lattice(p)
    g.set_state(*st, **SCAL)
    h = _host(g, st)
    g.evolve_host(*h, n_steps=steps)
    o = Oracle(p)
    o.set_state(*st, **SCAL)
    o.step(steps)
    for x, y in zip(h, o.get_state()):
        assert normwise(x.numpy().reshape(n, n, n), y) <= steps * 1e-12
    assert abs(g.scalars()["a"] / o.scalars()["a"] - 1) <= 1e-13


def test_refusals():
    """Pageable host memory, chunks out of range and a negative step count are
    LAT_EINVAL; zero steps leave the state alone."""
    n = 16
    p = lphi4(n, precision=32)
    st = random_state(n, 2, 32)
    g = Lattice(p)
    g.set_state(*st, **SCAL)
    for pinned, steps, chunks in ((False, 2, 0), (True, 2, 65), (True, 2, -1), (True, -1, 0)):
        h = _host(g, st, pinned)
        with pytest.raises(LatticeError) as e:
            g.evolve_host(*h, n_steps=steps, chunks=chunks)
        assert e.value.status == 1
    h = _host(g, st)
    before = [t.clone() for t in h]
    assert g.evolve_host(*h, n_steps=0).shape == (0, 8)
    for x, y in zip(h, before):
        assert torch.equal(x, y)
    assert g.scalars()["step"] == 0

