"""GPU parity of the z-slab path (lat_slab_* and paper_0911_5692_gb300.slab):
a lattice cut into 1-4 slabs held by one process on one GPU (halos by device
copies, shares added on the device; no slab waits on another) against the
single-lattice GPU path and the FP64 oracle; a one-rank NCCL group through
DistComm; slab handles refuse whole-lattice calls."""
import ctypes as C
import os

import numpy as np
import pytest
import torch

from gpu_helpers import normwise
from oracle.oracle import Oracle
from paper_0911_5692_gb300 import Lattice
from paper_0911_5692_gb300.slab import DistComm, LocalComm, SlabEvolution, SlabGPU, slab_ranges
from paper_0911_5692_gb300.workloads import lphi4, m2phi2, random_state

pytestmark = pytest.mark.gpu

SCAL = dict(t=0.0, a=1.05, ad=0.4, step=0)


def _case(model, n, prec):
    if model == "lphi4":
        p = lphi4(n, precision=prec)
        st = random_state(n, 5, prec, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-3), pi_mean=(0.5, 0.0), pi_amp=(1e-3, 1e-3))
    else:
        p = m2phi2(n, precision=prec)
        st = random_state(n, 6, prec, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-4), pi_mean=(0.3, 0.0), pi_amp=(1e-3, 1e-2))
    return p, st


def _slabs(p, st, parts):
    slabs = [SlabGPU(p, z0, nzl) for z0, nzl in slab_ranges(p["n"], parts)]
    for s in slabs:
        s.load(*st, **SCAL)
    return slabs


@pytest.mark.parametrize("parts", [1, 2, 3, 4])
def test_slabs_match_single_lattice_fp64(parts):
    n, steps = 32, 9
    p, st = _case("lphi4", n, 64)
    slabs = _slabs(p, st, parts)
    ev = SlabEvolution(slabs, LocalComm())
    ev.prepare()
    ev.step(steps)
    got = ev.gather()
    g = Lattice(p)
    g.set_state(*st, **SCAL)
    g.evolve(steps)
    for a, b in zip(got, g.get_state()):
        assert normwise(a, b) <= 1e-13
    o = Oracle(p)
    o.set_state(*st, **SCAL)
    o.step(steps)
    for a, b in zip(got, o.get_state()):
        assert normwise(a, b) <= steps * 1e-12
    for s in slabs:
        sc = s.scalars()
        assert sc["step"] == steps
        assert abs(sc["a"] / o.scalars()["a"] - 1) <= 1e-13


@pytest.mark.parametrize("model,n,parts", [("m2phi2", 64, 3), ("lphi4", 128, 4)])
def test_slabs_fp32_match_oracle(model, n, parts):
    steps = 4
    p, st = _case(model, n, 32)
    slabs = _slabs(p, st, parts)
    ev = SlabEvolution(slabs, LocalComm())
    ev.prepare()
    ev.step(steps)
    got = ev.gather()
    o = Oracle(p)
    o.set_state(*st, **SCAL)
    o.step(steps)
    for a, b in zip(got, o.get_state()):
        assert normwise(a, b) <= steps * 2e-6


def test_one_rank_nccl_group():
    import torch.distributed as dist
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    os.environ.setdefault("MASTER_PORT", "29561")
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda", 0))
    try:
        n, steps = 32, 5
        p, st = _case("lphi4", n, 64)
        (s,) = _slabs(p, st, 1)
        ev = SlabEvolution([s], DistComm())
        ev.prepare()
        ev.step(steps)
        g = Lattice(p)
        g.set_state(*st, **SCAL)
        g.evolve(steps)
        for a, b in zip(ev.gather(), g.get_state()):
            assert normwise(a, b) <= 1e-13
    finally:
        dist.destroy_process_group()


def test_slab_refuses_whole_lattice_calls():
    p, st = _case("lphi4", 32, 32)
    (s,) = _slabs(p, st, 1)
    L = s._L
    assert L.lat_evolve(s._h, 1) == 8          # LAT_ESTATE
    assert L.lat_init_fields(s._h) == 8
    assert L.lat_set_kernel(s._h, 1, 0, 0, 0) == 8
