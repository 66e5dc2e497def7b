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
from paper_0911_5692_gb300.slab import DistComm, LocalComm, SlabEvolution, SlabGPU, overlap_ranges, slab_ranges
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


@pytest.mark.parametrize("overlap", [False, True])
@pytest.mark.parametrize("model,n,parts", [("m2phi2", 64, 3), ("lphi4", 128, 4), ("lphi4", 256, 2), ("m2phi2", 256, 3),
                                          ("lphi4", 256, 10)])
def test_slabs_fp32_match_oracle(model, n, parts, overlap):
    """N = 256 takes the compiled warp-tile slab instance, the others the generic
    plane ring; overlap: interior planes first, then the boundary pairs. Ten
    slabs need more than one launch per schedule step (at most 8 slabs and 16
    ranges a launch)."""
    steps = 4
    p, st = _case(model, n, 32)
    slabs = _slabs(p, st, parts)
    ev = SlabEvolution(slabs, LocalComm(), overlap=overlap)
    assert ev.overlap == overlap
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


def _poison_halos(s):
    """NaN in every halo plane of the slab's current set (stored 0, nzl + 1, nzl + 2)."""
    with torch.cuda.stream(s.stream):
        for a in range(4):
            for q in (0, s.nzl + 1, s.nzl + 2):
                s.plane(a, q).fill_(float("nan"))


@pytest.mark.parametrize("n,prec,parts", [(256, 32, 2), (48, 64, 3)])
def test_interior_range_reads_no_halo(n, prec, parts):
    """Before each step the halo planes of every slab are NaN while the interior
    range (planes 2 .. nzl - 3) is stepped; the exchange then fills them and the
    boundary pairs are stepped. Any halo read by the interior range would carry
    a NaN into the fields or the sums (a sticky non-finite status). N = 256 FP32:
    the warp-tile slab instance; N = 48 FP64: the generic plane ring."""
    steps = 3
    p, st = _case("lphi4", n, prec)
    slabs = _slabs(p, st, parts)
    comm = LocalComm()
    ev = SlabEvolution(slabs, comm)
    ev.prepare()
    for _ in range(steps):
        for s in slabs:
            _poison_halos(s)
            zf, zc = overlap_ranges(s.nzl)[0]
            s.local_step_range(zf, zc, 0)
        comm.exchange(slabs)
        for s in slabs:
            for slot, (zf, zc) in enumerate(overlap_ranges(s.nzl)[1:], start=1):
                s.local_step_range(zf, zc, slot)
        totals = comm.allreduce(slabs, [s.range_total() for s in slabs])
        for s, t in zip(slabs, totals):
            s.advance(t, True)
    got = ev.gather()
    for s in slabs:
        assert np.isfinite(s.scalars()["S"]).all()
    o = Oracle(p)
    o.set_state(*st, **SCAL)
    o.step(steps)
    tol = steps * (2e-6 if prec == 32 else 1e-12)
    for a, b in zip(got, o.get_state()):
        assert normwise(a, b) <= tol


def test_range_arguments_checked():
    p, st = _case("lphi4", 32, 32)
    (s,) = _slabs(p, st, 1)
    L = s._L
    out = C.c_void_p(s.range_shares.data_ptr())
    for zf, zc in ((-1, 2), (0, 0), (31, 2), (0, 33)):
        assert L.lat_slab_step_range(s._h, zf, zc, out) == 1     # LAT_EINVAL
    assert L.lat_slab_step_range(s._h, 0, 32, None) == 1


def test_copy_regions_bit_exact():
    """lat_copy_regions moves every region whole (70 regions: two launches of
    at most 64), leaves the bytes around them alone and copies nothing for
    count 0."""
    from paper_0911_5692_gb300.lattice import load_library
    L = load_library()
    g = torch.Generator(device="cuda").manual_seed(3)
    words = 4 * 1031                      # 16.5 KB regions, not a multiple of the block stride
    src = torch.randint(-2**31, 2**31 - 1, (70, words + 8), dtype=torch.int32, device="cuda", generator=g)
    dst = torch.zeros_like(src)
    stream = torch.cuda.current_stream()
    d = (C.c_void_p * 70)(*[dst[i].data_ptr() for i in range(70)])
    q = (C.c_void_p * 70)(*[src[i].data_ptr() for i in range(70)])
    assert L.lat_copy_regions(d, q, 70, words * 4, C.c_void_p(stream.cuda_stream)) == 0
    torch.cuda.synchronize()
    assert torch.equal(dst[:, :words], src[:, :words])
    assert not dst[:, words:].any()
    assert L.lat_copy_regions(d, q, 0, words * 4, C.c_void_p(stream.cuda_stream)) == 0


@pytest.mark.parametrize("parts", [2, 4])
def test_fused_advance_matches_allreduce(parts):
    """lat_slab_advance_local (shares added in the order given, every slab
    advanced in one launch) gives the scalars of an allreduce followed by
    lat_slab_advance on each slab, to the rounding of the sum's order."""
    n = 64
    p, st = _case("m2phi2", n, 64)
    a = _slabs(p, st, parts)
    b = _slabs(p, st, parts)
    comm = LocalComm()
    for slabs in (a, b):
        comm.exchange(slabs)
    shares_a = [s.local_sums() for s in a]
    comm.reduce_advance(a, shares_a, False)
    totals = comm.allreduce(b, [s.local_sums() for s in b])
    for s, t in zip(b, totals):
        s.advance(t, False)
    for slabs in (a, b):
        comm.exchange(slabs)
    comm.reduce_advance(a, [s.local_step() for s in a], True)
    totals = comm.allreduce(b, [s.local_step() for s in b])
    for s, t in zip(b, totals):
        s.advance(t, True)
    for x, y in zip(a, b):
        sx, sy = x.scalars(), y.scalars()
        assert sx["step"] == sy["step"] == 1 and x.step_count == y.step_count == 1
        for k in ("t", "a", "ad"):
            assert abs(sx[k] - sy[k]) <= 1e-14 * max(1.0, abs(sy[k])), k
        for u, v in zip(sx["S"], sy["S"]):
            assert abs(u - v) <= 1e-14 * max(1.0, abs(v))
    sa = [x.scalars() for x in a]
    assert all(s == sa[0] for s in sa[1:])      # one total: every slab holds the same scalars


def test_fused_advance_refusals():
    from paper_0911_5692_gb300.lattice import load_library
    L = load_library()
    p, st = _case("lphi4", 32, 32)
    s32 = _slabs(p, st, 2)
    q, st2 = _case("lphi4", 48, 32)
    (s48,) = _slabs(q, st2, 1)
    sh = (C.c_void_p * 1)(s32[0].shares.data_ptr())
    mixed = (C.c_void_p * 2)(s32[0]._h.value, s48._h.value)
    assert L.lat_slab_advance_local(mixed, 2, sh, 1, 1) == 1        # slabs of different lattices
    g = Lattice(p)
    whole = (C.c_void_p * 1)(g._h.value)
    assert L.lat_slab_advance_local(whole, 1, sh, 1, 1) == 8        # not a slab: LAT_ESTATE


def _ranges_arg(ranges):
    flat = [int(v) for r in ranges for v in r]
    return (C.c_int32 * max(1, len(flat)))(*flat)


@pytest.mark.parametrize("n,prec,parts", [(256, 32, 4), (512, 32, 3), (256, 64, 2)])
def test_step_ranges_one_launch_matches_per_slab(n, prec, parts):
    """lat_slab_step_ranges over every slab's owned planes (and over the
    interior and boundary ranges of the overlapped schedule) writes the fields
    the per-slab launches write, bit for bit, and shares that add to theirs."""
    from paper_0911_5692_gb300.lattice import load_library
    L = load_library()
    p, st = _case("lphi4", n, prec)
    a = _slabs(p, st, parts)
    b = _slabs(p, st, parts)
    comm = LocalComm()
    for slabs in (a, b):
        SlabEvolution(slabs, comm).prepare()
    comm.exchange(a)
    comm.exchange(b)
    # a: one launch; b: one launch per slab
    got = comm.step_ranges(a, [(i, 0, s.nzl) for i, s in enumerate(a)], 0)
    assert len(got) == 1
    ref = [s.local_step() for s in b]          # queued on each slab's own stream
    torch.cuda.synchronize()
    total = sum(r.clone() for r in ref)
    assert torch.allclose(got[0], total, rtol=1e-12 if prec == 64 else 1e-5, atol=0)
    for x, y in zip(a, b):
        for k in range(8):
            assert torch.equal(x.buffers[k][1:x.nzl + 1], y.buffers[k][1:y.nzl + 1])
    # the overlapped schedule's two launches step the same planes
    c = _slabs(p, st, parts)
    SlabEvolution(c, comm).prepare()
    comm.exchange(c)
    comm.step_ranges(c, [(i, *overlap_ranges(s.nzl)[0]) for i, s in enumerate(c)], 0)
    comm.step_ranges(c, [(i, zf, zc) for i, s in enumerate(c) for zf, zc in overlap_ranges(s.nzl)[1:]], 1)
    torch.cuda.synchronize()
    for x, y in zip(c, b):
        for k in range(8):
            assert torch.equal(x.buffers[k][1:x.nzl + 1], y.buffers[k][1:y.nzl + 1])


def test_step_ranges_refusals():
    from paper_0911_5692_gb300.lattice import load_library
    L = load_library()
    p, st = _case("lphi4", 256, 32)
    slabs = _slabs(p, st, 2)
    hs = (C.c_void_p * 2)(slabs[0]._h.value, slabs[1]._h.value)
    out = C.c_void_p(slabs[0].shares.data_ptr())
    nzl = slabs[0].nzl
    for ranges, nr in (([(2, 0, 4)], 1), ([(0, -1, 4)], 1), ([(0, 0, nzl + 1)], 1), ([(0, 0, 0)], 1), ([(0, 0, 4)], 0),
                       ([(0, 0, 4)] * 17, 17)):
        assert L.lat_slab_step_ranges(hs, 2, _ranges_arg(ranges), nr, out) == 1
    assert L.lat_slab_step_ranges(hs, 9, _ranges_arg([(0, 0, 4)]), 1, out) == 1
    q, st2 = _case("lphi4", 128, 32)
    (other,) = _slabs(q, st2, 1)
    mixed = (C.c_void_p * 2)(slabs[0]._h.value, other._h.value)
    assert L.lat_slab_step_ranges(mixed, 2, _ranges_arg([(0, 0, 4)]), 1, out) == 1
    g = Lattice(p)
    whole = (C.c_void_p * 1)(g._h.value)
    assert L.lat_slab_step_ranges(whole, 1, _ranges_arg([(0, 0, 4)]), 1, out) == 8
    (small,) = _slabs(*_case("lphi4", 64, 32), 1)   # no compiled warp-tile slab kernel for N = 64
    one = (C.c_void_p * 1)(small._h.value)
    assert L.lat_slab_step_ranges(one, 1, _ranges_arg([(0, 0, 8)]), 1, C.c_void_p(small.shares.data_ptr())) == 7
