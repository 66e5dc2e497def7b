"""Z-slab decomposition on CPU ranks (gloo): the exchange plan, the
point-to-point halo traffic and the allreduce of paper_0911_5692_gb300.slab,
driven by world_size 2 and 3 process groups, against the single-domain FP64
oracle.

The slabs here compute with a plain numpy step written in this file (the
product's slabs compute in CUDA, tested in test_gpu_slab.py); the scalar
coefficients come from the oracle. What is under test is the host-side
orchestration: which planes go where, in which order, and how the shares are
added before the scale-factor update.
"""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle.oracle import Oracle
from paper_0911_5692_gb300.slab import (DistComm, SlabEvolution, halo_plan, overlap_ranges, recv_plane, send_plane,
                                        slab_ranges)
from paper_0911_5692_gb300.workloads import lphi4, m2phi2, random_state

N = 16
SCAL = dict(t=0.0, a=1.05, ad=0.4, step=0)


def _case(model):
    if model == "lphi4":
        p = lphi4(N, precision=64)
        st = random_state(N, 5, 64, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-3), pi_mean=(0.5, 0.0), pi_amp=(1e-3, 1e-3))
    else:
        p = m2phi2(N, precision=64)
        st = random_state(N, 6, 64, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-4), pi_mean=(0.3, 0.0), pi_amp=(1e-3, 1e-2))
    return p, st


def _lap(f, dx):
    """7-point Laplacian in x, y (periodic) of planes f[p] and z from p-1, p+1."""
    out = np.zeros_like(f[1:-1])
    c = f[1:-1]
    out += (np.roll(c, 1, axis=2) - c) + (np.roll(c, -1, axis=2) - c)
    out += (np.roll(c, 1, axis=1) - c) + (np.roll(c, -1, axis=1) - c)
    out += (f[:-2] - c) + (f[2:] - c)
    return out / (dx * dx)


class NumpySlab:
    """A slab computed with numpy on host tensors (the interface of SlabGPU)."""

    def __init__(self, params, z0, nzl):
        self.p = dict(params)
        self.n = params["n"]
        self.z0, self.nzl = z0, nzl
        self.dx = params["L"] / self.n
        self.dt = params["dt"]
        self.buffers = [torch.zeros((nzl + 3, self.n, self.n), dtype=torch.float64) for _ in range(8)]
        self.range_shares = torch.zeros((3, 4), dtype=torch.float64)
        self.step_count = 0
        self.orc = Oracle(params)
        d = self.orc.derived()
        self.beta = d["beta"]
        self.cdom0, self.pdom, self.kappa0, self.pint = d["cdom0"], d["pdom"], d["kappa0"], d["pint"]
        self.sc = {}

    def current_set(self):
        return self.step_count & 1

    def plane(self, a, p):
        return self.buffers[4 * self.current_set() + a][p]

    def load(self, f0, f1, pi0, pi1, t, a, ad, step):
        self.step_count = step
        self.sc = dict(t=t, a=a, ad=ad, step=step)
        idx = [(self.z0 - 1 + q) % self.n for q in range(self.nzl + 3)]
        s = self.current_set()
        for k, arr in enumerate((f0, f1, pi0, pi1)):
            self.buffers[4 * s + k].copy_(torch.from_numpy(np.ascontiguousarray(arr[idx])))

    def owned(self):
        s = self.current_set()
        return tuple(self.buffers[4 * s + k][1:self.nzl + 1].numpy().copy() for k in range(4))

    def _shares(self, g0, g1, gz0, gz1):
        """Shares of the four averages over owned planes g (nzl planes) with the
        plane above them gz (for the z differences)."""
        n3 = float(self.n) ** 3
        up0 = np.concatenate([g0[1:], gz0[None]], axis=0)
        up1 = np.concatenate([g1[1:], gz1[None]], axis=0)
        s = []
        for g, up in ((g0, up0), (g1, up1)):
            d = (np.roll(g, -1, axis=2) - g) ** 2 + (np.roll(g, -1, axis=1) - g) ** 2 + (up - g) ** 2
            s.append(d.sum() / (self.dx * self.dx) / n3)
        s.append((g0 ** self.beta / self.beta).sum() / n3)
        s.append((0.5 * g0 * g0 * g1 * g1).sum() / n3)
        return torch.tensor(s, dtype=torch.float64)

    def local_sums(self):
        s = self.current_set()
        f0 = self.buffers[4 * s + 0].numpy()
        f1 = self.buffers[4 * s + 1].numpy()
        return self._shares(f0[1:self.nzl + 1], f1[1:self.nzl + 1], f0[self.nzl + 1], f1[self.nzl + 1])

    def local_step(self):
        s = self.current_set()
        co = self.co
        f0 = self.buffers[4 * s + 0].numpy()
        f1 = self.buffers[4 * s + 1].numpy()
        p0 = self.buffers[4 * s + 2].numpy()
        p1 = self.buffers[4 * s + 3].numpy()
        dt = self.dt
        # kick and drift of the owned planes and of the plane above them
        # (stored 1 .. nzl + 1; the last one only for the z differences)
        c0, c1 = f0[1:self.nzl + 2], f1[1:self.nzl + 2]
        l0, l1 = _lap(f0[0:self.nzl + 3], self.dx), _lap(f1[0:self.nzl + 3], self.dx)
        dv0 = co["cdom"] * c0 ** (self.beta - 1) + co["kappa"] * c0 * c1 * c1
        dv1 = co["kappa"] * c0 * c0 * c1
        q0 = p0[1:self.nzl + 2] + dt * (co["cL"] * l0 + co["cF"] * c0 - dv0)
        q1 = p1[1:self.nzl + 2] + dt * (co["cL"] * l1 + co["cF"] * c1 - dv1)
        g0, g1 = c0 + dt * q0, c1 + dt * q1
        o = 1 - s
        self.buffers[4 * o + 0][1:self.nzl + 1] = torch.from_numpy(g0[:-1].copy())
        self.buffers[4 * o + 1][1:self.nzl + 1] = torch.from_numpy(g1[:-1].copy())
        self.buffers[4 * o + 2][1:self.nzl + 1] = torch.from_numpy(q0[:-1].copy())
        self.buffers[4 * o + 3][1:self.nzl + 1] = torch.from_numpy(q1[:-1].copy())
        return self._shares(g0[:-1], g1[:-1], g0[-1], g1[-1])

    def local_step_range(self, zfirst, zcount, slot):
        """Step owned planes [zfirst, zfirst + zcount) from a copy of the current
        set in which every stored plane outside the range's window (stored
        zfirst .. zfirst + zcount + 2) is NaN, so a read outside the window
        shows in the result."""
        s = self.current_set()
        lo, hi = zfirst, zfirst + zcount + 3          # stored window [lo, hi)
        win = []
        for k in range(4):
            a = self.buffers[4 * s + k].numpy().copy()
            a[:lo] = np.nan
            a[hi:] = np.nan
            win.append(a)
        f0, f1, p0, p1 = win
        co, dt = self.co, self.dt
        c0, c1 = f0[lo + 1:hi - 1], f1[lo + 1:hi - 1]            # planes zfirst .. zfirst + zcount
        l0, l1 = _lap(f0[lo:hi], self.dx), _lap(f1[lo:hi], self.dx)
        dv0 = co["cdom"] * c0 ** (self.beta - 1) + co["kappa"] * c0 * c1 * c1
        dv1 = co["kappa"] * c0 * c0 * c1
        q0 = p0[lo + 1:hi - 1] + dt * (co["cL"] * l0 + co["cF"] * c0 - dv0)
        q1 = p1[lo + 1:hi - 1] + dt * (co["cL"] * l1 + co["cF"] * c1 - dv1)
        g0, g1 = c0 + dt * q0, c1 + dt * q1
        o = 1 - s
        for k, v in enumerate((g0, g1, q0, q1)):
            self.buffers[4 * o + k][lo + 1:hi - 2] = torch.from_numpy(v[:-1].copy())
        self.range_shares[slot] = self._shares(g0[:-1], g1[:-1], g0[-1], g1[-1])

    def range_total(self):
        return self.range_shares.sum(dim=0)

    def advance(self, total, advance):
        S = total.numpy().tolist()
        sc = self.sc
        if advance:
            if self.p["expansion"]:
                sc["a"] = sc["a"] + self.dt * (self.co["y"] - sc["ad"])
                sc["ad"] = self.co["y"] - sc["ad"]
            sc["t"] += self.dt
            sc["step"] += 1
            self.step_count += 1
        sc["S"] = S
        self.co = self.orc.step_coefs(sc["a"], sc["ad"], S)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class SlowComm(DistComm):
    """DistComm as a slow network: post_exchange fills the receiving halo planes
    with NaN and receives into side buffers, which finish_exchange copies into
    the halos after the messages have landed. A step that reads a halo between
    the two calls reads NaN, whatever the timing of the messages."""

    def post_exchange(self, slabs):
        (s,) = slabs
        if self.world == 1:
            return super().post_exchange(slabs)
        up, down = self._global((self.rank + 1) % self.world), self._global((self.rank - 1) % self.world)
        reqs, side = [], []
        for msg in halo_plan():
            dst = s.plane(msg[2], recv_plane(msg, s.nzl))
            buf = torch.empty_like(dst)
            side.append((dst, buf))
            reqs.append(self.dist.irecv(buf, src=up if msg[0] == "down" else down, tag=msg[1], group=self.group))
        for msg in halo_plan():
            reqs.append(self.dist.isend(s.plane(msg[2], send_plane(msg, s.nzl)), dst=down if msg[0] == "down" else up,
                                        tag=msg[1], group=self.group))
        for dst, _ in side:
            dst.fill_(float("nan"))
        return reqs, side

    def finish_exchange(self, slabs, pending):
        if self.world == 1:
            return super().finish_exchange(slabs, pending)
        reqs, side = pending
        for r in reqs:
            r.wait()
        for dst, buf in side:
            dst.copy_(buf)


def _worker(rank, world, port, model, steps, out_dir, overlap=False):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, st = _case(model)
        z0, nzl = slab_ranges(N, world)[rank]
        s = NumpySlab(p, z0, nzl)
        s.load(*st, **SCAL)
        ev = SlabEvolution([s], SlowComm() if overlap else DistComm(), overlap=overlap)
        assert ev.overlap == (overlap and nzl >= 5)
        ev.prepare()
        ev.step(steps)
        parts = [None] * world
        dist.all_gather_object(parts, (z0, s.owned(), s.sc))
        if rank == 0:
            np.save(os.path.join(out_dir, "result.npy"), np.array(parts, dtype=object), allow_pickle=True)
    finally:
        dist.destroy_process_group()


def test_halo_plan_covers_every_halo_once():
    msgs = halo_plan()
    assert len({m[1] for m in msgs}) == len(msgs)
    nzl = 5
    recv = sorted((m[2], recv_plane(m, nzl)) for m in msgs)
    assert recv == sorted([(0, 0), (1, 0), (0, 6), (1, 6), (0, 7), (1, 7), (2, 6), (3, 6)])
    # the sender's planes are owned ones
    for m in msgs:
        assert 1 <= send_plane(m, nzl) <= nzl


def test_slab_ranges():
    assert slab_ranges(16, 3) == [(0, 5), (5, 5), (10, 6)]
    with pytest.raises(ValueError):
        slab_ranges(8, 5)


def test_overlap_ranges():
    assert overlap_ranges(4) is None
    assert overlap_ranges(5) == [(2, 1), (0, 2), (3, 2)]
    for nzl in range(5, 40):
        covered = sorted(z for zf, zc in overlap_ranges(nzl) for z in range(zf, zf + zc))
        assert covered == list(range(nzl))       # every owned plane exactly once
        zf, zc = overlap_ranges(nzl)[0]
        # the interior's window (stored zf .. zf + zc + 2) holds no halo plane
        assert zf >= 1 and zf + zc + 2 <= nzl


@pytest.mark.parametrize("world,model,overlap", [(1, "lphi4", False), (2, "lphi4", False), (3, "m2phi2", False),
                                                 (4, "lphi4", False), (1, "lphi4", True), (2, "m2phi2", True),
                                                 (3, "lphi4", True)])
def test_distributed_slabs_match_single_domain_oracle(tmp_path, world, model, overlap):
    """overlap: the exchange is posted, the interior stepped from a window that
    holds no halo, the exchange finished, the boundary pairs stepped; the
    receiving halos are NaN from the post until finish_exchange (SlowComm), so a
    range stepped out of order would fail."""
    steps = 7
    mp.start_processes(_worker, args=(world, _free_port(), model, steps, str(tmp_path), overlap), nprocs=world,
                       start_method="spawn", join=True)
    parts = np.load(os.path.join(tmp_path, "result.npy"), allow_pickle=True)
    parts = sorted(parts, key=lambda r: r[0])
    got = [np.concatenate([r[1][k] for r in parts], axis=0) for k in range(4)]
    p, st = _case(model)
    o = Oracle(p)
    o.set_state(*st, **SCAL)
    o.step(steps)
    for a, b in zip(got, o.get_state()):
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
    for r in parts:
        sc = r[2]
        assert sc["step"] == steps
        assert abs(sc["a"] - o.scalars()["a"]) <= 1e-14 * abs(o.scalars()["a"])
        for k in range(4):
            assert abs(sc["S"][k] - o.scalars()["S"][k]) <= 1e-12 * abs(o.scalars()["S"][k])


class NumpyLocalComm:
    """The one-process communicator's interface (slabs held together, as
    LocalComm offers it for slabs on one GPU) over NumpySlab: halos by copies,
    every slab's ranges stepped by one call (step_ranges, one summed share) and
    one call that adds the shares and advances every slab (reduce_advance).
    post_exchange leaves the receiving halos NaN until finish_exchange, so a
    range stepped before the exchange has landed and reading a halo fails."""

    def _plan(self, slabs):
        P = len(slabs)
        out = []
        for i, s in enumerate(slabs):
            above, below = slabs[(i + 1) % P], slabs[(i - 1) % P]
            for msg in halo_plan():
                nb = above if msg[0] == "down" else below
                out.append((s.plane(msg[2], recv_plane(msg, s.nzl)), nb.plane(msg[2], send_plane(msg, nb.nzl)).clone()))
        return out

    def exchange(self, slabs):
        for dst, src in self._plan(slabs):
            dst.copy_(src)

    def post_exchange(self, slabs):
        plan = self._plan(slabs)
        for dst, _ in plan:
            dst.fill_(float("nan"))
        return plan

    def finish_exchange(self, slabs, pending):
        for dst, src in pending:
            dst.copy_(src)

    def allreduce(self, slabs, shares):
        total = sum(shares)
        return [total] * len(slabs)

    def step_ranges(self, slabs, ranges, slot=0):
        used = {}
        total = torch.zeros(4, dtype=torch.float64)
        for i, zf, zc in ranges:
            j = used.get(i, 0)
            used[i] = j + 1
            slabs[i].local_step_range(zf, zc, j)
            total += slabs[i].range_shares[j]
        return [total]

    def reduce_advance(self, slabs, shares, advance):
        total = sum(shares)
        for s in slabs:
            s.advance(total, advance)


@pytest.mark.parametrize("parts,model,overlap", [(1, "lphi4", False), (3, "m2phi2", False), (4, "lphi4", False),
                                                 (2, "lphi4", True), (3, "m2phi2", True)])
def test_slabs_of_one_process_stepped_together(parts, model, overlap):
    """SlabEvolution with a communicator that steps every slab's ranges in one
    call and advances every slab in one call (the path slabs on one GPU take):
    the plain schedule (all owned planes at once) and the overlapped one (the
    interiors while the halos are NaN, then the boundary pairs) against the
    single-domain oracle."""
    steps = 6
    p, st = _case(model)
    slabs = []
    for z0, nzl in slab_ranges(N, parts):
        s = NumpySlab(p, z0, nzl)
        s.load(*st, **SCAL)
        slabs.append(s)
    ev = SlabEvolution(slabs, NumpyLocalComm(), overlap=overlap)
    assert ev.overlap == (overlap and min(s.nzl for s in slabs) >= 5)
    ev.prepare()
    ev.step(steps)
    got = [np.concatenate([s.owned()[k] for s in slabs], axis=0) for k in range(4)]
    o = Oracle(p)
    o.set_state(*st, **SCAL)
    o.step(steps)
    for a, b in zip(got, o.get_state()):
        assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
    for s in slabs:
        assert s.sc["step"] == steps and s.step_count == steps
        assert abs(s.sc["a"] - o.scalars()["a"]) <= 1e-14 * abs(o.scalars()["a"])


def test_plan_range_launches():
    """Ranges of many slabs cut into launches within lat_slab_step_ranges'
    limits (8 slabs, 16 ranges): every range once, in order, each launch's
    local slab indices mapping back to the slabs of its ranges."""
    from paper_0911_5692_gb300.slab import plan_range_launches
    cases = [
        [(i, 0, 10) for i in range(4)],                                  # one launch
        [(i, 0, 10) for i in range(20)],                                 # 20 slabs: 8 + 8 + 4
        [(i, zf, 2) for i in range(12) for zf in (0, 8)],                # two ranges per slab
        [(i % 3, 2 * i, 1) for i in range(40)],                          # 3 slabs, 40 ranges
    ]
    for ranges in cases:
        launches = plan_range_launches(ranges)
        back = []
        for ids, local in launches:
            assert 1 <= len(ids) <= 8 and 1 <= len(local) <= 16
            assert len(set(ids)) == len(ids)
            assert {r[0] for r in local} == set(range(len(ids)))
            back += [(ids[k], zf, zc) for k, zf, zc in local]
        assert back == ranges
    assert len(plan_range_launches([(i, 0, 10) for i in range(20)])) == 3
    assert plan_range_launches([]) == []
