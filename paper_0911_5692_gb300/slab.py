"""One lattice split into z-slabs (the multi-GPU form of the evolution).

The paper runs one lattice on one GPU and names multi-GPU runs as future work
(Sec. IV). Here a lattice of N^3 sites is cut into contiguous z ranges, one per
slab. Per step (Sec. II.B, eq. evo with eq. scalar-evo and eq. scale):

1. halo exchange of the current ping-pong set: every slab receives the f
   plane just below its range, the two f planes just above (the second for the
   look-ahead rim of the sums) and the pi plane just above;
2. the fused step on the owned planes (CUDA, ``lat_slab_step_range``), which
   writes the slab's share of the four volume averages of the new fields;
3. an allreduce adds the shares (four FP64 numbers);
4. the FP64 scale-factor update from the total (``lat_slab_advance``),
   identical on every slab.

With ``overlap`` (slabs of at least five planes) the exchange is posted first,
the owned planes 2 .. nzl - 3 (which read no halo plane) are stepped while it is
in flight, and planes 0, 1 and nzl - 2, nzl - 1 once it has completed; the
three ranges write three shares, added on the device.

This module is host-side orchestration only: the compute of each slab runs in
the CUDA library. Halo planes move by torch.distributed point-to-point calls
(one slab per rank; NCCL between GPUs) or, for slabs held by one process, by
device copies. The exchange and allreduce logic takes any slab object with the
interface of ``SlabGPU`` (views of its stored planes, ``local_sums``,
``local_step``, ``advance``).

Stored plane p of a slab with owned range [z0, z0 + nzl) is global plane
z0 - 1 + p (mod N): p = 0 halo below, 1..nzl owned, nzl + 1, nzl + 2 halos above.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .lattice import LatticeError, _check, load_library, make_params, staggered_buffers

# array index within a ping-pong set: f_phi, f_chi, pi_phi, pi_chi
F0, F1, P0, P1 = 0, 1, 2, 3


def slab_ranges(n: int, parts: int):
    """Balanced contiguous z ranges [(z0, nzl)] of `parts` slabs; every slab
    needs at least two planes (its two lowest planes are a neighbour's halo)."""
    out = [(r * n // parts, (r + 1) * n // parts - r * n // parts) for r in range(parts)]
    if min(nz for _, nz in out) < 2:
        raise ValueError(f"{parts} slabs of a {n}^3 lattice leave a slab with fewer than 2 planes")
    return out


def halo_plan():
    """Point-to-point messages of one exchange as (direction, tag, array, k):
    'down' messages go to the slab below and carry the sender's owned plane k
    (stored plane k = 1, 2: its two lowest) into the receiver's halo above
    (stored plane nzl + k); 'up' messages go to the slab above and carry the
    sender's top owned plane (stored nzl) into the receiver's halo below
    (stored 0). f of both fields goes down twice and up once; pi goes down once."""
    msgs, tag = [], 0
    for k in (1, 2):
        for a in (F0, F1):
            msgs.append(("down", tag, a, k))
            tag += 1
    for a in (P0, P1):
        msgs.append(("down", tag, a, 1))
        tag += 1
    for a in (F0, F1):
        msgs.append(("up", tag, a, 0))
        tag += 1
    return msgs


def send_plane(msg, nzl_sender: int) -> int:
    direction, _, _, k = msg
    return k if direction == "down" else nzl_sender


def recv_plane(msg, nzl_receiver: int) -> int:
    direction, _, _, k = msg
    return nzl_receiver + k if direction == "down" else 0


class SlabGPU:
    """One z-slab on the GPU, driven through lat_slab_* (device memory from torch)."""

    def __init__(self, params: dict, z0: int, nzl: int, device: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("SlabGPU needs a CUDA device; the library has no CPU path")
        self._torch = torch
        self._L = load_library()
        self.params = dict(params)
        self.n = int(params["n"])
        self.z0, self.nzl = int(z0), int(nzl)
        self.precision = int(params.get("precision", 32))
        self.dtype = torch.float32 if self.precision == 32 else torch.float64
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        n = self.n
        self.buffers = [b.view(self.nzl + 3, n, n)
                        for b in staggered_buffers(self._L, (self.nzl + 3) * n * n, self.dtype, self.device)]
        self.shares = torch.zeros(4, dtype=torch.float64, device=self.device)
        self.range_shares = torch.zeros((3, 4), dtype=torch.float64, device=self.device)
        torch.cuda.synchronize(self.device)
        self._p = make_params(params)
        arr = (C.c_void_p * 8)(*[b.data_ptr() for b in self.buffers])
        h = C.c_void_p()
        _check(self._L.lat_slab_create(C.byref(self._p), self.z0, self.nzl, C.c_void_p(self.stream.cuda_stream), arr,
                                       C.byref(h)), "lat_slab_create")
        self._h = h
        self.step_count = 0

    def close(self):
        if getattr(self, "_h", None):
            self._L.lat_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # stored planes of the current ping-pong set
    def current_set(self) -> int:
        return self.step_count & 1

    def plane(self, a: int, p: int):
        return self.buffers[4 * self.current_set() + a][p]

    def load(self, f0, f1, pi0, pi1, t=0.0, a=1.0, ad=0.0, step=0):
        """Upload this slab's part (with its halos) of full-lattice arrays [z][y][x]
        (host arrays, or device tensors of N^3 elements, gathered on the device)."""
        torch = self._torch
        self.step_count = int(step)
        v = (C.c_double * 4)(float(t), float(a), float(ad), float(step))
        _check(self._L.lat_set_scalars(self._h, v), "lat_set_scalars")
        idx = [(self.z0 - 1 + p) % self.n for p in range(self.nzl + 3)]
        s = self.current_set()
        n = self.n
        with torch.cuda.stream(self.stream):
            for k, arr in enumerate((f0, f1, pi0, pi1)):
                if isinstance(arr, torch.Tensor) and arr.is_cuda:
                    sel = torch.tensor(idx, dtype=torch.long, device=arr.device)
                    self.buffers[4 * s + k].copy_(arr.reshape(n, n, n).index_select(0, sel))
                else:
                    part = np.ascontiguousarray(np.asarray(arr)[idx])
                    self.buffers[4 * s + k].copy_(torch.from_numpy(part).to(self.dtype))
        self.stream.synchronize()

    def owned(self):
        """Owned planes of the current set as float64 numpy arrays (f0, f1, pi0, pi1)."""
        self.stream.synchronize()
        s = self.current_set()
        return tuple(self.buffers[4 * s + k][1:self.nzl + 1].double().cpu().numpy() for k in range(4))

    def scalars(self) -> dict:
        out = (C.c_double * 8)()
        _check(self._L.lat_get_scalars(self._h, out), "lat_get_scalars")
        return {"t": out[0], "a": out[1], "ad": out[2], "step": int(out[3]), "S": list(out[4:8])}

    def local_sums(self):
        _check(self._L.lat_slab_sums(self._h, C.c_void_p(self.shares.data_ptr())), "lat_slab_sums")
        return self.shares

    def local_step(self):
        _check(self._L.lat_slab_step(self._h, C.c_void_p(self.shares.data_ptr())), "lat_slab_step")
        return self.shares

    def local_step_range(self, zfirst: int, zcount: int, slot: int):
        """Step owned planes [zfirst, zfirst + zcount); their shares go to
        range_shares[slot] (slots 0..2)."""
        _check(self._L.lat_slab_step_range(self._h, int(zfirst), int(zcount),
                                           C.c_void_p(self.range_shares[slot].data_ptr())), "lat_slab_step_range")

    def range_total(self):
        """The sum of the three range shares (on the slab's stream)."""
        with self._torch.cuda.stream(self.stream):
            self.shares.copy_(self.range_shares.sum(dim=0))
        return self.shares

    def advance(self, total, advance: bool):
        _check(self._L.lat_slab_advance(self._h, C.c_void_p(total.data_ptr()), 1 if advance else 0),
               "lat_slab_advance")
        if advance:
            self.step_count += 1

    def sync(self):
        self.stream.synchronize()


def plan_range_launches(ranges, max_slabs: int = 8, max_ranges: int = 16):
    """Cut (slab index, first plane, planes) ranges into launches of at most
    `max_slabs` slabs and `max_ranges` ranges each (the limits of
    lat_slab_step_ranges): a list of (slab indices of the launch, its ranges
    with slab indices local to the launch), covering every range once, in order
    within each launch."""
    launches, cur_slabs, cur_ranges = [], [], []
    for i, zf, zc in ranges:
        if i not in cur_slabs and len(cur_slabs) == max_slabs or len(cur_ranges) == max_ranges:
            launches.append((cur_slabs, cur_ranges))
            cur_slabs, cur_ranges = [], []
        if i not in cur_slabs:
            cur_slabs.append(i)
        cur_ranges.append((cur_slabs.index(i), zf, zc))
    if cur_ranges:
        launches.append((cur_slabs, cur_ranges))
    return launches


class LocalComm:
    """All slabs of the lattice in this process (SlabGPU on one GPU): halos by
    device copies (lat_copy_regions: every plane of the exchange in one launch
    when the slabs share a stream, else one launch per slab), the allreduce and
    the scale-factor update of every slab in one launch
    (lat_slab_advance_local)."""

    def post_exchange(self, slabs):
        self.exchange(slabs)
        return None

    def finish_exchange(self, slabs, pending):
        pass

    @staticmethod
    def _copy(dst, src, stream):
        L = load_library()
        if not dst:
            return
        nbytes = dst[0].numel() * dst[0].element_size()
        d = (C.c_void_p * len(dst))(*[t.data_ptr() for t in dst])
        q = (C.c_void_p * len(src))(*[t.data_ptr() for t in src])
        _check(L.lat_copy_regions(d, q, len(dst), nbytes, C.c_void_p(stream.cuda_stream)), "lat_copy_regions")

    def exchange(self, slabs):
        P = len(slabs)
        plans = []
        for i, s in enumerate(slabs):
            above, below = slabs[(i + 1) % P], slabs[(i - 1) % P]
            dst, src = [], []
            for msg in halo_plan():
                nb = above if msg[0] == "down" else below
                dst.append(s.plane(msg[2], recv_plane(msg, s.nzl)))
                src.append(nb.plane(msg[2], send_plane(msg, nb.nzl)))
            plans.append((dst, src))
        if all(s.stream.cuda_stream == slabs[0].stream.cuda_stream for s in slabs):
            self._copy([d for dst, _ in plans for d in dst], [q for _, src in plans for q in src], slabs[0].stream)
            return
        for i, (s, (dst, src)) in enumerate(zip(slabs, plans)):
            s.stream.wait_stream(slabs[(i + 1) % P].stream)
            s.stream.wait_stream(slabs[(i - 1) % P].stream)
            self._copy(dst, src, s.stream)
        # a slab's planes are read above before it may write them again
        for i, s in enumerate(slabs):
            s.stream.wait_stream(slabs[(i + 1) % P].stream)
            s.stream.wait_stream(slabs[(i - 1) % P].stream)

    def step_ranges(self, slabs, ranges, slot: int = 0):
        """Step owned-plane ranges (slab index, first plane, planes) of the slabs
        on the first slab's stream, in as few launches of lat_slab_step_ranges
        as its limits allow (plan_range_launches: 8 slabs, 16 ranges a launch);
        returns the device tensors holding the shares, one per launch (for
        lattice sides without a compiled warp-tile slab kernel one per range,
        stepped by lat_slab_step_range). `slot` (0 or 1) keeps the shares of two
        calls of one step apart."""
        import torch
        L = load_library()
        s0 = slabs[0]
        launches = plan_range_launches(ranges)
        need = max(len(launches), len(ranges))
        buf = getattr(self, "_shares", None)
        if buf is None or buf.device != s0.shares.device or buf.shape[1] < need:
            buf = self._shares = torch.zeros((2, need, 4), dtype=torch.float64, device=s0.shares.device)
        for s in slabs[1:]:
            s0.stream.wait_stream(s.stream)
        out = []
        for j, (ids, local) in enumerate(launches):
            hs = (C.c_void_p * len(ids))(*[slabs[i]._h.value for i in ids])
            flat = [int(v) for r in local for v in r]
            arr = (C.c_int32 * len(flat))(*flat)
            st = L.lat_slab_step_ranges(hs, len(ids), arr, len(local), C.c_void_p(buf[slot, j].data_ptr()))
            if st == 7:                  # LAT_EUNSUPPORTED: one launch per range
                out = []
                for q, (i, zf, zc) in enumerate(ranges):
                    sl = slabs[i]
                    sl.stream.wait_stream(s0.stream)
                    _check(L.lat_slab_step_range(sl._h, int(zf), int(zc), C.c_void_p(buf[slot, q].data_ptr())),
                           "lat_slab_step_range")
                    s0.stream.wait_stream(sl.stream)
                    out.append(buf[slot, q])
                break
            _check(st, "lat_slab_step_ranges")
            out.append(buf[slot, j])
        for s in slabs[1:]:
            s.stream.wait_stream(s0.stream)
        return out

    def reduce_advance(self, slabs, shares, advance: bool):
        """Add the shares (device tensors of four doubles, in the order given)
        and advance the scalars of every slab with the total, in one launch on
        the first slab's stream."""
        L = load_library()
        s0 = slabs[0]
        for s in slabs[1:]:
            s0.stream.wait_stream(s.stream)
        hs = (C.c_void_p * len(slabs))(*[s._h.value for s in slabs])
        ptrs = (C.c_void_p * len(shares))(*[t.data_ptr() for t in shares])
        _check(L.lat_slab_advance_local(hs, len(slabs), ptrs, len(shares), 1 if advance else 0),
               "lat_slab_advance_local")
        for s in slabs[1:]:
            s.stream.wait_stream(s0.stream)
        if advance:
            for s in slabs:
                s.step_count += 1

    def allreduce(self, slabs, shares):
        import torch
        s0 = slabs[0]
        for s in slabs[1:]:
            s0.stream.wait_stream(s.stream)
        with torch.cuda.stream(s0.stream):
            total = torch.stack(list(shares)).sum(dim=0)
        for s in slabs[1:]:
            s.stream.wait_stream(s0.stream)
            total.record_stream(s.stream)
        return [total] * len(slabs)


class DistComm:
    """One slab per rank of a torch.distributed group: halos by point-to-point
    messages with the ranks above and below (modulo the group size), the
    allreduce by all_reduce. Works with any backend (NCCL with device tensors,
    gloo with host tensors)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def _global(self, r):
        return self.dist.get_global_rank(self.group, r) if self.group is not None else r

    def exchange(self, slabs):
        self.finish_exchange(slabs, self.post_exchange(slabs))

    def post_exchange(self, slabs):
        """Post the halo messages of the current set (ordered after the work
        queued so far on the slab's stream); returns the requests."""
        (s,) = slabs
        dist = self.dist
        with _stream_ctx(s):
            if self.world == 1:          # the whole lattice: halos are its own planes
                for msg in halo_plan():
                    s.plane(msg[2], recv_plane(msg, s.nzl)).copy_(s.plane(msg[2], send_plane(msg, s.nzl)))
                return []
            up, down = self._global((self.rank + 1) % self.world), self._global((self.rank - 1) % self.world)
            reqs = []
            for msg in halo_plan():      # receive 'down' messages from above, 'up' ones from below
                reqs.append(dist.irecv(s.plane(msg[2], recv_plane(msg, s.nzl)), src=up if msg[0] == "down" else down,
                                       tag=msg[1], group=self.group))
            for msg in halo_plan():      # send 'down' messages below, 'up' ones above
                reqs.append(dist.isend(s.plane(msg[2], send_plane(msg, s.nzl)), dst=down if msg[0] == "down" else up,
                                       tag=msg[1], group=self.group))
            return reqs

    def finish_exchange(self, slabs, reqs):
        """Wait for the posted messages (NCCL: the slab's stream waits; gloo:
        the host waits)."""
        with _stream_ctx(slabs[0]):
            for r in reqs:
                r.wait()

    def allreduce(self, slabs, shares):
        (sh,) = shares
        with _stream_ctx(slabs[0]):
            total = sh.clone()
            self.dist.all_reduce(total, group=self.group)
        return [total]


def _stream_ctx(slab):
    import contextlib
    stream = getattr(slab, "stream", None)
    if stream is None:
        return contextlib.nullcontext()
    import torch
    return torch.cuda.stream(stream)


def overlap_ranges(nzl: int):
    """The three z ranges of one overlapped slab step as (zfirst, zcount):
    the interior, which reads no halo plane, then the two boundary pairs; None
    for slabs of fewer than five planes (stepped whole)."""
    if nzl < 5:
        return None
    return [(2, nzl - 4), (0, 2), (nzl - 2, 2)]


class SlabEvolution:
    """Steps the slabs of one lattice together: ``slabs`` are the slabs this
    process holds (all of them with LocalComm, one with DistComm). With
    ``overlap`` the interior of every slab is stepped while its halo exchange
    is in flight (overlap_ranges)."""

    def __init__(self, slabs, comm, overlap: bool = True):
        self.slabs = list(slabs)
        self.comm = comm
        self.overlap = bool(overlap) and all(overlap_ranges(s.nzl) for s in self.slabs)

    def _advance(self, shares, advance: bool):
        """Steps 3 and 4: the allreduce of the shares and the scale-factor
        update, fused into one call where the communicator offers it (slabs of
        one process)."""
        fused = getattr(self.comm, "reduce_advance", None)
        if fused is not None:
            fused(self.slabs, shares, advance)
            return
        totals = self.comm.allreduce(self.slabs, shares)
        for s, t in zip(self.slabs, totals):
            s.advance(t, advance)

    def prepare(self):
        """Coefficients of the first step from the current fields (after a load)."""
        self.comm.exchange(self.slabs)
        self._advance([s.local_sums() for s in self.slabs], False)

    def step(self, n_steps: int = 1):
        fused = hasattr(self.comm, "reduce_advance")
        together = getattr(self.comm, "step_ranges", None)   # every slab of the process in one launch
        for _ in range(int(n_steps)):
            if self.overlap:
                pending = self.comm.post_exchange(self.slabs)
                if together is not None:
                    shares = together(self.slabs, [(i, *overlap_ranges(s.nzl)[0]) for i, s in enumerate(self.slabs)], 0)
                else:
                    for s in self.slabs:
                        zf, zc = overlap_ranges(s.nzl)[0]
                        s.local_step_range(zf, zc, 0)
                self.comm.finish_exchange(self.slabs, pending)
                if together is not None:
                    shares = shares + together(self.slabs, [(i, zf, zc) for i, s in enumerate(self.slabs)
                                                            for zf, zc in overlap_ranges(s.nzl)[1:]], 1)
                else:
                    for s in self.slabs:
                        for slot, (zf, zc) in enumerate(overlap_ranges(s.nzl)[1:], start=1):
                            s.local_step_range(zf, zc, slot)
                    if fused:    # the three range shares of every slab go to the fused sum as they are
                        shares = [s.range_shares[k] for s in self.slabs for k in range(3)]
                    else:
                        shares = [s.range_total() for s in self.slabs]
            else:
                self.comm.exchange(self.slabs)
                if together is not None:
                    shares = together(self.slabs, [(i, 0, s.nzl) for i, s in enumerate(self.slabs)], 0)
                else:
                    shares = [s.local_step() for s in self.slabs]
            self._advance(shares, True)

    def gather(self):
        """Full-lattice arrays (f0, f1, pi0, pi1) from the slabs of this process
        (LocalComm: all of them) in z order."""
        parts = [s.owned() for s in sorted(self.slabs, key=lambda s: s.z0)]
        return tuple(np.concatenate([p[k] for p in parts], axis=0) for k in range(4))


__all__ = ["slab_ranges", "halo_plan", "send_plane", "recv_plane", "overlap_ranges", "plan_range_launches", "SlabGPU",
           "LocalComm", "DistComm", "SlabEvolution", "LatticeError"]
