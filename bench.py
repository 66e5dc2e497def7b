#!/usr/bin/env python3
"""Throughput benchmark of the fused staggered-leapfrog step.

`python bench.py --gpus N --steps K --warmup W` evolves one lattice per GPU
(replicas, weak scaling: each rank runs its own independent lattice) for W
untimed and K timed steps and prints one JSON line on rank 0:
site-updates/s over all ranks, the step kernel's achieved HBM bandwidth against
the measured copy peak, an end-to-end figure through the C ABI with host
buffers, the FP64 oracle timed on the host cores, and SM clocks sampled during
the timed region.

`--impl reference` times the FP64 CPU oracle instead (rank 0 only), each step a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "lattice site-updates/s (2 fields, FP32) and % HBM roofline; adjoint/forward cost"
UNIT = "site-updates/s"
L2_BYTES = 129e6
FALLBACK_HBM_GBS = 6800.0
# GB300's nominal HBM3e bandwidth (8 TB/s class), reported beside the measured copy rate
NOMINAL_HBM_GBS = 8000.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="lphi4_512_fp32")
    ap.add_argument("--variant", type=int, default=0,
                    help="step kernel: 0 autotuned, 2 plane ring over full rows, 4 plane ring over x tiles, "
                         "5 x tiles one warp wide")
    ap.add_argument("--slabs", type=int, default=0,
                    help="z-slab mode: one lattice of the workload cut into z-slabs (phi stored whole); one rank: "
                         "this many slabs on its GPU; under torchrun: one slab per rank (NCCL halos and sums, the "
                         "interior stepped while the halos are in flight); strong scaling")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default kernel shape instead of autotuning it (lat_tune) before timing")
    ap.add_argument("--stencil", type=int, choices=[7, 27], default=7,
                    help="Laplacian: 7-point, or the paper's 27-point stencil (Sec. II.C)")
    ap.add_argument("--expansion", type=int, choices=[1, 2], default=1,
                    help="scale-factor update: 1 eq. scale, 2 the L = 1/H form (one more pass per step)")
    ap.add_argument("--ty", type=int, default=0)
    ap.add_argument("--zr", type=int, default=0)
    ap.add_argument("--depth", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the adjoint, ensemble and FP32-vs-FP64 measurements")
    return ap.parse_args()


def workload(name):
    from paper_0911_5692_gb300.workloads import WORKLOADS
    w = WORKLOADS[name]
    p = dict(w["params"])
    return p


def model_name(p):
    return "lphi4" if p["model"] == 0 else "m2phi2"


def config_of(name, p, world):
    n = p["n"]
    esize = 4 if p["precision"] == 32 else 8
    state = 8 * n ** 3 * esize
    return {"workload": name, "potential": model_name(p), "stencil": int(p.get("stencil", 7)), "n": n, "sites": n ** 3,
            "precision": p["precision"],
            "storage": "phi as an FP64 homogeneous mode + fluctuation arrays" if p.get("split") else "fields whole",
            "expansion": bool(p["expansion"]),
            "scale_factor": {0: "static", 1: "eq. scale", 2: "L = 1/H form"}[int(p["expansion"])],
            "global_batch": world, "lattices_per_gpu": 1,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": f"inputs larger than L2: {state / 2 / 1e6:.0f} MB read + {state / 2 / 1e6:.0f} MB written per step"
                  if state / 2 > L2_BYTES else "state fits in L2"}


STEP_KERNEL_SOURCES = {
    7: ("lat_step_fast.cu", "lat_step_march.cu", "lat_march.cuh", "lat_common.cuh", "lat_pairs.cuh", "lat_async.cuh",
        "lat_kernels.h", "lat_site.cuh"),
    27: ("lat_step27.cu", "lat_march.cuh", "lat_common.cuh", "lat_pairs.cuh", "lat_async.cuh", "lat_kernels.h",
         "lat_site.cuh"),
}


VARIANT_SOURCES = {(7, 4): ("lat_step_xt.cu",), (7, 5): ("lat_step_xw.cu", "lat_xw.cuh", "lat_layout.cuh"),
                   (27, 5): ("lat_step27w.cu",)}


def kernel_source_hash(stencil=7, variant=2):
    """Hash of the sources the fused step kernels of a stencil (and, for the
    x-tiled variants 4 and 5, their own files) are built from: a recorded
    DRAM-traffic figure is valid only for these exact sources."""
    d = os.path.join(ROOT, "paper_0911_5692_gb300", "csrc")
    h = hashlib.sha256()
    files = STEP_KERNEL_SOURCES[stencil] + VARIANT_SOURCES.get((stencil, variant), ())
    for f in files:
        h.update(f.encode())
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def traffic_record(name, variant, stencil=7, depth=None):
    """DRAM bytes per launch of the step kernel from a committed ncu summary, if it
    was taken on the current kernel sources with the same shape; else None."""
    path = os.path.join(ROOT, "profiles", "step_traffic.json")
    try:
        recs = json.load(open(path))
    except Exception:
        return None
    hsh = kernel_source_hash(stencil, variant)
    for r in recs.get("records", []):
        if (r.get("kernel_hash") == hsh and r.get("workload") == name and r.get("variant") == variant
                and r.get("stencil", 7) == stencil and r.get("depth") == depth):
            return r.get("dram_bytes_per_launch")
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu_id)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1])); mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model():
    """The host CPU's model name (lscpu), else the machine type."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


def cpu_baseline(p, seconds, one_thread_seconds=6.0):
    """The FP64 oracle as it stands, on this host's cores, on a bounded sample of
    the workload: steps of the full lattice from a seeded synthetic state until
    `seconds` have passed, with OpenMP over all cores; then the same on one
    thread for `one_thread_seconds`."""
    import numpy as np
    from oracle.oracle import Oracle, set_threads
    from paper_0911_5692_gb300.workloads import random_state
    n = p["n"]
    st = random_state(n, 1, precision=p["precision"], f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-4), pi_mean=(0.3, 0.0),
                      pi_amp=(1e-3, 1e-2))
    o = Oracle(p)
    o.set_state(*st, t=0.0, a=1.0, ad=0.5)
    del st

    def timed(limit):
        o.step(1)
        steps = 0
        t0 = time.perf_counter()
        while True:
            o.step(1)
            steps += 1
            el = time.perf_counter() - t0
            if el >= limit:
                return steps, el

    cores = os.cpu_count()
    all_threads = set_threads(cores)
    steps, el = timed(seconds)
    set_threads(1)
    steps1, el1 = timed(one_thread_seconds)
    set_threads(all_threads)
    return {"value": n ** 3 * steps / el, "unit": UNIT, "cores": all_threads, "kind": "oracle",
            "sample": f"{steps} FP64 oracle steps of the full {n}^3 {model_name(p)} lattice from a seeded "
                      f"synthetic state ({el:.1f} s, OpenMP over {all_threads} host threads)",
            "cpu_model": cpu_model(),
            "one_thread": {"value": n ** 3 * steps1 / el1, "unit": UNIT, "cores": 1,
                           "sample": f"{steps1} steps of the same lattice on one thread ({el1:.1f} s)"}}


def state_error(x, ref, stride=1):
    """FP32 against FP64: normwise max|x - ref| / max|ref| per array of (f_phi,
    f_chi, pi_phi, pi_chi), and against the fluctuation part of the inflaton's
    arrays (max|x - ref| / max|ref - <ref>|), on every stride-th site per axis."""
    import numpy as np
    names = ("f_phi", "f_chi", "pi_phi", "pi_chi")
    err = {}
    for k, (a, b) in enumerate(zip(x, ref)):
        a, b = a[::stride, ::stride, ::stride], b[::stride, ::stride, ::stride]
        diff = float(np.max(np.abs(a - b)))
        err[names[k]] = diff / max(float(np.max(np.abs(b))), 1e-300)
        if k in (0, 2):
            err[names[k] + "_fluct"] = diff / max(float(np.max(np.abs(b - b.mean()))), 1e-300)
    return err


def fp64_twin(p, local):
    """An FP64 lattice of the same parameters, phi stored whole, initialised from
    the same seed by its own pipeline: the reference of the FP32 errors."""
    from paper_0911_5692_gb300 import Lattice
    g = Lattice(dict(p, precision=64, split=0), device=local)
    g.init_fields()
    return g


def measure_adjoint(local, name="lphi4_128_fp32", n=None, steps=None, fp64=False):
    """Cost of the reverse-mode derivative on the 128^3 lambda phi^4 workload:
    J = <chi^2> after its 2000 steps and dJ/d(f, pi, g^2) by lat_adjoint
    (sqrt(n) checkpointing), against the plain forward evolution of the same
    steps. ratio_total = adjoint call / forward; ratio_backward = (adjoint call -
    forward) / forward, the recomputation plus reverse sweep per forward step.
    n, steps: the same model on another lattice side (dt = dx / 20) and step
    count (at 128^3 part of the state stays in L2)."""
    import torch
    from paper_0911_5692_gb300 import Lattice
    from paper_0911_5692_gb300.workloads import WORKLOADS
    w = WORKLOADS[name]
    p, steps = dict(w["params"]), int(steps or w["steps"])
    if n:
        p["n"] = int(n)
        p["dt"] = p["L"] / n / 20
        name = f"{name.split('_')[0]}_{n}_fp{p['precision']}"
    g = Lattice(p, device=local)
    g.init_fields()
    g.sync()
    blob = g.save_checkpoint()
    g.evolve(64)
    g.sync()
    res = {}
    for rep in range(2):
        g.load_checkpoint(blob)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.evolve(steps)
        g.sync()
        tf = time.perf_counter() - t0
        g.load_checkpoint(blob)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        J, _, _, dg2 = g.adjoint(steps)
        torch.cuda.synchronize()
        ta = time.perf_counter() - t0
        K = int(math.ceil(math.sqrt(steps)))
        # the reverse steps alone: the call less its forward pass and less the
        # recomputation of every segment but its last step (derived, not timed apart)
        rev = ta - tf - tf * (1.0 - 1.0 / K)
        res = {"workload": name, "n": p["n"], "steps": steps, "forward_s": tf, "adjoint_s": ta,
               "ratio_total": ta / tf, "ratio_backward": (ta - tf) / tf, "ratio_reverse_step": rev / tf,
               "J": J, "dJ_dg2": dg2, "checkpoint_every": K,
               "definitions": "ratio_total: the whole gradient (forward pass with checkpoints, recomputation, "
                              "reverse sweep) per forward evolution; ratio_backward: recomputation + reverse "
                              "sweep per forward step; ratio_reverse_step: one reverse step per forward step, "
                              "derived as (adjoint - forward - (1 - 1/K) forward) / forward",
               "timing": "wall clock, second of two runs"}
    if fp64:
        # the same gradient from the same FP32-representable start with FP64 fields
        g.load_checkpoint(blob)
        J32, df32, dp32, dg32 = g.adjoint(steps)
        g.load_checkpoint(blob)
        st = g.get_state()
        sc = g.scalars()
        g.close()
        h = Lattice(dict(p, precision=64), device=local)
        h.set_state(*st, t=sc["t"], a=sc["a"], ad=sc["ad"], step=sc["step"])
        J64, df64, dp64, dg64 = h.adjoint(steps)
        import numpy as np
        err = {"J_rel": abs(J32 / J64 - 1), "dJ_dg2_rel": abs(dg32 / dg64 - 1)}
        for i, f in enumerate(("phi", "chi")):
            for nm, a, b in (("dJ_df", df32, df64), ("dJ_dpi", dp32, dp64)):
                a_, b_ = a[i].double().cpu().numpy(), b[i].cpu().numpy()
                err[f"{nm}_{f}"] = float(np.max(np.abs(a_ - b_)) / max(float(np.max(np.abs(b_))), 1e-300))
        res["fp64_error"] = dict(err, against="FP64 gradient on the GPU from the same start (the FP64 path is "
                                               "pinned to the oracle's adjoint), normwise per array")
        h.close()
    return res


def measure_ensemble(local, steps=200):
    """The 64-member ensemble (N in 32, 48, 64, 96; g^2/lambda log-uniform in
    [50, 500]; FP32, phi stored split) in one persistent launch per evolve call,
    after autotuning; and the FP32 error against the same ensemble in FP64
    (largest per-member normwise error) after the timed steps."""
    import torch
    from paper_0911_5692_gb300 import Ensemble
    from paper_0911_5692_gb300.workloads import ensemble_64
    members = ensemble_64(split=1)
    ens = Ensemble(members, device=local)
    ens.init_fields()
    ens.tune(20)
    ens.evolve(5)
    ens.sync()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record(ens.stream)
    ens.evolve(steps)
    e.record(ens.stream)
    ens.sync()
    ms = s.elapsed_time(e) / steps
    info = ens.info()
    su = info["sites"] / (ms / 1e3)
    peaks = measured_peaks()
    peak = float(peaks["hbm_gbs"]) if peaks and peaks.get("hbm_gbs") else FALLBACK_HBM_GBS
    ref = Ensemble(ensemble_64(precision=64), device=local)
    ref.init_fields()
    ref.evolve(5 + steps)
    ref.sync()
    worst = {}
    for i in range(len(members)):
        err = state_error(ens.member(i).get_state_exact(), ref.member(i).get_state())
        for k, v in err.items():
            worst[k] = max(worst.get(k, 0.0), v)
    ref.close()
    return {"workload": "ensemble_64", "members": info["members"], "sites": info["sites"], "steps": steps,
            "ms_per_step": ms, "value": su, "unit": UNIT, "hbm_frac": su * 32 / 1e9 / peak,
            "storage": "phi split (FP64 homogeneous mode + FP32 fluctuations)",
            "launch": {"blocks": info["blocks"], "threads": info["threads"], "graph": bool(info["graph"]),
                       "launches_per_evolve": info["launches"],
                       "ty_by_side": {str(p["n"]): t for p, t in zip(members, info["ty"])},
                       "depth": info["depth"], "tile_cap": info["tile_cap"],
                       "tuned_over": "block size x tile-height cap x prefetch depth (lat_batch_tune)"},
            "fp64_error": dict(worst, steps=steps + 5, against="the same 64 members in FP64 (phi whole), same "
                                                                  "seeds; largest per-member normwise error")}


def measure_slabs(local, parts=4, steps=200):
    """One 512^3 FP32 lambda phi^4 lattice (phi stored whole) cut into `parts`
    z-slabs on one GPU, all on one stream: the halo planes of all slabs in one
    copy launch, the owned planes of all slabs in one step launch, the shares
    added and every slab's scale factor advanced in one launch; two steps (one
    per ping-pong parity) captured in a CUDA graph and replayed. Both schedules
    (plain: exchange, then each slab whole; overlap: each slab's interior,
    exchange, boundary pairs) against the same lattice stepped whole. On one GPU
    nothing overlaps; the line measures what the slab form costs in extra
    launches and copies."""
    import numpy as np
    import torch
    from paper_0911_5692_gb300 import Lattice
    from paper_0911_5692_gb300.slab import LocalComm, SlabEvolution, SlabGPU, slab_ranges
    from paper_0911_5692_gb300.workloads import lphi4
    p = lphi4(512, precision=32)
    n = p["n"]
    lat = Lattice(p, device=local)
    lat.init_fields()
    sc0 = lat.scalars()
    arrs = [lat.get_state_device(f, w) for w in (0, 1) for f in (0, 1)]   # f0, f1, pi0, pi1

    def timed(run, k):
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        s.record(stream)
        for _ in range(k):
            run()
        e.record(stream)
        torch.cuda.synchronize()
        return s.elapsed_time(e)

    stream = lat.stream
    lat.evolve(32)
    whole_ms = timed(lambda: lat.evolve(steps), 1) / steps
    out = {"workload": "lphi4_512_fp32 (phi whole)", "slabs": parts, "steps": steps, "whole_ms_per_step": whole_ms}
    stream = torch.cuda.Stream(device=local)
    slabs = [SlabGPU(p, z0, nzl, device=local, stream=stream) for z0, nzl in slab_ranges(n, parts)]
    for overlap in (False, True):
        for sl in slabs:
            sl.load(*arrs, t=sc0["t"], a=sc0["a"], ad=sc0["ad"], step=sc0["step"])
        ev = SlabEvolution(slabs, LocalComm(), overlap=overlap)
        ev.prepare()
        ev.step(2)                      # uncaptured: kernel configuration, shared-memory opt-ins
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            ev.step(2)
        for sl in slabs:                # the capture ran nothing: the host step counts go back
            sl.step_count -= 2

        def replay():
            with torch.cuda.stream(stream):     # the graph runs on the stream the events are recorded on
                g.replay()
            for sl in slabs:
                sl.step_count += 2
        replay()
        ms = timed(replay, steps // 2) / (2 * (steps // 2))
        for sl in slabs:
            assert np.isfinite(sl.scalars()["S"]).all()
        out["overlap" if overlap else "plain"] = {"ms_per_step": ms, "value": n ** 3 / (ms / 1e3), "unit": UNIT,
                                                  "over_whole": ms / whole_ms,
                                                  "launches_per_step": (2 if overlap else 1) + 2}
        del g
    for sl in slabs:
        sl.close()
    lat.close()
    return out


def measure_stencil27(local, names=("m2phi2_256_fp32", "lphi4_512_fp32"), steps=100):
    """The step with the paper's 27-point Laplacian (Sec. II.C) on the same
    workloads; m2phi2 at 256^3 in FP32 is the configuration of the paper's own
    timing (0.022 s per step on a GTX 260)."""
    import torch
    from paper_0911_5692_gb300 import Lattice
    peaks = measured_peaks()
    peak = float(peaks["hbm_gbs"]) if peaks and peaks.get("hbm_gbs") else FALLBACK_HBM_GBS
    out = []
    for name in names:
        p = dict(workload(name), stencil=27)
        n = p["n"]
        lat = Lattice(p, device=local)
        lat.init_fields()
        tuned = lat.tune(32)
        lat.evolve(10)
        lat.sync()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(lat.stream)
        lat.evolve(steps)
        e.record(lat.stream)
        lat.sync()
        ms = s.elapsed_time(e) / steps
        info = lat.kernel_info()
        su = n ** 3 / (ms / 1e3)
        rec = {"workload": name, "stencil": 27, "steps": steps, "ms_per_step": ms, "value": su, "unit": UNIT,
               "hbm_frac": su * 32 / 1e9 / peak,
               "launch": {"blocks": info["blocks"], "threads": info["threads"], "ty": info["ty"],
                          "depth": info["depth"], "smem": info["smem"],
                          "tuned_over": tuned["candidates"]}}
        if name == "m2phi2_256_fp32":
            rec["paper_s_per_step"] = 0.022
            rec["vs_paper"] = 0.022 / (ms / 1e3)
            ref = fp64_twin(p, local)
            ref.evolve(10 + steps)
            rec["fp64_error"] = dict(state_error(lat.get_state_exact(), ref.get_state(), stride=max(1, n // 32)),
                                     steps=10 + steps, subset=f"every {max(1, n // 32)}th site per axis",
                                     against="FP64 27-point lattice (phi whole), same seed")
            ref.close()
        out.append(rec)
        lat.close()
    return out


def measure_diagnostics(local, name, every=512, steps=2048):
    """Cost of the periodic diagnostics on the benchmark workload: 2048 steps with
    the per-site energy density and pressure (lat_energy_field) taken every 512
    steps, the interval of the paper's runs, against 2048 plain steps (CUDA
    events on the lattice's stream); and one call each of the field, the volume
    averages (lat_energies) and the binned spectrum (lat_spectrum)."""
    import time
    import torch
    from paper_0911_5692_gb300 import Lattice
    p = workload(name)
    n = p["n"]
    lat = Lattice(p, device=local)
    lat.init_fields()
    rho = torch.empty((n, n, n), dtype=lat.dtype, device=lat.device)
    pres = torch.empty_like(rho)
    lat.evolve(64)
    lat.energy_field(rho, pres)
    lat.sync()

    def timed(with_field):
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(lat.stream)
        for _ in range(steps // every):
            lat.evolve(every)
            if with_field:
                lat.energy_field(rho, pres)
        e.record(lat.stream)
        lat.sync()
        return s.elapsed_time(e)

    plain = min(timed(False) for _ in range(2))
    withf = min(timed(True) for _ in range(2))
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record(lat.stream)
    for _ in range(5):
        lat.energy_field(rho, pres)
    e.record(lat.stream)
    lat.sync()
    field_ms = s.elapsed_time(e) / 5
    t0 = time.perf_counter()
    lat.energies()
    energies_ms = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    lat.spectrum(0, n // 2)
    spectrum_ms = (time.perf_counter() - t0) * 1e3
    lat.close()
    return {"workload": name, "every": every, "steps": steps, "ms_plain": plain, "ms_with_energy_field": withf,
            "overhead": withf / plain - 1.0, "energy_field_ms": field_ms,
            "energies_ms_wall": energies_ms, "spectrum_ms_wall": spectrum_ms}


def measure_step(local, name="m2phi2_256_fp32", steps=300):
    """The fused 7-point step of another workload with the autotuned kernel
    shape (m^2 phi^2 at 256^3 FP32 is the configuration of the paper's own
    timing). CUDA events over graph replays after warm-up; the state (537 MB at
    256^3) exceeds L2."""
    import torch
    from paper_0911_5692_gb300 import Lattice
    p = workload(name)
    n = p["n"]
    esize = 4 if p["precision"] == 32 else 8
    lat = Lattice(p, device=local)
    lat.init_fields()
    tuned = lat.tune(64)
    lat.evolve(32)
    lat.sync()
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    s.record(lat.stream)
    lat.evolve(steps)
    e.record(lat.stream)
    lat.sync()
    ms = s.elapsed_time(e) / steps
    info = lat.kernel_info()
    peaks = measured_peaks()
    peak = float(peaks["hbm_gbs"]) if peaks and peaks.get("hbm_gbs") else FALLBACK_HBM_GBS
    gbs = 8 * esize * n ** 3 / (ms / 1e3) / 1e9
    lat.close()
    return {"workload": name, "steps": steps, "ms_per_step": ms, "value": n ** 3 / (ms / 1e3), "unit": UNIT,
            "achieved_GBs": gbs, "hbm_frac": gbs / peak, "hbm_frac_of_nominal": gbs / NOMINAL_HBM_GBS,
            "kernel": {"variant": info["variant"], "blocks": info["blocks"], "threads": info["threads"],
                       "ty": info["ty"], "depth": info["depth"], "tuned_over": tuned["candidates"]}}


def measure_lform(local, name, steps=320):
    """The L = 1/H form of the scale-factor update (DEFROST's choice, Sec. II.B)
    against eq. scale on the benchmark workload: per-step time of each (CUDA
    events over graph replays, the two runs alternated twice, best of each), the
    extra read-only pass's cost as their difference and its bandwidth against
    its 16 B (FP32) of algorithmic reads per site."""
    import torch
    from paper_0911_5692_gb300 import Lattice
    peaks = measured_peaks()
    peak = float(peaks["hbm_gbs"]) if peaks and peaks.get("hbm_gbs") else FALLBACK_HBM_GBS
    base = workload(name)
    n = base["n"]
    esize = 4 if base["precision"] == 32 else 8
    lats = {}
    for e in (1, 2):
        lat = Lattice(dict(base, expansion=e), device=local)
        lat.init_fields()
        lat.evolve(64)
        lat.sync()
        lats[e] = lat
    best = {1: float("inf"), 2: float("inf")}
    for _ in range(2):
        for e in (1, 2):
            lat = lats[e]
            s = torch.cuda.Event(enable_timing=True)
            t = torch.cuda.Event(enable_timing=True)
            s.record(lat.stream)
            lat.evolve(steps)
            t.record(lat.stream)
            lat.sync()
            best[e] = min(best[e], s.elapsed_time(t) / steps)
    a1, a2 = lats[1].scalars()["a"], lats[2].scalars()["a"]
    info = lats[2].kernel_info()
    ref = fp64_twin(dict(base, expansion=2), local)
    ref.evolve(64 + 2 * steps)
    stride = max(1, n // 32)
    err = dict(state_error(lats[2].get_state_exact(), ref.get_state(), stride=stride),
               hubble_length_rel=abs(lats[2].hubble_length() / ref.hubble_length() - 1), steps=64 + 2 * steps,
               subset=f"every {stride}th site per axis", against="FP64 lattice in the L = 1/H form (phi whole), "
                                                               "same seed")
    ref.close()
    for lat in lats.values():
        lat.close()
    pass_ms = best[2] - best[1]
    gbs = 4 * esize * n ** 3 / (pass_ms / 1e3) / 1e9 if pass_ms > 0 else None
    return {"workload": name, "steps": steps, "ms_per_step_eq_scale": best[1], "ms_per_step_lform": best[2],
            "value": n ** 3 / (best[2] / 1e3), "unit": UNIT, "lform_pass_ms": pass_ms,
            "lform_pass_GBs": gbs, "lform_pass_hbm_frac": gbs / peak if gbs else None,
            "launches_per_step": info["launches_per_step"],
            "a_rel_gap_after_run": a2 / a1 - 1.0, "fp64_error": err}


def measure_fp32_error(local, name, steps=200):
    """FP32 against FP64 on the GPU for a workload: the FP32 lattice as the
    workload stores it (phi split into an FP64 homogeneous mode and FP32
    fluctuations) and an FP64 lattice with phi whole, both initialised from the
    same seed by their own pipelines, `steps` steps, normwise error on the strided
    subset of 32^3 sites, against the whole field and against its fluctuation
    part."""
    from paper_0911_5692_gb300 import Lattice
    p = workload(name)
    n = p["n"]
    g64 = fp64_twin(p, local)
    g32 = Lattice(dict(p, precision=32), device=local)
    g32.init_fields()
    g32.evolve(steps)
    g64.evolve(steps)
    stride = max(1, n // 32)
    err = state_error(g32.get_state_exact(), g64.get_state(), stride=stride)
    s32, s64 = g32.scalars(), g64.scalars()
    g32.close()
    g64.close()
    return {"steps": steps, "subset": f"every {stride}th site per axis", "fp32_storage":
            "phi split" if p.get("split") else "fields whole", "normwise": err, "a_rel": abs(s32["a"] / s64["a"] - 1)}


def measure_run_statistics(local, name="m2phi2_256_fp32", every=250):
    """Statistics over the whole run of a workload (its own step count): the FP32
    lattice as the workload stores it (phi split) against an FP64 lattice with
    phi whole, both initialised from the same seed by their own pipelines, the
    volume statistics of lat_energies compared every `every` steps: the largest
    relative deviation of a, rho, <phi>, var phi and var chi over the run, <chi>
    relative to the spread of chi, and the step at which var chi first left its
    starting value by 1 % (the growth of the resonance)."""
    import math as _m
    from paper_0911_5692_gb300 import Lattice
    from paper_0911_5692_gb300.workloads import WORKLOADS
    p = workload(name)
    steps = int(WORKLOADS[name]["steps"])
    g64 = fp64_twin(p, local)
    g32 = Lattice(dict(p, precision=32), device=local)
    g32.init_fields()
    keys = {"a": "a", "rho": "rho", "mean_phi": "mean0", "var_phi": "var0", "var_chi": "var1"}
    worst = {k: 0.0 for k in keys}
    worst["mean_chi_over_std_chi"] = 0.0
    var_chi0 = None
    grows_at = None
    trace = []
    done = 0
    while done < steps:
        k = min(every, steps - done)
        g32.evolve(k)
        g64.evolve(k)
        done += k
        e32, e64 = g32.energies(), g64.energies()
        for key, ek in keys.items():
            worst[key] = max(worst[key], abs(e32[ek] - e64[ek]) / max(abs(e64[ek]), 1e-300))
        worst["mean_chi_over_std_chi"] = max(worst["mean_chi_over_std_chi"],
                                             abs(e32["mean1"] - e64["mean1"]) / max(_m.sqrt(max(e64["var1"], 0.0)), 1e-300))
        if var_chi0 is None:
            var_chi0 = e64["var1"]
        elif grows_at is None and abs(e64["var1"] / var_chi0 - 1.0) > 0.01:
            grows_at = done
        trace.append([done, e64["var1"], e64["a"]])
    g32.close()
    g64.close()
    return {"workload": name, "steps": steps, "every": every, "max_rel_dev": worst, "bound": 1e-3,
            "within_bound": all(v <= 1e-3 for v in worst.values()), "var_chi_leaves_start_at_step": grows_at,
            "var_chi_and_a_fp64": trace[:: max(1, len(trace) // 10)],
            "against": "FP64 lattice (phi whole) from the same seed, its own initialisation"}


def run_reference(args):
    """The FP64 CPU oracle timed as the reference arm, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import numpy as np
    from oracle.oracle import Oracle
    from paper_0911_5692_gb300.workloads import random_state
    p = dict(workload(args.workload), stencil=args.stencil, expansion=args.expansion)
    n_full = p["n"]
    # per-site cost from a short calibration, then the sample lattice that keeps
    # the whole (warmup + steps) run near 90 s
    cal = dict(p, n=32)
    o = Oracle(cal)
    o.set_state(*random_state(32, 2, precision=64), t=0.0, a=1.0, ad=0.5)
    o.step(2)
    t0 = time.perf_counter(); o.step(10); per_site = (time.perf_counter() - t0) / (10 * 32 ** 3)
    budget = 90.0 / max(1, args.steps + args.warmup)
    ns = int((budget / per_site) ** (1 / 3)) // 4 * 4
    ns = max(8, min(n_full, ns))
    sp = dict(p, n=ns)
    o = Oracle(sp)
    o.set_state(*random_state(ns, 3, precision=p["precision"], f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-4),
                              pi_mean=(0.3, 0.0), pi_amp=(1e-3, 1e-2)), t=0.0, a=1.0, ad=0.5)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t0
    value = ns ** 3 * args.steps / el
    cores = os.cpu_count()
    sample = (f"each step: one FP64 oracle leapfrog step of a {ns}^3 lattice with the {n_full}^3 workload's "
              f"model, couplings, dx and dt (OpenMP over {cores} host cores)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(args.workload, p, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import ctypes as C

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_0911_5692_gb300 import Lattice

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    p = dict(workload(args.workload), stencil=args.stencil, expansion=args.expansion)
    p["seed"] = p.get("seed", 0) + rank          # independent replica per rank
    n = p["n"]
    esize = 4 if p["precision"] == 32 else 8
    lat = Lattice(p, device=local)
    tuned = None
    lat.init_fields()
    if args.variant or args.ty or args.zr or args.depth:
        lat.set_kernel(args.variant, args.ty, args.zr, args.depth)
    elif not args.no_tune:
        tuned = lat.tune(64)     # untimed; the state is kept
    info = lat.kernel_info()
    lat.evolve(args.warmup)
    lat.sync()

    props = torch.cuda.get_device_properties(local)
    gpu_id = getattr(props, "uuid", None)
    gpu_id = f"GPU-{gpu_id}" if gpu_id is not None and not str(gpu_id).startswith("GPU-") else (gpu_id or local)
    clocks = ClockSampler(gpu_id)
    clocks.start()
    time.sleep(0.3)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    start.record(lat.stream)
    lat.evolve(args.steps)
    end.record(lat.stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks.stop()
    ms = start.elapsed_time(end)
    lat.sync()   # raises on a sticky device error (non-finite fields)
    t = torch.tensor([ms], dtype=torch.float64, device=f"cuda:{local}")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    sec = ms_max / 1e3
    value = world * n ** 3 * args.steps / sec
    ms_per_step = ms_max / args.steps

    # end to end through the C ABI with host buffers (lat_evolve_host): every step
    # uploads the stored state (4 arrays) from pinned host memory, advances one
    # step (the sums of the uploaded fields, then the fused step) and copies the
    # evolved state back into the same host arrays, with the scalars of every
    # step; the copies run in z-chunks, one stream per direction, so a step's
    # download and the next step's upload share the link. The same steps call by
    # call (lat_upload_state, lat_evolve, lat_download_state, lat_get_scalars:
    # one direction at a time) are timed after it.
    E = max(1, args.e2e_steps)
    host = []
    for w in (2, 3):
        for f in (0, 1):
            d = lat.get_state_device(f, w)
            hbuf = torch.empty_like(d, device="cpu").pin_memory()
            hbuf.copy_(d)
            host.append(hbuf)
    lib, h = lat._L, lat._h
    out8 = (C.c_double * 8)()
    rows = (C.c_double * (8 * E))()
    bufs = (C.c_void_p * 4)(*[hbuf.data_ptr() for hbuf in host])   # f0, f1, pi0, pi1 as stored

    def e2e_leg(run):
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        run()
        te = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device=f"cuda:{local}")
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        return world * n ** 3 * E / float(te.item())

    def call_by_call():
        for _ in range(E):
            assert lib.lat_upload_state(h, bufs, 0) == 0
            assert lib.lat_evolve(h, 1) == 0
            assert lib.lat_download_state(h, bufs, 0) == 0
            assert lib.lat_get_scalars(h, out8) == 0

    def host_resident():
        st = lib.lat_evolve_host(h, bufs, E, 0, rows)
        if st != 0:
            raise RuntimeError(f"lat_evolve_host: status {st}")

    e2e_value = e2e_leg(host_resident)
    e2e_serial = e2e_leg(call_by_call)
    del host

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    peaks = measured_peaks()
    if peaks and peaks.get("hbm_gbs"):
        peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    else:
        peak, peak_src = FALLBACK_HBM_GBS, "fallback"
    bytes_per_launch = 32 * n ** 3 if esize == 4 else 64 * n ** 3
    achieved = bytes_per_launch / (ms_per_step / 1e3) / 1e9
    traffic = traffic_record(args.workload, info["variant"], args.stencil, info["depth"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if esize == 4 else "f64", "data": "synthetic",
        "config": config_of(args.workload, p, world),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_source": peak_src,
                     "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                     "algorithmic_bytes_per_launch": bytes_per_launch,
                     "kernel": f"fused step variant {info['variant']}"
                               f"{', 27-point Laplacian' if args.stencil == 27 else ''} ({info['blocks']} blocks x "
                               f"{info['threads']} threads, ty={info['ty']}, zr={info['zr']}, depth={info['depth']})"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * n ** 3 * esize,
                "d2h_bytes_per_step": 4 * n ** 3 * esize + 8 * 8, "steps": E,
                "per_step": "upload of the stored state from pinned host memory, one step, download of the "
                            "evolved state and the scalars",
                "call": "lat_evolve_host (copies in 16 z-chunks, one stream per direction: a step's download "
                        "overlaps the next step's upload)",
                "call_by_call": {"value": e2e_serial, "unit": UNIT,
                                 "calls": "lat_upload_state, lat_evolve(1), lat_download_state, lat_get_scalars"}},
        "gpu_launches": args.steps * info["launches_per_step"],
        "tune": ({"chosen": {k: tuned[k] for k in ("variant", "ty", "zr", "depth", "blocks")},
                  "candidates": tuned["candidates"], "best_ms": tuned["best_ms"], "slowest_ms": tuned["slowest_ms"],
                  "by": "lat_tune: 64 steps per candidate shape on this lattice, CUDA events"}
                 if tuned else None),
        "clocks": clocks.summary(),
        "context": {"paper_gtx260_256cubed_su_per_s": 7.6e8,
                    "paper_gtx260_128cubed_su_per_s": 6.2e8,
                    "paper_speedup_vs_defrost_xeon_256cubed": 14.5,
                    "paper_speedup_vs_latticeeasy_256cubed": 58.0,
                    "ours_over_paper_gpu": value / world / 7.6e8,
                    "note": "paper (Sec. III, context only, other hardware): GTX 260 SP216, 27-point stencil, "
                            "0.022 s/step at 256^3 (< 900 s for 2^18 steps at 128^3); 14.5x DEFROST's 0.32 s/step "
                            "on a Xeon, a further 4x over LATTICEEASY. ours_over_paper_gpu compares this 7-point "
                            "line per GPU; the same configuration with the 27-point stencil is timed under "
                            "stencil27 (vs_paper)"},
    }
    if not args.no_extras and world == 1:
        lat.close()
        line["step_256"] = measure_step(local, "m2phi2_256_fp32", steps=1000)
        line["fp32_vs_fp64"] = measure_fp32_error(local, args.workload)
        line["fp32_vs_fp64_256"] = measure_fp32_error(local, "m2phi2_256_fp32")
        line["adjoint"] = measure_adjoint(local, fp64=True)
        line["adjoint_256"] = measure_adjoint(local, n=256, steps=400)
        line["ensemble"] = measure_ensemble(local)
        line["stencil27"] = measure_stencil27(local)
        line["diagnostics"] = measure_diagnostics(local, args.workload)
        line["lform"] = measure_lform(local, args.workload)
        line["slabs_1gpu"] = measure_slabs(local)
        line["run_statistics_256"] = measure_run_statistics(local)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(p, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_slabs(args):
    """bench.py --slabs: the workload's lattice (phi stored whole) cut into z-slabs.
    One rank: args.slabs slabs on one GPU (halos by device copies, the plain
    schedule, two steps per CUDA-graph replay). N ranks: one slab per rank, halos
    by NCCL point-to-point messages, the interior of each slab stepped while
    they are in flight, the four sums by all_reduce. value = the lattice's site
    updates per second (the whole job)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_0911_5692_gb300 import Lattice
    from paper_0911_5692_gb300.slab import DistComm, LocalComm, SlabEvolution, SlabGPU, slab_ranges

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    p = dict(workload(args.workload), split=0)
    n = p["n"]
    esize = 4 if p["precision"] == 32 else 8
    parts = world if world > 1 else max(1, args.slabs)
    ranges = slab_ranges(n, parts)
    mine = [ranges[rank]] if world > 1 else ranges
    # every rank builds the same initial state (same seed) and keeps its part
    lat = Lattice(p, device=local)
    lat.init_fields()
    sc0 = lat.scalars()
    arrs = [lat.get_state_device(f, w) for w in (0, 1) for f in (0, 1)]
    lat.close()
    stream = torch.cuda.Stream(device=local)
    slabs = [SlabGPU(p, z0, nzl, device=local, stream=stream) for z0, nzl in mine]
    for sl in slabs:
        sl.load(*arrs, t=sc0["t"], a=sc0["a"], ad=sc0["ad"], step=sc0["step"])
    del arrs
    ev = SlabEvolution(slabs, DistComm() if world > 1 else LocalComm(), overlap=world > 1)
    ev.prepare()
    K = max(2, args.steps // 2 * 2)
    if world == 1:
        ev.step(2)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            ev.step(2)
        for sl in slabs:
            sl.step_count -= 2

        def run(k):
            for _ in range(k // 2):
                with torch.cuda.stream(stream):
                    g.replay()
                for sl in slabs:
                    sl.step_count += 2
    else:
        def run(k):
            ev.step(k)
    run(max(2, args.warmup // 2 * 2))
    torch.cuda.synchronize()
    gpu_id = torch.cuda.get_device_properties(local)
    gpu_id = getattr(gpu_id, "uuid", None)
    gpu_id = f"GPU-{gpu_id}" if gpu_id is not None and not str(gpu_id).startswith("GPU-") else (gpu_id or local)
    clocks = ClockSampler(gpu_id)
    clocks.start()
    time.sleep(0.3)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    start.record(stream)
    run(K)
    end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks.stop()
    t = torch.tensor([start.elapsed_time(end)], dtype=torch.float64, device=f"cuda:{local}")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item()) / K
    for sl in slabs:
        assert np.isfinite(sl.scalars()["S"]).all()
    value = n ** 3 / (ms / 1e3)

    # end to end: every step the owned planes of each slab go up from pinned host
    # memory and come back after the step, with the scalars
    E = max(2, args.e2e_steps)
    host = []
    for sl in slabs:
        s = sl.current_set()
        host.append([sl.buffers[4 * s + k][1:sl.nzl + 1].cpu().pin_memory() for k in range(4)])
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(E):
        for sl, hb in zip(slabs, host):
            s = sl.current_set()
            with torch.cuda.stream(stream):
                for k in range(4):
                    sl.buffers[4 * s + k][1:sl.nzl + 1].copy_(hb[k], non_blocking=True)
        ev.step(1)
        for sl, hb in zip(slabs, host):
            s = sl.current_set()
            with torch.cuda.stream(stream):
                for k in range(4):
                    hb[k].copy_(sl.buffers[4 * s + k][1:sl.nzl + 1], non_blocking=True)
        stream.synchronize()
        for sl in slabs:
            sl.scalars()
    te = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device=f"cuda:{local}")
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e_value = n ** 3 * E / float(te.item())
    if rank != 0:
        dist.destroy_process_group()
        return
    peaks = measured_peaks()
    peak, peak_src = ((float(peaks["hbm_gbs"]), "measured") if peaks and peaks.get("hbm_gbs")
                      else (FALLBACK_HBM_GBS, "fallback"))
    per_gpu_bytes = 8 * esize * n ** 3 / world
    achieved = per_gpu_bytes / (ms / 1e3) / 1e9
    own_bytes = 4 * esize * sum(nzl for _, nzl in mine) * n * n
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f32" if esize == 4 else "f64", "data": "synthetic",
        "config": dict(config_of(args.workload, p, world), global_batch=1,
                       parallelism=f"zslab{parts}" + (" on one GPU" if world == 1 else "")),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": per_gpu_bytes,
                     "kernel": "fused slab step (variant 5 slab instance where compiled), all ranges of one step"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": own_bytes,
                "d2h_bytes_per_step": own_bytes + 64 * len(slabs), "steps": E,
                "per_step": "the owned planes of every slab up from pinned host memory, one step, back, and the scalars"},
        # per step: one rank holding every slab: one halo copy, one launch over all
        # its slabs' planes, one fused sum + scale-factor update; a rank of many:
        # its slab's three ranges and the scale-factor update
        "gpu_launches": K * (3 if world == 1 else 4),
        "clocks": clocks.summary(),
        "slabs": {"count": parts, "schedule": "overlap" if ev.overlap else "plain",
                  "planes": [nzl for _, nzl in ranges]},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.slabs:
        run_slabs(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
