"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every entry point include/lattice.h declares, the
ctypes structs match the C layout, and parameter validation (which runs before
any CUDA call) rejects bad inputs with the documented status codes."""
import ctypes as C
import math
import os
import re
import subprocess

import pytest

import paper_0911_5692_gb300 as pkg
from paper_0911_5692_gb300 import lattice as lat
from paper_0911_5692_gb300.workloads import lphi4, m2phi2

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lattice.h")


def declared_symbols():
    hdr = open(HEADER).read()
    return set(re.findall(r"^(?:lat_status|void|const char\*)\s+(lat_\w+)\(", hdr, re.M))


def test_library_exports_every_declared_symbol():
    L = pkg.load_library()
    decl = declared_symbols()
    assert decl == set(pkg.EXPORTED)
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.library_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (lat_\w+)$", out, re.M))
    assert decl <= exported, decl - exported
    for name in decl:
        assert getattr(L, name) is not None


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lattice.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(lat_params), '
                   'offsetof(lat_params, seed), offsetof(lat_params, fluct), offsetof(lat_params, stencil), '
                   'offsetof(lat_params, split), sizeof(lat_energy_report), '
                   'offsetof(lat_energy_report, var));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [C.sizeof(lat.LatParams), lat.LatParams.seed.offset, lat.LatParams.fluct.offset,
                    lat.LatParams.stencil.offset, lat.LatParams.split.offset, C.sizeof(lat.LatEnergyReport),
                    lat.LatEnergyReport.var.offset]


def test_status_strings():
    L = pkg.load_library()
    for code in range(9):
        assert L.lat_status_string(code)
    assert L.lat_status_string(0) == b"ok"


def _create_status(params):
    L = pkg.load_library()
    p = lat.make_params(params)
    h = C.c_void_p()
    st = L.lat_create(C.byref(p), None, C.byref(h))
    if st == 0:
        L.lat_destroy(h)
    else:
        assert h.value is None
    return st


@pytest.mark.parametrize("bad", [
    dict(n=30),               # N must be a multiple of 4
    dict(n=2),                # too small
    dict(n=2048),             # too large
    dict(precision=16),
    dict(model=7),
    dict(dt=-1.0),
    dict(L=0.0),
    dict(phi0=(0.0, 0.0)),    # A = 1/phi0 undefined
    dict(A=1.0, B=1.0, r=1.0, s=0.0),   # violates s - 2r + 3 = 0
    dict(expansion=3),
    dict(stencil=9),          # 7 (or 0) and 27 points only
    dict(split=2),            # phi stored whole (0) or split (1)
])
def test_validation_rejects_bad_parameters(bad):
    p = dict(lphi4(16), **bad)
    assert _create_status(p) == 1  # LAT_EINVAL


def test_validation_rejects_unstable_time_step():
    p = lphi4(16)
    p["dt"] = 2.5 * p["L"] / 16   # dt > 2 dx / sqrt(12)
    assert _create_status(p) == 2  # LAT_ECFL
    q = m2phi2(64, g2=2.5e-5)     # heavy chi at dt = 2^-10: w dt > 2
    assert _create_status(q) == 2


def test_stability_bound_follows_the_stencil():
    """The leapfrog is stable while dt^2 (k_max^2 + m_eff^2) <= 4, with
    k_max^2 = max over the Brillouin zone of -L(k): 12/dx^2 for the 7-point
    stencil, 92/(15 dx^2) for the 27-point one (at k dx = (pi, pi, pi), where the
    oracle's stencil gives the same value). Between the two bounds the 7-point
    lattice is refused and the 27-point one passes the check (creation then stops
    at the missing device on this host, with another status)."""
    import numpy as np
    from oracle.oracle import laplacian27
    n = 16
    p = lphi4(n)
    dx = p["L"] / n
    # k_max^2 of the oracle's stencil: the checkerboard mode at k dx = (pi, pi, pi)
    z, y, x = np.meshgrid(np.arange(4), np.arange(4), np.arange(4), indexing="ij")
    mode = (-1.0) ** (x + y + z)
    kmax2 = -laplacian27(mode, dx)[0, 0, 0] / mode[0, 0, 0]
    assert abs(kmax2 * dx * dx - 92 / 15) < 1e-12
    p["g2"] = 0.0   # no chi mass: m_eff^2 = 3 (cdom0 = 1, A phi0 = 1 in the default rescaling)
    meff2 = 3.0
    between = 2.0 / math.sqrt(0.5 * (12.0 / dx ** 2 + 92 / 15 / dx ** 2) + meff2)
    p7 = dict(p, dt=between, stencil=7)
    p27 = dict(p, dt=between, stencil=27)
    assert _create_status(p7) == 2
    assert _create_status(p27) != 2
    above = 2.0 / math.sqrt(92 / 15 / dx ** 2 + meff2) * 1.01
    assert _create_status(dict(p, dt=above, stencil=27)) == 2


def test_null_arguments():
    L = pkg.load_library()
    assert L.lat_create(None, None, None) == 1
    assert L.lat_evolve(None, 1) == 1
    assert L.lat_sync(None) == 1
    assert L.lat_energy_field(None, None, None) == 1
    assert L.lat_upload_state(None, None, 0) == 1
    assert L.lat_get_hubble_length(None, None) == 1
    assert L.lat_set_hubble_length(None, 1.0) == 1
    assert L.lat_download_state(None, None, 0) == 1
    assert L.lat_get_background(None, None) == 1
    assert L.lat_set_background(None, None) == 1
    assert L.lat_recenter(None) == 1
    assert L.lat_tune(None, 10, None) == 1
    assert L.lat_batch_tile_heights(None, None) == 1
    assert L.lat_batch_shape(None, None) == 1
    assert L.lat_batch_set_shape(None, 256, 8, 1) == 1
    assert L.lat_slab_advance_local(None, 1, None, 1, 1) == 1
    assert L.lat_copy_regions(None, None, 1, 16, None) == 1
    assert L.lat_evolve_host(None, None, 1, 0, None) == 1
    assert L.lat_slab_step_ranges(None, 1, None, 1, None) == 1
    L.lat_destroy(None)


def test_copy_regions_argument_errors():
    """lat_copy_regions checks its arguments before any CUDA call: a size or a
    pointer that is not a multiple of 16 bytes, a null entry and a negative
    count are LAT_EINVAL; nothing to copy is LAT_OK."""
    L = pkg.load_library()
    P = C.c_void_p
    good = (P * 2)(4096, 8192)
    odd = (P * 2)(4096, 8200)
    null = (P * 2)(4096, None)
    assert L.lat_copy_regions(good, good, 2, 24, None) == 1
    assert L.lat_copy_regions(odd, good, 2, 32, None) == 1
    assert L.lat_copy_regions(good, null, 2, 32, None) == 1
    assert L.lat_copy_regions(good, good, -1, 32, None) == 1
    assert L.lat_copy_regions(good, good, 0, 32, None) == 0
    assert L.lat_copy_regions(good, good, 2, 0, None) == 0


def test_slab_advance_local_argument_errors():
    L = pkg.load_library()
    P = C.c_void_p
    hs = (P * 1)(None)
    sh = (P * 1)(None)
    assert L.lat_slab_advance_local(hs, 0, sh, 1, 1) == 1
    assert L.lat_slab_advance_local(hs, 65, sh, 1, 1) == 1
    assert L.lat_slab_advance_local(hs, 1, sh, 0, 1) == 1
    assert L.lat_slab_advance_local(hs, 1, sh, 193, 1) == 1
    assert L.lat_slab_advance_local(hs, 1, sh, 1, 1) == 1      # null handle


@pytest.mark.parametrize("case", ["null_phi", "null_chi", "null_out", "precision", "model", "L", "small"])
def test_static_sums_argument_errors(case):
    """lat_field_sums_static validates its arguments before any CUDA call: null
    pointers, a precision other than 32 or 64, an unknown model, L <= 0 and
    n < 4 give LAT_EINVAL."""
    L = pkg.load_library()
    buf = (C.c_double * 8)()
    ptr = C.cast(buf, C.c_void_p)
    args = dict(f_phi=ptr, f_chi=ptr, n=16, precision=32, model=0, L=10.0, out=ptr)
    if case == "null_phi":
        args["f_phi"] = None
    elif case == "null_chi":
        args["f_chi"] = None
    elif case == "null_out":
        args["out"] = None
    elif case == "precision":
        args["precision"] = 16
    elif case == "model":
        args["model"] = 7
    elif case == "L":
        args["L"] = 0.0
    else:
        args["n"] = 2
    st = L.lat_field_sums_static(args["f_phi"], args["f_chi"], args["n"], args["precision"], args["model"],
                                 args["L"], args["out"], None)
    assert st == 1


@pytest.mark.parametrize("array_bytes", [64 * 4, 36 ** 3 * 8, 256 ** 3 * 4, 512 ** 3 * 4, 1024 ** 3 * 4, 130 * 130 * 515 * 8])
def test_buffer_layout(array_bytes):
    """lat_buffer_layout (host only): eight non-overlapping arrays in one
    allocation, 128-byte aligned, with starts that differ modulo 2 KB."""
    L = pkg.load_library()
    off = (C.c_uint64 * 8)()
    total = C.c_uint64()
    assert L.lat_buffer_layout(array_bytes, off, C.byref(total)) == 0
    o = list(off)
    assert o[0] == 0 and all(x % 128 == 0 for x in o)
    assert all(o[k + 1] - o[k] >= array_bytes for k in range(7))
    assert total.value >= o[7] + array_bytes
    assert len({x % 2048 for x in o}) == 8


def test_buffer_layout_argument_errors():
    L = pkg.load_library()
    off = (C.c_uint64 * 8)()
    total = C.c_uint64()
    assert L.lat_buffer_layout(0, off, C.byref(total)) == 1
    assert L.lat_buffer_layout((1 << 40) + 1, off, C.byref(total)) == 1
    assert L.lat_buffer_layout(4096, None, C.byref(total)) == 1
    assert L.lat_buffer_layout(4096, off, None) == 1
