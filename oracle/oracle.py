"""ctypes wrapper around the FP64 CPU oracle (lattice_oracle.c).

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this module. The product library never
does; it shares no code with the oracle.

The oracle follows the paper's equations one by one (Sainio, arXiv:0911.5692,
Sec. II.B): rescaling to program units, eq. scalar-evo, eq. scale, the
staggered leapfrog eq. evo, eq. rho-pres and the DEFROST-style initial
conditions. See the header of lattice_oracle.c for the equation list.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lattice_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblattice_oracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_ENONFINITE = 0, 1, 3, 5


class OrcParams(C.Structure):
    _fields_ = [
        ("n", C.c_int32), ("model", C.c_int32), ("expansion", C.c_int32), ("stencil", C.c_int32),
        ("L", C.c_double), ("dt", C.c_double),
        ("lam", C.c_double), ("m", C.c_double), ("g2", C.c_double),
        ("phi0", C.c_double * 2), ("dphi0", C.c_double * 2),
        ("eight_pi_G", C.c_double),
        ("A", C.c_double), ("B", C.c_double), ("r", C.c_double), ("s", C.c_double),
        ("kcut", C.c_double), ("fluct", C.c_double),
        ("seed", C.c_uint64),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            P = C.c_void_p
            dp = C.POINTER(C.c_double)
            L.orc_create.argtypes = [C.POINTER(OrcParams), C.POINTER(P)]
            L.orc_destroy.argtypes = [P]
            L.orc_get_derived.argtypes = [P, dp]
            L.orc_array.argtypes = [P, C.c_int, C.c_int]
            L.orc_array.restype = dp
            L.orc_get_scalars.argtypes = [P, dp]
            L.orc_set_scalars.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_int64]
            L.orc_chi_fraction.argtypes = [P, dp, C.POINTER(dp), C.POINTER(dp), dp]
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_set_threads.restype = C.c_int
            L.orc_get_ell.argtypes = [P]
            L.orc_get_ell.restype = C.c_double
            L.orc_set_ell.argtypes = [P, C.c_double]
            L.orc_laplacian.argtypes = [C.c_int, C.c_double, dp, dp]
            L.orc_grad2_mean.argtypes = [C.c_int, C.c_double, dp]
            L.orc_grad2_mean.restype = C.c_double
            L.orc_sums.argtypes = [P]
            L.orc_scale_update.argtypes = [P, dp, dp, dp]
            L.orc_step.argtypes = [P, C.c_int64]
            L.orc_init_fields.argtypes = [P]
            L.orc_energies.argtypes = [P, dp]
            L.orc_energy_field.argtypes = [P, dp, dp]
            L.orc_spectrum.argtypes = [P, C.c_int, C.c_int, dp, dp, C.POINTER(C.c_int64)]
            L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
            L.orc_normal.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32]
            L.orc_normal.restype = C.c_double
            L.orc_fft1.argtypes = [C.c_int, dp, dp, dp, dp, C.c_int]
            L.orc_fft3.argtypes = [C.c_int, dp, dp, C.c_int]
            L.orc_laplacian27.argtypes = [C.c_int, C.c_double, dp, dp]
            L.orc_grad2_mean27.argtypes = [C.c_int, C.c_double, dp]
            L.orc_grad2_mean27.restype = C.c_double
            L.orc_set_g2.argtypes = [P, C.c_double]
            L.orc_adjoint.argtypes = [P, C.c_int64, C.POINTER(dp), C.POINTER(dp), dp]
            L.orc_step_coefs.argtypes = [P, C.c_double, C.c_double, dp, dp]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(d: dict) -> OrcParams:
    p = OrcParams()
    p.n = int(d["n"]); p.model = int(d.get("model", 0)); p.expansion = int(d.get("expansion", 1))
    p.stencil = int(d.get("stencil", 7))
    p.L = float(d.get("L", 10.0)); p.dt = float(d["dt"])
    p.lam = float(d.get("lam", 0.0)); p.m = float(d.get("m", 0.0)); p.g2 = float(d.get("g2", 0.0))
    phi0 = d.get("phi0", (1.0, 0.0)); dphi0 = d.get("dphi0", (0.0, 0.0))
    p.phi0[0], p.phi0[1] = float(phi0[0]), float(phi0[1])
    p.dphi0[0], p.dphi0[1] = float(dphi0[0]), float(dphi0[1])
    p.eight_pi_G = float(d.get("eight_pi_G", 1.0))
    p.A = float(d.get("A", 0.0)); p.B = float(d.get("B", 0.0))
    p.r = float(d.get("r", 0.0)); p.s = float(d.get("s", 0.0))
    p.kcut = float(d.get("kcut", 0.0)); p.fluct = float(d.get("fluct", 1.0))
    p.seed = int(d.get("seed", 0))
    return p


class OracleError(RuntimeError):
    pass


def _check(st: int, what: str):
    if st != ORC_OK:
        raise OracleError(f"{what} failed with status {st}")


class Oracle:
    """One FP64 lattice: fields f_i at t+dt/2, momenta pi_i at t, a at t+dt/2, a' at t."""

    def __init__(self, params: dict):
        self._L = lib()
        self.params = dict(params)
        self._p = make_params(params)
        h = C.c_void_p()
        _check(self._L.orc_create(C.byref(self._p), C.byref(h)), "orc_create")
        self._h = h
        self.n = self._p.n

    def close(self):
        if getattr(self, "_h", None):
            self._L.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- arrays (views onto oracle memory; copy before the oracle is destroyed)
    def array(self, field: int, what: int) -> np.ndarray:
        ptr = self._L.orc_array(self._h, field, what)
        n = self.n
        return np.ctypeslib.as_array(ptr, shape=(n, n, n))

    def get_state(self):
        """(f0, f1, pi0, pi1) copies, each [z][y][x]."""
        return tuple(self.array(i, w).copy() for w in (0, 1) for i in (0, 1))

    def set_state(self, f0, f1, pi0, pi1, t=0.0, a=1.0, ad=0.0, step=0):
        for i, arr in enumerate((f0, f1)):
            self.array(i, 0)[...] = np.asarray(arr, dtype=np.float64)
        for i, arr in enumerate((pi0, pi1)):
            self.array(i, 1)[...] = np.asarray(arr, dtype=np.float64)
        self._L.orc_set_scalars(self._h, float(t), float(a), float(ad), int(step))

    def derived(self) -> dict:
        out = (C.c_double * 10)()
        self._L.orc_get_derived(self._h, out)
        keys = ("A", "B", "r", "s", "beta", "cdom0", "pdom", "kappa0", "pint", "dx")
        return dict(zip(keys, list(out)))

    def scalars(self) -> dict:
        out = (C.c_double * 8)()
        self._L.orc_get_scalars(self._h, out)
        return {"t": out[0], "a": out[1], "ad": out[2], "step": int(out[3]), "S": list(out[4:8])}

    def ell(self) -> float:
        """The L = 1/H form's l = a/a' (program time) at the momentum time."""
        return self._L.orc_get_ell(self._h)

    def set_ell(self, ell: float):
        self._L.orc_set_ell(self._h, float(ell))

    def init_fields(self):
        _check(self._L.orc_init_fields(self._h), "orc_init_fields")

    def step(self, nsteps: int = 1):
        _check(self._L.orc_step(self._h, int(nsteps)), "orc_step")

    def scale_update(self):
        a1, ah, add = C.c_double(), C.c_double(), C.c_double()
        _check(self._L.orc_scale_update(self._h, C.byref(a1), C.byref(ah), C.byref(add)), "orc_scale_update")
        return a1.value, ah.value, add.value

    ENERGY_KEYS = ("t", "a", "ad", "H", "rho", "p", "w", "curv_resid", "kin0", "kin1",
                   "grad0", "grad1", "pot", "mean0", "mean1", "var0", "var1")

    def energies(self) -> dict:
        out = (C.c_double * 17)()
        _check(self._L.orc_energies(self._h, out), "orc_energies")
        return dict(zip(self.ENERGY_KEYS, list(out)))

    def energy_field(self):
        """Energy density and pressure at every site (eq. rho-pres per site), as
        two (n, n, n) arrays [z][y][x] in the units of energies()."""
        n3 = self.n ** 3
        rho = np.zeros(n3)
        pres = np.zeros(n3)
        _check(self._L.orc_energy_field(self._h, _dp(rho), _dp(pres)), "orc_energy_field")
        shp = (self.n,) * 3
        return rho.reshape(shp), pres.reshape(shp)

    def set_g2(self, g2: float):
        """Change the coupling g^2 (kappa0 follows); the state is kept."""
        _check(self._L.orc_set_g2(self._h, float(g2)), "orc_set_g2")
        self.params["g2"] = float(g2)

    def vjp(self, nsteps: int, fbar, pibar, abar: float = 0.0, adbar: float = 0.0):
        """Reverse-mode product of nsteps steps with the adjoint (fbar, pibar,
        abar, adbar) of the final state. Returns (fbar0, pibar0, abar0, adbar0,
        dkappa0, dg2): the adjoint of the state at the start, of kappa0 and of
        g^2. The lattice ends advanced by nsteps."""
        n3 = self.n ** 3
        fb = [np.ascontiguousarray(np.asarray(fbar[i], dtype=np.float64).reshape(n3)).copy() for i in (0, 1)]
        pb = [np.ascontiguousarray(np.asarray(pibar[i], dtype=np.float64).reshape(n3)).copy() for i in (0, 1)]
        fps = (C.POINTER(C.c_double) * 2)(_dp(fb[0]), _dp(fb[1]))
        pps = (C.POINTER(C.c_double) * 2)(_dp(pb[0]), _dp(pb[1]))
        sb = np.array([abar, adbar, 0.0, 0.0], dtype=np.float64)
        _check(self._L.orc_adjoint(self._h, int(nsteps), fps, pps, _dp(sb)), "orc_adjoint")
        shp = (self.n,) * 3
        return ([f.reshape(shp) for f in fb], [q.reshape(shp) for q in pb], sb[0], sb[1], sb[2], sb[3])

    def step_coefs(self, a: float, ad: float, S) -> dict:
        """Coefficients of a step from its starting scalars (a, a', averages S):
        cL, cF, cdom, kappa and y = a'_n + a'_{n+1}."""
        s = np.ascontiguousarray(np.asarray(S, dtype=np.float64))
        out = np.zeros(5)
        _check(self._L.orc_step_coefs(self._h, float(a), float(ad), _dp(s), _dp(out)), "orc_step_coefs")
        return dict(zip(("cL", "cF", "cdom", "kappa", "y"), out.tolist()))

    def chi2_mean(self) -> float:
        """Observable J = <f1^2>, the volume mean of the squared program-unit chi."""
        f1 = self.array(1, 0)
        return float(np.sum(f1 * f1, dtype=np.float64) / f1.size)

    def chi2_gradient(self, nsteps: int):
        """J = <f1^2> after nsteps steps from the current state, and its gradient
        with respect to the current (f, pi) and g^2. Returns (J, dJ/df [2 arrays],
        dJ/dpi [2 arrays], dJ/dg2). The lattice ends advanced by nsteps."""
        n = self.n
        st = self.get_state()
        sc = self.scalars()
        self.step(nsteps)
        J = self.chi2_mean()
        f1 = self.array(1, 0).copy()
        self.set_state(*st, t=sc["t"], a=sc["a"], ad=sc["ad"], step=sc["step"])
        zeros = np.zeros((n, n, n))
        fb, pb, _, _, _, dg2 = self.vjp(nsteps, [zeros, 2.0 * f1 / n ** 3], [zeros, zeros])
        return J, fb, pb, dg2

    def chi_fraction(self, with_gradient: bool = False):
        """Observable 1: the fraction of the energy density in chi at the momentum
        time of the stored state (orc_chi_fraction). With with_gradient, also its
        gradient with respect to the stored f, pi (two arrays each), a, a' and
        its direct derivative with respect to g^2 (at a fixed state)."""
        n, n3 = self.n, self.n ** 3
        J = C.c_double()
        if not with_gradient:
            _check(self._L.orc_chi_fraction(self._h, C.byref(J), None, None, None), "orc_chi_fraction")
            return J.value
        fb = [np.zeros(n3) for _ in range(2)]
        pb = [np.zeros(n3) for _ in range(2)]
        sb = np.zeros(3)
        fps = (C.POINTER(C.c_double) * 2)(_dp(fb[0]), _dp(fb[1]))
        pps = (C.POINTER(C.c_double) * 2)(_dp(pb[0]), _dp(pb[1]))
        _check(self._L.orc_chi_fraction(self._h, C.byref(J), fps, pps, _dp(sb)), "orc_chi_fraction")
        shp = (n,) * 3
        return J.value, [f.reshape(shp) for f in fb], [q.reshape(shp) for q in pb], sb[0], sb[1], sb[2]

    def chi_fraction_gradient(self, nsteps: int):
        """Observable 1 after nsteps steps from the current state and its gradient
        with respect to the current (f, pi) and g^2, as chi2_gradient."""
        st = self.get_state()
        sc = self.scalars()
        self.step(nsteps)
        J, fb, pb, ab, adb, dg2_direct = self.chi_fraction(with_gradient=True)
        self.set_state(*st, t=sc["t"], a=sc["a"], ad=sc["ad"], step=sc["step"])
        fb0, pb0, _, _, _, dg2 = self.vjp(nsteps, fb, pb, ab, adb)
        return J, fb0, pb0, dg2 + dg2_direct

    def spectrum(self, field: int, nbins: int):
        k = np.zeros(nbins); p = np.zeros(nbins); c = np.zeros(nbins, dtype=np.int64)
        _check(self._L.orc_spectrum(self._h, field, nbins, _dp(k), _dp(p),
                                    c.ctypes.data_as(C.POINTER(C.c_int64))), "orc_spectrum")
        return k, p, c


# -- free functions -------------------------------------------------------------

def laplacian(f: np.ndarray, dx: float) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    lib().orc_laplacian(f.shape[0], float(dx), _dp(f), _dp(out))
    return out


def laplacian27(f: np.ndarray, dx: float) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    lib().orc_laplacian27(f.shape[0], float(dx), _dp(f), _dp(out))
    return out


def grad2_mean27(f: np.ndarray, dx: float) -> float:
    f = np.ascontiguousarray(f, dtype=np.float64)
    return lib().orc_grad2_mean27(f.shape[0], float(dx), _dp(f))


def grad2_mean(f: np.ndarray, dx: float) -> float:
    f = np.ascontiguousarray(f, dtype=np.float64)
    return lib().orc_grad2_mean(f.shape[0], float(dx), _dp(f))


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xffffffff for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def normal(seed: int, field: int, quantity: int, site: int) -> float:
    return lib().orc_normal(int(seed), int(field), int(quantity), int(site))


def fft1(x: np.ndarray, sign: int = -1) -> np.ndarray:
    x = np.asarray(x, dtype=np.complex128)
    xr = np.ascontiguousarray(x.real); xi = np.ascontiguousarray(x.imag)
    yr = np.empty_like(xr); yi = np.empty_like(xi)
    lib().orc_fft1(len(x), _dp(xr), _dp(xi), _dp(yr), _dp(yi), int(sign))
    return yr + 1j * yi


def fft3(x: np.ndarray, sign: int = -1) -> np.ndarray:
    x = np.asarray(x, dtype=np.complex128)
    re = np.ascontiguousarray(x.real); im = np.ascontiguousarray(x.imag)
    lib().orc_fft3(x.shape[0], _dp(re), _dp(im), int(sign))
    return re + 1j * im


def set_threads(n: int) -> int:
    """Threads of the oracle's OpenMP loops (timing only; results do not depend
    on it). n <= 0 leaves the count; returns the count in effect."""
    return int(lib().orc_set_threads(int(n)))
