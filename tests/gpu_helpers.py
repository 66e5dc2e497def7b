"""Shared helpers of the GPU parity tests: run the CUDA path and the FP64 oracle
from the same seeded state and compare them normwise."""
import numpy as np

from oracle.oracle import Oracle
from paper_0911_5692_gb300 import Lattice


def normwise(x, ref):
    """max |x - ref| / max |ref| (per field and per quantity)."""
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(np.asarray(x) - ref)) / (den if den > 0 else 1.0))


def paired(params, state, scalars=(0.0, 1.0, 0.0, 0), variant=0, ty=0, zr=0):
    """A GPU lattice and an oracle lattice holding the same state."""
    g = Lattice(params)
    if variant:
        g.set_kernel(variant, ty, zr)
    t, a, ad, step = scalars
    g.set_state(*state, t=t, a=a, ad=ad, step=step)
    o = Oracle(params)
    o.set_state(*state, t=t, a=a, ad=ad, step=step)
    return g, o


def compare_states(g, o, tol, what=""):
    gs = g.get_state()
    os_ = o.get_state()
    errs = {}
    for name, x, r in zip(("f0", "f1", "p0", "p1"), gs, os_):
        errs[name] = normwise(x, r)
    worst = max(errs.values())
    assert worst <= tol, f"{what} normwise errors {errs} > {tol}"
    return errs
