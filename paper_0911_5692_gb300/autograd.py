"""torch.autograd binding of the lattice evolution's reverse-mode derivative.

``LatticeEvolve.apply(f, pi, g2, lattice, n_steps, scalars, ckpt_every, observable)``
runs n_steps of the staggered leapfrog (Sec. II.B, eq. evo) on ``lattice`` from
the fields ``f`` and momenta ``pi`` (CUDA tensors of shape (2, n, n, n) in the
lattice dtype, phi then chi) with coupling ``g2`` (a 0-d float64 tensor), and
returns the observable of the final state as a 0-d float64 CUDA tensor:
observable 0 (default), J = <chi^2> of the final fields; observable 1, the
fraction of the energy density in chi (lat_adjoint). Its
backward pass is the library's hand-written adjoint (lat_adjoint: sqrt(n)
checkpointing with recomputation, exact for the discrete scheme including the
a(t) coupling), not autograd's tape: when any input needs a gradient the
forward call computes J and the gradient in one lat_adjoint call and backward
only scales them by the incoming gradient. ``scalars`` is the dict of
Lattice.set_scalars (t, a, ad, step) of the starting state.
"""
from __future__ import annotations

import torch


class LatticeEvolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, pi, g2, lattice, n_steps, scalars, ckpt_every=0, observable=0):
        n = lattice.n
        assert f.shape == (2, n, n, n) and pi.shape == (2, n, n, n)
        assert f.dtype == lattice.dtype and pi.dtype == lattice.dtype and f.is_cuda and pi.is_cuda
        lattice.set_g2(float(g2))
        lattice.set_scalars(**scalars)
        torch.cuda.current_stream(f.device).synchronize()
        for i in (0, 1):
            lattice.set_state_device(i, 0, f[i].reshape(-1))
            lattice.set_state_device(i, 1, pi[i].reshape(-1))
        if any(ctx.needs_input_grad[:3]):
            J, df, dp, dg2 = lattice.adjoint(int(n_steps), int(observable), int(ckpt_every))
            ctx.save_for_backward(df, dp)
            ctx.dg2 = dg2
        else:
            lattice.evolve(int(n_steps))
            J = lattice.adjoint(0, int(observable))[0]
        ctx.g2_meta = (g2.device, g2.dtype) if torch.is_tensor(g2) else (torch.device("cpu"), torch.float64)
        return torch.tensor(J, dtype=torch.float64, device=f.device)

    @staticmethod
    def backward(ctx, gJ):
        df, dp = ctx.saved_tensors
        gf = (gJ.to(df.dtype) * df) if ctx.needs_input_grad[0] else None
        gp = (gJ.to(dp.dtype) * dp) if ctx.needs_input_grad[1] else None
        gg = None
        if ctx.needs_input_grad[2]:
            dev, dt = ctx.g2_meta
            gg = (gJ.to(torch.float64).cpu() * ctx.dg2).to(device=dev, dtype=dt)
        return gf, gp, gg, None, None, None, None, None
