"""Multi-step accuracy of the split pressure gradient (Sec. 5.4, Eqs. (32)-(34)).

The split replaces (1/rho) grad p^{n+1} by (1/rho_0) grad p^{n+1} +
(1/rho - 1/rho_0) grad p_hat with the extrapolation p_hat = 2p^n - p^{n-1},
which is exact when grad p_hat = grad p^{n+1} and otherwise depends on how
smooth the pressure is in time and on the density ratio (the paragraph after
Eq. (34)).  This driver measures that error over a sequence of steps in which
the unsplit pressure is known exactly:

  * fixed density rho (tanh layer, ratio rho_l/rho_g) and constraint S;
  * a velocity u_div with D u_div = S, from a constant-density projection
    (beta = 0, so the split projection is the exact classic projection);
  * the exact pressure P(t_n) = Q cos(n phi) + R sin(n phi) with smooth Q, R
    (phi = omega dt, the phase advance per step);
  * at step n the predicted velocity u*_n = u_div + dt G P(t_n) / rho_f, so that
    the unsplit projection (Eqs. (29)-(30)) returns exactly P(t_n); it is
    formed with the correction of Eq. (33) applied with p = p_hat = -P(t_n);
  * the split projection of step n takes p_hat from its own two previous
    pressures (the first step from the exact P(t_{-1}), P(t_{-2})), and
    e_n = max |p_n - P(t_n)| / max |P(t_n)|.

Also reported: the error with the exact history (p^n, p^{n-1} = P(t_{n-1}),
P(t_{n-2})), which isolates the one-step splitting error from its
accumulation.  The numerical work runs in the backend's projection calls; the
default backend is libppe through the C ABI on the GPU.
"""
from __future__ import annotations

import math

import numpy as np

from . import fields


class GpuBackend:
    """libppe on one GPU (torch tensors as device memory)."""

    def __init__(self, shape_xyz, lengths, precision=None):
        import torch

        from . import ppe
        self.torch, self.ppe = torch, ppe
        nx, ny, nz = shape_xyz
        self.plan = ppe.Plan(nx, ny, nz, *lengths, precision=ppe.FP64 if precision is None else precision,
                             compat_tol=0.0)

    def dev(self, a):
        return self.torch.from_numpy(np.ascontiguousarray(a)).cuda()

    def empty(self, like):
        return self.torch.empty_like(like)

    def project(self, u, v, w, S, rho, p_n, p_nm1, dt):
        o = [self.empty(rho), self.empty(u), self.empty(v), self.empty(w)]
        self.plan.project(u, v, w, S, rho, p_n, p_nm1, dt, *o)
        return o

    def correct(self, u, v, w, rho, p, p_n, p_nm1, dt, rho0):
        o = [self.empty(u), self.empty(v), self.empty(w)]
        self.plan.correct(u, v, w, rho, p, p_n, p_nm1, dt, *o, rho0=rho0)
        return o

    @staticmethod
    def lin(a, x, b, y):
        return a * x + b * y

    @staticmethod
    def maxabs(x):
        return float(x.abs().max())

    def close(self):
        self.plan.close()


def run(n=64, rho_l=640.0, rho_g=120.0, phi=0.05, steps=40, amplitude=1.0e4, seed=0, width=6.0, backend=None):
    """One sequence; returns dict(errors, errors_exact_history, max_error, final_error, growth, ...)."""
    fl = fields.make_fields(n, n, n, seed=seed, recipe="multimode", width=width, rho_l=rho_l, rho_g=rho_g)
    lengths = (fl.lx, fl.ly, fl.lz)
    own = backend is None
    B = GpuBackend((n, n, n), lengths) if own else backend
    try:
        rho = B.dev(fl.rho)
        S = B.dev(fl.S)
        rho0 = float(fl.rho.min())
        zero = B.dev(np.zeros(fl.shape))
        # u_div: constant density, p_hat = 0  ->  the classic projection, D u_div = S
        _, ud, vd, wd = B.project(B.dev(fl.u), B.dev(fl.v), B.dev(fl.w), S, B.dev(np.full(fl.shape, rho0)), zero,
                                  zero, fl.dt)
        Q = B.dev(fields.smooth_field(n, n, n, seed=seed + 1, amplitude=amplitude))
        R = B.dev(fields.smooth_field(n, n, n, seed=seed + 2, amplitude=amplitude))

        def P(k):
            return B.lin(math.cos(k * phi), Q, math.sin(k * phi), R)

        hist = [P(-1), P(-2)]  # p^n, p^{n-1} of the split sequence
        errs, errs_exact = [], []
        for k in range(steps):
            q = P(k)
            mq = B.lin(-1.0, q, 0.0, q)
            us, vs, ws = B.correct(ud, vd, wd, rho, mq, mq, mq, fl.dt, rho0)  # u_div + dt G q / rho_f
            p_split = B.project(us, vs, ws, S, rho, hist[0], hist[1], fl.dt)[0]
            p_exact_hist = B.project(us, vs, ws, S, rho, P(k - 1), P(k - 2), fl.dt)[0]
            scale = B.maxabs(q)
            errs.append(B.maxabs(B.lin(1.0, p_split, -1.0, q)) / scale)
            errs_exact.append(B.maxabs(B.lin(1.0, p_exact_hist, -1.0, q)) / scale)
            hist = [p_split, hist[0]]
        half = max(1, steps // 2)
        growth = (max(errs[half:]) / max(errs[:half])) if max(errs[:half]) > 0 else float("nan")
        return {"grid": n, "rho_ratio": rho_l / rho_g, "phi": phi, "steps": steps, "errors": errs,
                "errors_exact_history": errs_exact, "max_error": max(errs), "final_error": errs[-1],
                "max_error_exact_history": max(errs_exact), "growth": growth}
    finally:
        if own:
            B.close()


def sweep(n=64, ratios=((640.0, 120.0), (640.0, 60.0), (1000.0, 100.0), (1000.0, 10.0)),
          phis=(0.2, 0.1, 0.05, 0.025), steps=40):
    """The error table over density ratios and phase advances per step."""
    rows = []
    for rl, rg in ratios:
        for phi in phis:
            r = run(n=n, rho_l=rl, rho_g=rg, phi=phi, steps=steps)
            rows.append({k: r[k] for k in ("rho_ratio", "phi", "max_error", "final_error",
                                           "max_error_exact_history", "growth")})
    return rows


if __name__ == "__main__":
    import json
    import sys
    print(json.dumps(sweep(n=int(sys.argv[1]) if len(sys.argv) > 1 else 64), indent=1))
