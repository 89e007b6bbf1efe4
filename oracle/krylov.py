"""Preconditioned and flexible conjugate gradients (Sec. 5.1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Zero initial guess by default.  The paper stops on a 1e8 reduction of the
natural P^{-1}-norm of the residual; the solvers here stop on the l2
relative residual ||r_k|| / ||b|| (the reading used for the DOFs/s metric)
and record the natural-norm history as well.

Pins: an exact preconditioner gives convergence in one iteration; unpre-
conditioned CG on an SPD matrix reaches the scipy direct solve.
"""

from __future__ import annotations

import numpy as np


def pcg(A, b, M=None, rtol=1e-8, maxit=1000, x0=None, flexible=False):
    """Returns (x, info) with info = {iterations, history_l2,
    history_natural, converged}.  A, M: callables or matrices."""
    Aop = A if callable(A) else (lambda v: A @ v)
    Mop = (lambda v: v.copy()) if M is None else (M if callable(M) else (lambda v: M @ v))
    x = np.zeros_like(b) if x0 is None else np.array(x0, float, copy=True)
    r = b - Aop(x)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, {"iterations": 0, "history_l2": [0.0], "history_natural": [0.0],
                   "converged": True}
    z = Mop(r)
    p = z.copy()
    rz = float(r @ z)
    hist = [np.linalg.norm(r) / bn]
    nat0 = np.sqrt(abs(rz))
    hnat = [1.0]
    it = 0
    converged = hist[-1] <= rtol
    while not converged and it < maxit:
        q = Aop(p)
        pq = float(p @ q)
        if not (pq > 0.0):
            raise np.linalg.LinAlgError("CG breakdown: p^T A p <= 0")
        a = rz / pq
        x += a * p
        r_old = r
        r = r - a * q
        it += 1
        hist.append(np.linalg.norm(r) / bn)
        if hist[-1] <= rtol:
            converged = True
            break
        z_new = Mop(r)
        rz_new = float(r @ z_new)
        hnat.append(np.sqrt(abs(rz_new)) / nat0)
        if flexible:
            beta = float(z_new @ (r - r_old)) / rz
        else:
            beta = rz_new / rz
        rz = rz_new
        p = z_new + beta * p
    return x, {"iterations": it, "history_l2": hist, "history_natural": hnat,
               "converged": converged}
