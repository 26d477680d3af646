"""BFGS fit of the parameters (Section II.B, eq. 7) and fitting errors (the check_errors
report) -- test infrastructure.

The paper minimises the loss of eq. 7 with BFGS and reports fitting errors; it gives no
further detail.  Reading used here (and by the library's driver):
  * variables u = theta / D with D_p = max(|theta0_p|, 1e-12 max|theta0|) (1 if theta0 = 0):
    the parameters span many orders of magnitude;
  * textbook BFGS on u with the inverse-Hessian update H <- (I - r s y^T) H (I - r y s^T)
    + r s s^T, r = 1 / (s.y), skipped when s.y <= 0 (Nocedal & Wright, Algorithm 6.1);
    H starts as I and is rescaled to (s.y / y.y) I just before the first update;
  * backtracking Armijo line search: step 1, halved up to 40 times until
    L(u + t d) <= L(u) + 1e-4 t g.d; no acceptable step ends the fit;
  * stop when max|g_u| <= gtol max(1, |L|) or after max_iter accepted steps.
Errors: energy per atom |E_k - E*_k| / N_k (max, mean, RMS over configurations), force
|F_i - F*_i| (max, mean, RMS over atoms), virial |W_ab - W*_ab| (max, mean, RMS over
configurations and components).
"""
from __future__ import annotations

import numpy as np


def scales(theta0):
    a = np.abs(np.asarray(theta0, np.float64))
    top = a.max() if a.size else 0.0
    if top == 0.0:
        return np.ones_like(a)
    return np.maximum(a, 1e-12 * top)


def bfgs(loss_grad, theta0, max_iter=50, gtol=1e-8):
    """loss_grad(theta) -> (L, dL/dtheta).  Returns (theta, L, accepted steps)."""
    D = scales(theta0)
    u = np.asarray(theta0, np.float64) / D
    L, g = loss_grad(D * u)
    g = D * g
    H = None
    it = 0
    while it < max_iter:
        if np.abs(g).max() <= gtol * max(1.0, abs(L)):
            break
        d = -(H @ g) if H is not None else -g
        gd = float(g @ d)
        t = 1.0
        ok = False
        for _ in range(41):
            un = u + t * d
            Ln, gn = loss_grad(D * un)
            if Ln <= L + 1e-4 * t * gd:
                ok = True
                break
            t *= 0.5
        if not ok:
            break
        gn = D * gn
        s = un - u
        y = gn - g
        sy = float(s @ y)
        if H is None:
            H = np.eye(len(u)) * (sy / float(y @ y) if sy > 0 else 1.0)
        if sy > 0:
            r = 1.0 / sy
            V = np.eye(len(u)) - r * np.outer(s, y)
            H = V @ H @ V.T + r * np.outer(s, s)
        u, L, g = un, Ln, gn
        it += 1
    return D * u, L, it


def errors(E, F, W, E_ref, F_ref, W_ref, atom_offset):
    n = np.diff(atom_offset).astype(np.float64)
    de = np.abs(E - E_ref) / np.maximum(n, 1.0)
    df = np.sqrt(((F - F_ref) ** 2).sum(axis=1))
    out = [de.max(initial=0.0), de.mean() if de.size else 0.0, np.sqrt((de ** 2).mean()) if de.size else 0.0,
           df.max(initial=0.0), df.mean() if df.size else 0.0, np.sqrt((df ** 2).mean()) if df.size else 0.0]
    if W_ref is None:
        out += [0.0, 0.0, 0.0]
    else:
        dw = np.abs(W - W_ref).ravel()
        out += [dw.max(initial=0.0), dw.mean() if dw.size else 0.0, np.sqrt((dw ** 2).mean()) if dw.size else 0.0]
    return np.array(out)
