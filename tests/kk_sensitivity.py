"""How far the oracle's own Kamada-Kawai result moves when its FP32 start
moves by one ulp (Section 3.1, Newton-Raphson sweeps from random starts).

A GPU run rounds every Newton step to FP32, so it can follow the FP64 oracle
only where the oracle's result does not hinge on rounding-sized changes of
its input.  `oracle_spread` runs the oracle from an FP32 start and from four
copies of it in which every coordinate moved by one FP32 ulp (up or down at
random, seeded), and reports how far the perturbed runs end from the
unperturbed one: a component whose spread exceeds the comparison tolerance
is one where the sweeps amplify rounding by that much, and only such a
component may differ from the oracle in a GPU comparison.  Test helper only
(oracle and numpy; no CUDA)."""
from __future__ import annotations

import numpy as np

import oracle

ULP_STARTS = 4


def ulp_starts(x32, y32, k=ULP_STARTS):
    """k copies of the FP32 start, each coordinate one ulp up or down."""
    x32 = np.asarray(x32, np.float32)
    y32 = np.asarray(y32, np.float32)
    for s in range(k):
        rng = np.random.default_rng(100 + s)

        def move(a):
            to = np.where(rng.random(len(a)) < 0.5, np.float32(-np.inf), np.float32(np.inf)).astype(np.float32)
            return np.nextafter(a, to).astype(np.float32)
        yield move(x32), move(y32)


def energy_close(e, e_ref):
    """KK energies agree: relative 1e-4, plus 1e-9 absolute for layouts whose
    minimum is exactly 0 (trees drawn with every distance realised)."""
    return abs(e - e_ref) <= 1e-4 * abs(e_ref) + 1e-9


def min_curvature_ratio(x32, y32, d, sweeps, l=1.0):
    """Replays the oracle's Gauss-Seidel sweeps node step by node step (its
    own gradient/Hessian and step routines, in its order) and returns the
    smallest |lambda_min| / |lambda_max| of the 2x2 Hessians it met, with the
    final positions (equal to oracle.kk_run's).  Below about 1e-4 the small
    curvature is a difference of near-equal FP32 terms (1 - l dx^2 / r^3 as
    the path straightens), which an FP32 Hessian cannot resolve, so an FP32
    run steps differently along that flat direction."""
    x = np.asarray(x32, np.float64).copy()
    y = np.asarray(y32, np.float64).copy()
    worst = np.inf
    for _ in range(sweeps):
        for m in range(len(x)):
            o = oracle.kk_grad_hess(x, y, d, l, m)
            H = [[o[2], o[3]], [o[3], o[4]]]
            ev = np.abs(np.linalg.eigvalsh(H))
            if ev.max() > 0:
                worst = min(worst, ev.min() / ev.max())
            st, moved = oracle.kk_step(o[:2], H, l)
            if moved:
                x[m] += st[0]
                y[m] += st[1]
    return worst, x, y


def oracle_spread(x32, y32, d, sweeps, l=1.0, k=ULP_STARTS):
    """Runs the oracle from the FP32 start and from k one-ulp moves of it.

    Returns ((x, y, energies) of the unperturbed run, the largest position
    difference of a perturbed run from it, and whether some perturbed run
    ends at an energy that energy_close rejects)."""
    ox, oy, e, _, _ = oracle.kk_run(np.asarray(x32, np.float64), np.asarray(y32, np.float64), d, l, sweeps)
    dp, other_energy = 0.0, False
    for xp, yp in ulp_starts(x32, y32, k):
        px, py, ep, _, _ = oracle.kk_run(xp.astype(np.float64), yp.astype(np.float64), d, l, sweeps)
        dp = max(dp, float(np.max(np.hypot(px - ox, py - oy))))
        if sweeps > 0 and not energy_close(ep[-1], e[-1]):
            other_energy = True
    return (ox, oy, e), dp, other_energy
