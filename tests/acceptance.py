"""The library's acceptance test of an integrand value, restated for the tests
(Sec. IV.A, Eq. eq_interval_accept, library reading): a sample's value is
kept when its certified rounding-error bound E, carried to y = I/g like I,
is at most tol * max(|y|, floor).  The FP64 dump returns E at the FP64 unit,
the double-double dump at its own unit, so one function serves both."""
import numpy as np

from oracle.estimate import weight

TOL = 1e-10


def scaled(x, lg):
    """x / g for each sample, with g = 2^lg (the oracle's weight)."""
    return np.array([weight(float(a), float(b)) for a, b in zip(x, lg)])


def rejected(y, E, lg, tol=TOL, floor=0.0):
    Ey = scaled(E, lg)
    with np.errstate(invalid="ignore", over="ignore"):
        bad = ~np.isfinite(y) | ~np.isfinite(Ey)
        if tol > 0:
            bad |= Ey > tol * np.maximum(np.abs(y), floor)
    return bad


def bound_holds(I_got, E, I_exact):
    """|I_got - I_exact| <= E on every finite sample; the exact value is the
    oracle's rational result rounded once to double, hence the 2^-52 |I|."""
    fin = np.isfinite(I_got)
    err = np.abs(I_got - I_exact)[fin]
    return bool(np.all(err <= E[fin] + 2.0 ** -52 * np.abs(I_exact[fin])))
