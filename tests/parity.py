"""Comparison helpers for GPU-versus-oracle parity (test helper, no method arithmetic).

Tolerances (stated readings of the paper, see the design notes):
  * eigenvalues within 1e-10 ||H||, residuals ||H y - theta y|| <= 1e-10 ||H||;
  * the same eigenvalue set in the window, except that when the nev-th and (nev+1)-th distances
    to sigma differ by <= 1e-10 ||H|| either member is accepted;
  * observables within 1e-8 for eigenvectors with ||res|| / gap <= 1e-9 (Davis-Kahan: the
    eigenvector error is bounded by residual / gap); other eigenvectors are compared through
    their eigenvalues only.
"""
import numpy as np

EIG_TOL = 1e-10
OBS_TOL = 1e-8


def match_windows(ev_gpu, ev_orc, hnorm, tol=EIG_TOL):
    """Return the max |difference| after pairing ascending windows (asserts equal sizes)."""
    ev_gpu = np.sort(np.asarray(ev_gpu))
    ev_orc = np.sort(np.asarray(ev_orc))
    assert ev_gpu.shape == ev_orc.shape
    d = np.abs(ev_gpu - ev_orc)
    return d.max() / hnorm


def window_equivalent(ev_gpu, spectrum, sigma, nev, hnorm, tol=EIG_TOL):
    """Check ev_gpu is a valid nearest-nev window of the full (or larger) oracle spectrum."""
    spectrum = np.sort(np.asarray(spectrum))
    dist = np.abs(spectrum - sigma)
    order = np.lexsort((spectrum, dist))
    want = np.sort(spectrum[order[:nev]])
    ev_gpu = np.sort(np.asarray(ev_gpu))
    if np.abs(ev_gpu - want).max() <= tol * hnorm:
        return True
    # tie at the window edge: every GPU value must be within tol of some spectrum value whose
    # distance does not exceed the nev-th distance by more than tol
    edge = dist[order[nev - 1]]
    for x in ev_gpu:
        j = np.argmin(np.abs(spectrum - x))
        if abs(spectrum[j] - x) > tol * hnorm or dist[j] > edge + tol * hnorm:
            return False
    return len(np.unique(np.round(ev_gpu / (tol * hnorm)))) == nev


def well_conditioned(evals_all, evals, resid, guard=1e-9):
    """Mask of eigenvectors whose residual / gap (to the rest of the spectrum) is <= guard."""
    evals_all = np.sort(np.asarray(evals_all))
    mask = np.zeros(len(evals), dtype=bool)
    for j, (x, r) in enumerate(zip(evals, resid)):
        others = evals_all[np.abs(evals_all - x) > 1e-14 * max(1.0, abs(x))]
        gap = np.min(np.abs(others - x)) if len(others) else np.inf
        # an exact degeneracy (another eigenvalue within 1e-14) leaves the vector undefined
        close = np.sum(np.abs(evals_all - x) <= 1e-14 * max(1.0, abs(x)))
        mask[j] = close == 1 and (r / gap if gap > 0 else np.inf) <= guard
    return mask
