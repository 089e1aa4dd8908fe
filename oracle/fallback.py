"""FP64 reference of the surrogate's MD-fallback decision -- TEST INFRASTRUCTURE.

Only the test suite may use this module; the CUDA library never imports it and
shares no code with it.  The paper runs MD at every quadrature point (Sec. 2.1,
Fig. 1); the learned surrogate with an MD fallback is an addition of the
hot-path specification, whose readings are followed here:

* Ensemble indicator: K members predict the stress sigma_k (6 Voigt
  components) of a point; the indicator is the norm of the per-component
  sample standard deviation over the members divided by the norm of the member
  mean, the latter floored at s_floor:
      spread = || std_k sigma_k || / max(|| mean_k sigma_k ||, s_floor).
* Decision per point and increment:
    - "tripped" (flag 1) when the spread exceeds spread_on, or when the point
      was tripped at the previous increment and its spread still exceeds
      spread_off (hysteresis: it stays on MD until the spread falls to
      spread_off or below);
    - otherwise "forced" (flag 2) when MD is forced for every point (the
      first increments, so that each r-cell has an MD state to fall back to);
    - otherwise the surrogate (flag 0).
  A spread that is not a number trips (the comparison "spread <= threshold"
  fails for it), so an undefined indicator always falls back to MD.
* Stress used by the FE update: the MD first Piola-Kirchhoff stress where the
  flag is nonzero, otherwise P = J sigma F^{-T} of the ensemble-mean Cauchy
  stress sigma (Eq. Pmd).
"""
from __future__ import annotations

import numpy as np

SURROGATE, TRIPPED, FORCED = 0, 1, 2


def ensemble_stats(S, s_floor):
    """S: (K, n, 6) member predictions.  Returns the mean (n, 6) and the spread (n,)."""
    S = np.asarray(S, dtype=np.float64)
    K = S.shape[0]
    mean = S.mean(axis=0)
    if K > 1:
        var = ((S - mean) ** 2).sum(axis=0) / (K - 1)
    else:
        var = np.zeros_like(mean)
    spread = np.sqrt(var.sum(axis=-1)) / np.maximum(np.linalg.norm(mean, axis=-1), s_floor)
    return mean, spread


def decide(spread, prev_flag, spread_on, spread_off, force_md):
    """Fallback flag of every point for this increment (see the module text)."""
    spread = np.asarray(spread, dtype=np.float64)
    prev = np.asarray(prev_flag)
    out = np.empty(spread.shape, dtype=np.int32)
    for i in range(spread.size):
        s = spread.flat[i]
        above_on = not (s <= spread_on)
        stays = prev.flat[i] == TRIPPED and not (s <= spread_off)
        if above_on or stays:
            out.flat[i] = TRIPPED
        elif force_md:
            out.flat[i] = FORCED
        else:
            out.flat[i] = SURROGATE
    return out


def cauchy_to_pk1(F, s_voigt):
    """P = J sigma F^{-T} for a Voigt Cauchy stress (xx yy zz xy xz yz), Eq. Pmd."""
    F = np.asarray(F, dtype=np.float64).reshape(3, 3)
    s = np.asarray(s_voigt, dtype=np.float64)
    sig = np.array([[s[0], s[3], s[4]], [s[3], s[1], s[5]], [s[4], s[5], s[2]]])
    return np.linalg.det(F) * sig @ np.linalg.inv(F).T


def merge_P(flags, s_mean, F, P_md):
    """Per point: the MD stress where flagged, the surrogate's P elsewhere."""
    n = len(flags)
    P = np.zeros((n, 3, 3))
    for e in range(n):
        P[e] = np.asarray(P_md[e]).reshape(3, 3) if flags[e] else cauchy_to_pk1(F[e], s_mean[e])
    return P
