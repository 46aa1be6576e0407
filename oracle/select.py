"""Adaptive coefficient filtering (oracle, test infrastructure only).

Supp. Sec. 1 ("Adaptive Filter Strategy"):
  1.1 budget:  E_{j,o} = sum_k |A_{j,o,k,c_ref}|^2 with c_ref = alpha,
               N_{j,o} = #k,  S = E^a N^b,
               K_{j,o} = max(10, floor(K_tot S / sum S))
  1.2 joint magnitude  v(k) = || A_{j,o,k,(R,G,B,alpha)} ||_2
  1.3 MAD threshold    sigma = median|v - median v| / 0.6745,  T = lambda sigma,
                       C = {k : v(k) >= T}
  1.4 top-K            K' = min(K_{j,o}, |C|),  keep v(k) >= max(T, v_(K'))
Readings where the supplement is silent or garbled:
  * a, b and lambda are not given: a = b = 0.5, lambda = 3 (the exponent
    symbol also collides with the opacity alpha in the text).
  * max(10, .) can push sum K above K_tot; the max is kept as written.
  * Median of an even count is the mean of the two middle values.
  * Ties at v_(K') are all kept (literal ">="), so a count can exceed K'.
  * If C is empty nothing is kept.
  * Only non-zero coefficients are kept: Sec. 4.3 states that every retained
    index corresponds to a non-zero coefficient (this also stops a zero
    threshold from keeping whole empty regions).
  * The sparse encoding keeps all four channels per index (the supplement
    writes vals in R^K; RGBA needs R^{K x 4}).

Precision: with dtype=float64 everything is FP64.  With dtype=float32 every
operation that decides which index is kept (v, the medians, sigma, T) is
taken in IEEE float32 in a fixed order -- v = sqrt(((a0 a0 + a1 a1) + a2 a2)
+ a3 a3), each product and sum rounded -- so that a float32 kernel taking the
same decision in the same precision can be compared index for index.
"""

import math

import numpy as np


def allocate_budget(E, N, K_tot, alpha_E=0.5, beta_N=0.5, min_per_band=10):
    """Per-subband counts K_{j,o} (Supp. Sec. 1.1); E, N lists in subband order."""
    E = np.asarray(E, dtype=np.float64)
    N = np.asarray(N, dtype=np.float64)
    S = E ** alpha_E * N ** beta_N
    total = S.sum()
    out = []
    for s in S:
        share = K_tot * s / total if total > 0 else 0.0
        out.append(max(min_per_band, int(math.floor(share))))
    return out


def joint_magnitude(A, dtype=np.float64):
    """v(k) for A of shape (4, ...) (Supp. Sec. 1.2)."""
    A = np.asarray(A, dtype=dtype)
    acc = A[0] * A[0]
    for c in range(1, 4):
        acc = acc + A[c] * A[c]
    return np.sqrt(acc)


def median(values, dtype=np.float64):
    """Textbook median: middle of the sorted values, mean of the two middles if even."""
    s = np.sort(np.asarray(values, dtype=dtype).reshape(-1))
    n = s.size
    if n % 2 == 1:
        return s[n // 2]
    half = dtype(0.5)
    return (s[n // 2 - 1] + s[n // 2]) * half


def select_subband(A, K, lam=3.0, dtype=np.float64):
    """Keep mask (shape A.shape[1:]) for one subband's coefficients A (4, ...).

    Returns (mask, info) with info = dict(T, sigma, K_eff, vK, n_candidates).
    """
    v = joint_magnitude(A, dtype)
    med = median(v, dtype)
    mad = median(np.abs(v - med), dtype)
    sigma = dtype(mad / dtype(0.6745))
    T = dtype(dtype(lam) * sigma)
    cand = v >= T
    n_c = int(cand.sum())
    K_eff = min(int(K), n_c)
    if K_eff == 0:
        return np.zeros(v.shape, dtype=bool), dict(T=T, sigma=sigma, K_eff=0, vK=None,
                                                   n_candidates=n_c)
    vals = np.sort(v[cand].reshape(-1))[::-1]
    vK = vals[K_eff - 1]
    thr = max(T, vK)
    mask = (v >= thr) & (v > 0)
    return mask, dict(T=T, sigma=sigma, K_eff=K_eff, vK=vK, n_candidates=n_c)
