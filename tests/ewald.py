"""Textbook Ewald sum for point charges in a cubic periodic box (test pin only).

E = E_real + E_recip + E_self with splitting parameter alpha:
  E_real  = 1/2 sum_{i != j or n != 0} q_i q_j erfc(alpha r)/r
  E_recip = (2 pi / V) sum_{k != 0} exp(-k^2 / 4 alpha^2) / k^2 |S(k)|^2
  E_self  = -alpha / sqrt(pi) sum_i q_i^2
  E_bg    = -pi (sum_i q_i)^2 / (2 V alpha^2)   (neutralising background)
in Gaussian units (multiply by k_e for eV). Independent of the oracle.
"""
import itertools
import math

import numpy as np
from scipy.special import erfc


def ewald(pos, q, L, alpha=None, nimg=2, kmax=10):
    n = len(q)
    alpha = alpha if alpha is not None else 5.0 / L
    E_real = 0.0
    F = np.zeros((n, 3))
    shifts = np.array(list(itertools.product(range(-nimg, nimg + 1), repeat=3)), dtype=float) * L
    for i in range(n):
        d = pos[i] - pos  # (n,3)
        for s in shifts:
            dd = d + s
            r = np.sqrt((dd * dd).sum(1))
            m = r > 1e-12
            rr = r[m]
            E_real += 0.5 * q[i] * np.sum(q[m] * erfc(alpha * rr) / rr)
            g = (erfc(alpha * rr) / rr ** 2 + 2 * alpha / math.sqrt(math.pi) * np.exp(-(alpha * rr) ** 2) / rr) / rr
            F[i] += q[i] * np.sum((q[m] * g)[:, None] * dd[m], axis=0)
    V = L ** 3
    E_rec = 0.0
    ks = np.array([k for k in itertools.product(range(-kmax, kmax + 1), repeat=3) if any(k)], dtype=float)
    kv = 2 * math.pi * ks / L
    k2 = (kv * kv).sum(1)
    f = np.exp(-k2 / (4 * alpha * alpha)) / k2
    phase = pos @ kv.T                      # (n, K)
    S = (q[:, None] * np.exp(1j * phase)).sum(0)
    E_rec = (2 * math.pi / V) * float(np.sum(f * np.abs(S) ** 2))
    # F_i = (4 pi q_i / V) sum_k k f(k) Im(exp(i k.r_i) S*(k))
    im = np.imag(np.exp(1j * phase) * np.conj(S)[None, :])
    F += (4 * math.pi / V) * q[:, None] * ((im * f[None, :]) @ kv)
    E_self = -alpha / math.sqrt(math.pi) * float(np.sum(q * q))
    # uniform neutralising background for a charged box (k = 0 term of the sum)
    E_bg = -math.pi * float(np.sum(q)) ** 2 / (2.0 * V * alpha * alpha)
    return E_real + E_rec + E_self + E_bg, F
