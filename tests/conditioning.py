"""Condition number of the even-odd normal operator for unit links, in closed
form; it scales the bound on a solve's error, ||x - x*|| / ||x*|| <= cond * r
for a relative residual r of the CG system (used by the parity tests).

A plane wave of momentum p diagonalises the free hop as the 4x4 spin matrix
h(p) = a - i K, a = 2 sum_mu cos p_mu, K = 2 sum_mu gamma_mu sin p_mu
(Hermitian, K^2 = |s|^2 with |s| = 2 sqrt(sum_mu sin^2 p_mu)).  h is normal,
with eigenvalues a -+ i|s|, and Mhat = 1 - kappa^2 H_eo H_oe acts on the even
sites as 1 - kappa^2 h^2, so its singular values are |1 - kappa^2 (a -+ i|s|)^2|
and cond(Mhat^dag Mhat) is the squared ratio of the largest to the smallest.
Momenta: p_mu = 2 pi n / L_mu, shifted by half a unit in time when the time
boundary is antiperiodic.
"""
import numpy as np


def free_singular_values(dims, kappa, t_antiperiodic=True):
    ps = []
    for mu, n in enumerate(dims):
        shift = 0.5 if (mu == 3 and t_antiperiodic) else 0.0
        ps.append(2 * np.pi * (np.arange(n) + shift) / n)
    P = np.meshgrid(*ps, indexing="ij")
    a = 2 * sum(np.cos(p) for p in P)
    s = 2 * np.sqrt(sum(np.sin(p) ** 2 for p in P))
    return np.concatenate([np.abs(1 - kappa ** 2 * (a - 1j * s) ** 2).ravel(),
                           np.abs(1 - kappa ** 2 * (a + 1j * s) ** 2).ravel()])


def free_cond_eo(dims, kappa, t_antiperiodic=True):
    sv = free_singular_values(dims, kappa, t_antiperiodic)
    return float((sv.max() / sv.min()) ** 2)
