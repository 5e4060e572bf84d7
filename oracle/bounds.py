"""Rounding-error quantities of Section 4, test infrastructure only.

gamma_n(u)  = n u / (1 - n u)                                  (Section 4)
eps_A       = sqrt(n) gamma_n^h        backward error of fl(A x), Eq. (er-Ax-ge)
eps_r       = (gamma_n^h + eps_A + gamma_n^h eps_A + (n+1) u_h)
              (1 + u_h)/(1 - 2 n u_h) + eps_A + u_h            (Lemma 1)
eps_T       = 4 n (3n + 1) kappa(A) u_l                        (Lemma 2)
Lemma 2:      || I - A^1/2 T_E A^1/2 ||_2 <= eps_T / (1 - eps_T)  when eps_T < 1
Theorem 1:    gamma = ||I - A^1/2 T_E A^1/2|| + gamma_2^h ||T_E|| ||A||
                      + beta(x) (u_h + (1 + gamma_2^h) eps_r ||T_E|| ||A||)
              beta(x) = max( sqrt(l1 ln)/(rho - l1), sqrt(l2 ln)/(l2 - rho) )
              and, if gamma < 1 and l1 < rho(x_i) < l2,
              q(x_{i+1}) <= (gamma + (1-gamma) l1/l2)^2 q(x_i),
              q(x) = (rho(x) - l1)/(l2 - rho(x)).
"""
from __future__ import annotations

import math

import numpy as np

U_H = 2.0 ** -53
U_L = 2.0 ** -24


def gamma_n(n, u):
    return n * u / (1.0 - n * u)


def eps_A(n, u_h=U_H):
    return math.sqrt(n) * gamma_n(n, u_h)


def eps_r(n, u_h=U_H):
    g = gamma_n(n, u_h)
    ea = eps_A(n, u_h)
    return (g + ea + g * ea + (n + 1) * u_h) * (1 + u_h) / (1 - 2 * n * u_h) + ea + u_h


def eps_T(n, kappa, u_l=U_L):
    return 4.0 * n * (3 * n + 1) * kappa * u_l


def lemma2_bound(n, kappa, u_l=U_L):
    e = eps_T(n, kappa, u_l)
    return e / (1.0 - e) if e < 1 else math.inf


def sqrtm_spd(A):
    w, V = np.linalg.eigh(A)
    return (V * np.sqrt(w)) @ V.conj().T


def precond_gap(A, T_E):
    """|| I - A^1/2 T_E A^1/2 ||_2 for explicit matrices."""
    S = sqrtm_spd(A)
    M = np.eye(A.shape[0]) - S @ T_E @ S
    return float(np.linalg.norm(0.5 * (M + M.conj().T), 2))


def beta(rho, lam):
    l1, l2, ln = lam[0], lam[1], lam[-1]
    return max(math.sqrt(l1 * ln) / (rho - l1), math.sqrt(l2 * ln) / (l2 - rho))


def theorem1_gamma(A, T_E, rho, lam, u_h=U_H):
    n = A.shape[0]
    g2 = gamma_n(2, u_h)
    nT = float(np.linalg.norm(T_E, 2))
    nA = float(lam[-1])
    return (precond_gap(A, T_E) + g2 * nT * nA
            + beta(rho, lam) * (u_h + (1 + g2) * eps_r(n, u_h) * nT * nA))


def q_ratio(rho, lam):
    return (rho - lam[0]) / (lam[1] - rho)
