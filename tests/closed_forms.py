"""Closed forms of the underlying Fokker-Planck model used as references by
the tests (no part of the method's discretisation)."""
import numpy as np
from scipy.linalg import expm


def shear(s, rate):
    k = np.zeros((s, s))
    k[0, 1] = rate
    return k


def dumbbell_cov_exact(rate, t, s=3, H=1.0, zeta=4.0, kBT=1.0):
    """Second moments <q q^T>(t) of the Hookean dumbbell Fokker-Planck equation
    (Sec. 2.1, one bond, A = 2) in simple shear, from <q q^T>(0) = (kBT/H) I:
    the moment equation C' = L C + C L^T + (4 kBT / zeta) I with
    L = kappa - (2H/zeta) I, solved exactly by the matrix exponential of the
    augmented linear system."""
    a = 2.0 * H / zeta
    L = shear(s, rate) - a * np.eye(s)
    n = s * s
    aug = np.zeros((n + 1, n + 1))
    aug[:n, :n] = np.kron(np.eye(s), L) + np.kron(L, np.eye(s))
    aug[:n, n] = (4.0 * kBT / zeta) * np.eye(s).ravel()
    x0 = np.append(np.eye(s).ravel() * kBT / H, 1.0)
    return (expm(aug * t) @ x0)[:n].reshape(s, s)
