"""FP64 CPU oracle of the VDS hot path (arXiv 2603.12550).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.  It
shares no code with the CUDA library.

Parts:
  * ``vds_oracle.c`` (compiled here with gcc, FP64, OpenMP over particles):
    density, entropy gradient, energy, explicit and implicit steps, stress,
    median pair distance, pair counts, reduced-order refresh sums.
  * this module (numpy, FP64): the density estimate at query points and
    Appendix A's grid density error, Silverman bandwidth, POD by the method of
    snapshots, project/lift, the linearised reduced step, err_MOR, the batched
    work-queue order.

Pins (tests/test_oracle_*.py) tie every function to something other than
itself: library densities, closed forms, invariants, finite differences,
linear special cases solved by numpy, and brute force on tiny inputs.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vds_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_lib = None

OR_OK, OR_EARG, OR_EDOMAIN, OR_ENOCONV = 0, -1, -3, -4


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle status {code}")
        self.code = code


def _so_path():
    with open(_SRC, "rb") as f:
        tag = hashlib.sha1(f.read()).hexdigest()[:12]
    return os.path.join(_BUILD, f"liboracle_{tag}.so")


def build() -> str:
    """Compile vds_oracle.c (gcc, -O2, OpenMP, strict IEEE FP64) if needed."""
    path = _so_path()
    if not os.path.exists(path):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-fno-fast-math", "-std=c11", "-D_GNU_SOURCE",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, path)
    return path


class OrParams(ctypes.Structure):
    _fields_ = [("spring", ctypes.c_int), ("nb", ctypes.c_int), ("s", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("H", ctypes.c_double * 8),
                ("b", ctypes.c_double), ("kBT", ctypes.c_double),
                ("zeta", ctypes.c_double), ("h", ctypes.c_double),
                ("dt", ctypes.c_double), ("kappa", ctypes.c_double * 9),
                ("tol", ctypes.c_double), ("jfloor", ctypes.c_double)]


def params(nb, s, H=1.0, kBT=1.0, zeta=4.0, h=0.3, dt=0.0, kappa=None,
           spring=0, b=0.0, tol=1e-10, max_iter=50, jfloor=1e-14) -> OrParams:
    p = OrParams()
    p.spring, p.nb, p.s, p.max_iter = int(spring), int(nb), int(s), int(max_iter)
    Hs = np.broadcast_to(np.asarray(H, dtype=np.float64), (nb,))
    for j in range(nb):
        p.H[j] = float(Hs[j])
    p.b, p.kBT, p.zeta, p.h, p.dt, p.tol = float(b), float(kBT), float(zeta), float(h), float(dt), float(tol)
    p.jfloor = float(jfloor)
    k = np.zeros((s, s)) if kappa is None else np.asarray(kappa, dtype=np.float64).reshape(s, s)
    for c in range(s * s):
        p.kappa[c] = float(k.flat[c])
    return p


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            fp = ctypes.POINTER(ctypes.c_float)
            lp = ctypes.POINTER(ctypes.c_long)
            ip = ctypes.POINTER(ctypes.c_int)
            pp = ctypes.POINTER(OrParams)
            L, I, D = ctypes.c_long, ctypes.c_int, ctypes.c_double
            sig = {
                "or_density": [dp, L, I, D, dp],
                "or_entropy_grad": [dp, L, I, D, dp, dp],
                "or_energy_grad": [dp, L, I, pp, dp, dp, dp],
                "or_explicit_steps": [dp, L, I, pp, I],
                "or_implicit_steps": [dp, L, I, pp, I, ip],
                "or_stress": [dp, L, I, pp, dp, dp],
                "or_median_pairdist": [dp, L, I, dp],
                "or_count_pairs": [dp, L, I, D, lp, lp],
                "or_count_pairs_f32": [fp, L, I, ctypes.c_float, lp, lp],
                "or_refresh_sums": [dp, L, I, D, dp, dp, I, I, dp, dp, dp],
                "or_entropy_grad_rows": [dp, L, I, D, dp, lp, L, dp],
                "or_density_rows": [dp, L, I, D, lp, L, dp],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            lib.or_rouse.argtypes = [I, I]
            lib.or_rouse.restype = D
            lib.or_rouse_inv.argtypes = [I, I, I]
            lib.or_rouse_inv.restype = D
            _lib = lib
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(st):
    if st != OR_OK:
        raise OracleError(st)


# ------------------------------------------------------------ C-backed parts

def density(q, h):
    """rho_I = sum_J exp(-|q_I - q_J|^2 / 2h^2), self term included."""
    q, qp = _d(q)
    N, D = q.shape
    rho, rp = _d(np.empty(N))
    _check(_L().or_density(qp, N, D, h, rp))
    return rho


def entropy_grad(q, h, rho=None):
    """S_I = -(1/h^2) sum_J khat_IJ (q_I - q_J)(1/rho_I + 1/rho_J)."""
    q, qp = _d(q)
    N, D = q.shape
    if rho is None:
        rho = density(q, h)
    rho, rp = _d(rho)
    S, Sp = _d(np.empty((N, D)))
    _check(_L().or_entropy_grad(qp, N, D, h, rp, Sp))
    return S


def density_rows(q, h, rows):
    """rho_I for the particles in ``rows`` only (the same sums as density)."""
    q, qp = _d(q)
    N, D = q.shape
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    rho, rp = _d(np.empty(len(rows)))
    _check(_L().or_density_rows(qp, N, D, h, rows.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                                len(rows), rp))
    return rho


def density_at(q, h, y, chunk=16):
    """Kernel density estimate of the cloud q at the points y (Eq.
    model_DeteParAppr): f(y_J) = (1/N) sum_I (2 pi h^2)^(-D/2)
    exp(-|y_J - q_I|^2 / (2 h^2)), differences taken coordinate by coordinate
    in FP64."""
    q = np.asarray(q, dtype=np.float64)
    y = np.atleast_2d(np.asarray(y, dtype=np.float64))
    N, D = q.shape
    f = np.empty(y.shape[0])
    for a in range(0, y.shape[0], chunk):
        d = y[a:a + chunk, None, :] - q[None, :, :]
        f[a:a + chunk] = np.exp(-np.sum(d * d, axis=2) / (2.0 * h * h)).sum(axis=1)
    return f / N * (2.0 * np.pi * h * h) ** (-D / 2.0)


def grid_points(D, values=(-2.0, 0.0, 2.0)):
    """All points of the mesh values^D (Appendix A takes {-2, 0, 2}), the
    last coordinate varying fastest."""
    v = np.asarray(values, dtype=np.float64)
    return np.stack(np.meshgrid(*([v] * D), indexing="ij"), axis=-1).reshape(-1, D)


def density_error(f, f0):
    """Appendix A's l2 and l-infinity relative differences of two density
    estimates on the same points (f0 the reference)."""
    f, f0 = np.asarray(f, np.float64), np.asarray(f0, np.float64)
    return (float(np.sqrt(np.sum((f - f0) ** 2) / np.sum(f0 ** 2))),
            float(np.max(np.abs(f - f0)) / np.max(np.abs(f0))))


def entropy_grad_rows(q, h, rho, rows):
    """S_I for the particles in ``rows`` only (rho: density of all particles)."""
    q, qp = _d(q)
    N, D = q.shape
    rho, rp = _d(rho)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    S, Sp = _d(np.empty((len(rows), D)))
    _check(_L().or_entropy_grad_rows(qp, N, D, h, rp, rows.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                                     len(rows), Sp))
    return S


def spring_grad(q, p: OrParams):
    """grad Psi(q_I) per particle (Hookean or FENE), N x D."""
    q = np.asarray(q, dtype=np.float64)
    N, D = q.shape
    s, nb = p.s, p.nb
    qb = q.reshape(N, nb, s)
    H = np.array([p.H[j] for j in range(nb)])
    if p.spring == 0:
        f = np.broadcast_to(H, (N, nb))
    else:
        f = H[None, :] / (1.0 - (qb ** 2).sum(-1) / p.b)
    return (qb * f[:, :, None]).reshape(N, D)


def energy_grad(q, p: OrParams, want_grad=True):
    """Returns (E, g, rho): E = (1/N) sum [kBT ln f_h + Psi], g = N dE/dq."""
    q, qp = _d(q)
    N, D = q.shape
    E = ctypes.c_double()
    g, gp = _d(np.empty((N, D)))
    rho, rp = _d(np.empty(N))
    _check(_L().or_energy_grad(qp, N, D, ctypes.byref(p), ctypes.byref(E),
                               gp if want_grad else None, rp))
    return E.value, (g if want_grad else None), rho


def energy(q, p: OrParams):
    return energy_grad(q, p, want_grad=False)[0]


def explicit_steps(q, p: OrParams, nsteps):
    q = np.array(q, dtype=np.float64, copy=True)
    _, qp = _d(q)
    qp = q.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    N, D = q.shape
    _check(_L().or_explicit_steps(qp, N, D, ctypes.byref(p), int(nsteps)))
    return q


def implicit_steps(q, p: OrParams, nsteps, raise_on_error=True):
    """Returns (q_new, iters per step, status)."""
    q = np.array(q, dtype=np.float64, copy=True)
    qp = q.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    N, D = q.shape
    it = (ctypes.c_int * max(1, int(nsteps)))()
    st = _L().or_implicit_steps(qp, N, D, ctypes.byref(p), int(nsteps), it)
    if raise_on_error:
        _check(st)
    return q, np.array(it[:nsteps]), st


def stress(q, p: OrParams):
    """Returns (tau s x s, qq D x D)."""
    q, qp = _d(q)
    N, D = q.shape
    tau, tp = _d(np.empty((p.s, p.s)))
    qq, qqp = _d(np.empty((D, D)))
    _check(_L().or_stress(qp, N, D, ctypes.byref(p), tp, qqp))
    return tau, qq


def kramers(tau, p: OrParams):
    """Kramers form tau - n (N-1) kBT Id with n = 1 (Eq. experiments_equilibriumStress)."""
    return tau - p.nb * p.kBT * np.eye(p.s)


def median_pairdist(q):
    q, qp = _d(q)
    N, D = q.shape
    m = ctypes.c_double()
    _check(_L().or_median_pairdist(qp, N, D, ctypes.byref(m)))
    return m.value


def median_bandwidth(q):
    """h = med / sqrt(2 ln N) (Eq. model_bandwidth, natural log)."""
    N = q.shape[0]
    return median_pairdist(q) / np.sqrt(2.0 * np.log(N))


def median_pairdist_count(q):
    """The same lower median of the N(N-1)/2 pair distances (Eq.
    model_bandwidth) where sorting them does not fit in memory: the k-th
    smallest squared distance, k = (M-1)/2 + 1 counted from one, is the least
    r2 with #{J<K : |q_J - q_K|^2 <= r2} >= k.  Found by bisection on r2 over
    the doubles, each probe one FP64 pair count, until lo and hi are adjacent
    doubles; hi is then the order statistic itself."""
    q = np.asarray(q, dtype=np.float64)
    N = q.shape[0]
    M = N * (N - 1) // 2
    k = (M - 1) // 2 + 1
    lo, hi = 0.0, 1.0
    while count_pairs(q, hi)[1] < k:
        lo, hi = hi, 2.0 * hi
    if count_pairs(q, 0.0)[1] >= k:
        return 0.0
    while True:
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if count_pairs(q, mid)[1] >= k:
            hi = mid
        else:
            lo = mid
    return float(np.sqrt(hi))


def median_bandwidth_count(q):
    """median_bandwidth through median_pairdist_count (large N)."""
    return median_pairdist_count(q) / np.sqrt(2.0 * np.log(q.shape[0]))


def count_pairs(q, r2):
    q, qp = _d(q)
    N, D = q.shape
    lt, le = ctypes.c_long(), ctypes.c_long()
    _check(_L().or_count_pairs(qp, N, D, float(r2), ctypes.byref(lt), ctypes.byref(le)))
    return lt.value, le.value


def count_pairs_f32(q32, r2):
    q32 = np.ascontiguousarray(q32, dtype=np.float32)
    N, D = q32.shape
    lt, le = ctypes.c_long(), ctypes.c_long()
    _check(_L().or_count_pairs_f32(q32.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                   N, D, ctypes.c_float(r2), ctypes.byref(lt), ctypes.byref(le)))
    return lt.value, le.value


def rouse(nb):
    L = _L()
    return np.array([[L.or_rouse(j, k) for k in range(nb)] for j in range(nb)])


def rouse_inv(nb):
    L = _L()
    return np.array([[L.or_rouse_inv(j, k, nb) for k in range(nb)] for j in range(nb)])


def refresh_sums(q, h, rho, Phi, s):
    """(W1, W2, c) of the frozen Brownian terms; Phi is (N*s) x r."""
    q, qp = _d(q)
    N, D = q.shape
    Phi, up = _d(Phi)
    r = Phi.shape[1]
    rho, rp = _d(rho)
    W1, w1 = _d(np.empty((N * s, r)))
    W2, w2 = _d(np.empty((N * s, r)))
    c, cp = _d(np.empty(N))
    _check(_L().or_refresh_sums(qp, N, D, h, rp, up, s, r, w1, w2, cp))
    return W1, W2, c


# ------------------------------------------------------------ numpy parts

def silverman_bandwidth(q):
    """h = sigma (4 / ((D+2) N))^(1/(D+4)), sigma = mean per-coordinate sample
    standard deviation (ddof = 1).  Not in the paper (a common KDE rule)."""
    q = np.asarray(q, dtype=np.float64)
    N, D = q.shape
    sigma = np.mean(np.std(q, axis=0, ddof=1))
    return sigma * (4.0 / ((D + 2) * N)) ** (1.0 / (D + 4))


def snapshots_from_states(states, s, nb):
    """Snapshot matrix X of Sec. 3.1: one column per (snapshot l, bond k), l
    major; column = q_k(t_l) flattened as rows (I, alpha).  Shape (N s) x (L nb)."""
    cols = []
    for q in states:
        q = np.asarray(q, dtype=np.float64)
        N = q.shape[0]
        for k in range(nb):
            cols.append(q[:, s * k:s * k + s].reshape(N * s))
    return np.stack(cols, axis=1)


def pod_build(X, energy=0.9999, r_max=64, r_fixed=0):
    """POD by the method of snapshots (Sec. 2.3, Sec. 3.1): the nonzero
    eigenpairs of X X^T come from C = X^T X = V Lambda V^T as
    U = X V Lambda^{-1/2}.  Rank: r_fixed if > 0, else the smallest r with
    sum_{i<=r} lambda_i >= energy * sum_i lambda_i, capped at r_max.  Sign:
    the largest-magnitude entry of every column is positive (ties: lowest
    row).  Returns dict(Phi, lam (all, descending), r)."""
    X = np.asarray(X, dtype=np.float64)
    C = X.T @ X
    lam, V = np.linalg.eigh(C)
    order = np.argsort(-lam, kind="stable")
    lam, V = lam[order], V[:, order]
    r = int(r_fixed) if r_fixed > 0 else select_rank(lam, energy, r_max)
    Phi = X @ V[:, :r] / np.sqrt(lam[:r])
    for t in range(r):
        i = int(np.argmax(np.abs(Phi[:, t])))
        if Phi[i, t] < 0:
            Phi[:, t] = -Phi[:, t]
    return dict(Phi=Phi, lam=lam, r=r)


def select_rank(lam, energy, r_max):
    """Smallest r with cumulative energy fraction >= energy, capped at r_max."""
    lam = np.asarray(lam, dtype=np.float64)
    tot = lam.sum()
    cum = 0.0
    for i, l in enumerate(lam):
        cum += l
        if cum >= energy * tot:
            return min(i + 1, r_max)
    return min(len(lam), r_max)


def project(Phi, q, s, nb):
    """p_{k:} = U^T q_{k:} (Eq. model_pq); returns P (r x nb)."""
    q = np.asarray(q, dtype=np.float64)
    N = q.shape[0]
    Q = np.stack([q[:, s * k:s * k + s].reshape(N * s) for k in range(nb)], axis=1)
    return Phi.T @ Q


def lift(Phi, P, s, nb):
    """q~_{k:} = U p_{k:} (Eq. model_pq); returns N x (nb s)."""
    Q = Phi @ P
    N = Q.shape[0] // s
    return np.concatenate([Q[:, k].reshape(N, s) for k in range(nb)], axis=1)


def x_h(Phi, kappa, s):
    """X^H_st = sum_I sum_{alpha beta} U_(I alpha)s G_{alpha beta} U_(I beta)t (Sec. 2.4)."""
    N = Phi.shape[0] // s
    r = Phi.shape[1]
    U = Phi.reshape(N, s, r)
    GU = np.einsum("ab,Ibt->Iat", np.asarray(kappa, dtype=np.float64).reshape(s, s), U)
    return np.einsum("Ias,Iat->st", U, GU)


def x_b(Phi, q, h, s):
    """Frozen Brownian matrices of Sec. 2.4 at state q:
      X^B1_st = -(1/h^2) sum_(I a) U_(Ia)s sum_K Z_IK (U_(Ia)t - U_(Ka)t) / rho_I
      X^B2_st = -(1/h^2) sum_(I a) U_(Ia)s sum_K Z_IK (U_(Ia)t - U_(Ka)t) / rho_K
    with Z_IK the kernel and rho_I = sum_J Z_IJ.  Returns (XB1, XB2, rho)."""
    q = np.asarray(q, dtype=np.float64)
    N = q.shape[0]
    rho = density(q, h)
    W1, W2, c = refresh_sums(q, h, rho, Phi, s)
    r = Phi.shape[1]
    U = Phi.reshape(N, s, r)
    W1 = W1.reshape(N, s, r)
    W2 = W2.reshape(N, s, r)
    # sum_K Z_IK (U_(Ia)t - U_(Ka)t) = rho_I U_(Ia)t - W1_(Ia)t, since the row
    # sum of Z is rho_I; divided by rho_I for X^B1.
    inner1 = (rho[:, None, None] * U - W1) / rho[:, None, None]
    # sum_K Z_IK (U_(Ia)t - U_(Ka)t) / rho_K = c_I U_(Ia)t - W2_(Ia)t.
    inner2 = c[:, None, None] * U - W2
    t1 = np.einsum("Ias,Iat->st", U, inner1)
    t2 = np.einsum("Ias,Iat->st", U, inner2)
    return -t1 / h ** 2, -t2 / h ** 2, rho


def reduced_rhs(P, XH, XB, p: OrParams):
    """Right-hand side of Eq. model_DymReduced in matrix form (P is r x nb):
    Pdot = X^H P - (kBT/zeta) (X^B1 + X^B2) P A - (1/zeta) P diag(H) A."""
    nb = p.nb
    A = rouse(nb)
    H = np.array([p.H[j] for j in range(nb)])
    return XH @ P - (p.kBT / p.zeta) * (XB @ P @ A) - (1.0 / p.zeta) * (P * H[None, :]) @ A


def velocity(q, p: OrParams):
    """Full-order particle velocity of Eq. model_DymRepPar:
    v_{k,I} = kappa q_{k,I} - (1/zeta) sum_j A_kj g_{I,j}."""
    q = np.asarray(q, dtype=np.float64)
    N, D = q.shape
    s, nb = p.s, p.nb
    _, g, _ = energy_grad(q, p)
    A = rouse(nb)
    kap = np.array(p.kappa[:s * s]).reshape(s, s)
    qb = q.reshape(N, nb, s)
    gb = g.reshape(N, nb, s)
    v = np.einsum("ab,Ikb->Ika", kap, qb) - np.einsum("kj,Ija->Ika", A, gb) / p.zeta
    return v.reshape(N, D)


def velocity_rows(q, p: OrParams, rho, rows):
    """The particle velocity of Eq. model_DymRepPar for the particles in
    ``rows`` only, given the density rho of all particles:
    v_{k,I} = kappa q_{k,I} - (1/zeta) sum_j A_kj g_{I,j}, g = kBT S + grad Psi."""
    q = np.asarray(q, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    s, nb = p.s, p.nb
    g = p.kBT * entropy_grad_rows(q, p.h, rho, rows) + spring_grad(q[rows], p)
    A = rouse(nb)
    kap = np.array(p.kappa[:s * s]).reshape(s, s)
    n = len(rows)
    qb = q[rows].reshape(n, nb, s)
    gb = g.reshape(n, nb, s)
    v = np.einsum("ab,Ikb->Ika", kap, qb) - np.einsum("kj,Ija->Ika", A, gb) / p.zeta
    return v.reshape(n, nb * s)


def explicit_step_rows(q, p: OrParams, rho, rows):
    """One explicit Euler step (Appendix A) of the particles in ``rows``,
    given the density rho of all particles: q_I + dt v_I."""
    q = np.asarray(q, dtype=np.float64)
    return q[np.asarray(rows, dtype=np.int64)] + p.dt * velocity_rows(q, p, rho, rows)


def score_rhs(P, Phi, p: OrParams, layers):
    """Reduced RHS with the learned score in place of the entropy gradient:
    Pdot = U^T [kappa q~ - (1/zeta)(A (x) I)(kBT (s - mean s) + grad Psi)],
    q~ = U P, s = s_theta(q~) (FP64 forward of the given network), the mean
    taken over particles."""
    from . import mlp
    q = lift(Phi, P, p.s, p.nb)
    N, D = q.shape
    s, _ = mlp.forward(mlp.as64(layers), q)
    s = s - s.mean(axis=0)
    g = p.kBT * s + spring_grad(q, p)
    A = rouse(p.nb)
    kap = np.array(p.kappa[:p.s * p.s]).reshape(p.s, p.s)
    qb, gb = q.reshape(N, p.nb, p.s), g.reshape(N, p.nb, p.s)
    v = np.einsum("ab,Ikb->Ika", kap, qb) - np.einsum("kj,Ija->Ika", A, gb) / p.zeta
    return project(Phi, v.reshape(N, D), p.s, p.nb)


def galerkin_rhs(P, Phi, p: OrParams):
    """Mode i: Pdot = U^T v(U P) (Eq. model_DymRepParPod at the lifted state)."""
    q = lift(Phi, P, p.s, p.nb)
    return project(Phi, velocity(q, p), p.s, p.nb)


def reduced_run(P0, Phi, p: OrParams, nsteps, refresh_every):
    """Explicit Euler on Eq. model_DymReduced with X^B1, X^B2 frozen and
    rebuilt at the lifted state every ``refresh_every`` steps (Sec. 2.4,
    Sec. 3.2)."""
    s = p.s
    kap = np.array(p.kappa[:s * s]).reshape(s, s)
    XH = x_h(Phi, kap, s)
    P = np.array(P0, dtype=np.float64)
    XB = None
    for n in range(nsteps):
        if n % refresh_every == 0:
            q = lift(Phi, P, s, p.nb)
            B1, B2, _ = x_b(Phi, q, p.h, s)
            XB = B1 + B2
        P = P + p.dt * reduced_rhs(P, XH, XB, p)
    return P


def convect_upwind(Q, u, shape, dx, dt, bc=0):
    """One first-order upwind step of dQ/dt + u . grad_x Q = 0 (the
    convection term u . grad_x q of Eq. model_DymRepPar, u . grad_x p of Eq.
    model_DymReduced) on a structured grid nx x ny x nz of nodes, node
    g = ix + nx (iy + ny iz); Q is (G, M) (M values per node), u (G, 3).
    Each axis of extent > 1 contributes
      max(u_b, 0) (Q[g] - Q[g - e_b]) / dx_b + min(u_b, 0) (Q[g + e_b] - Q[g]) / dx_b,
    the neighbour beyond a boundary being the opposite boundary node (bc 0,
    periodic) or the boundary node itself (bc 1, zero gradient)."""
    nx, ny, nz = shape
    Q = np.asarray(Q, dtype=np.float64)
    M = Q.shape[1]
    F = Q.reshape(nz, ny, nx, M)
    U = np.asarray(u, dtype=np.float64).reshape(nz, ny, nx, 3)
    out = F.copy()
    for b, axis, n in ((0, 2, nx), (1, 1, ny), (2, 0, nz)):
        if n == 1:
            continue
        if bc == 0:
            lo, hi = np.roll(F, 1, axis=axis), np.roll(F, -1, axis=axis)
        else:
            idx = np.arange(n)
            lo = np.take(F, np.maximum(idx - 1, 0), axis=axis)
            hi = np.take(F, np.minimum(idx + 1, n - 1), axis=axis)
        ub = U[..., b][..., None]
        out = out - dt / dx[b] * (np.maximum(ub, 0.0) * (F - lo) + np.minimum(ub, 0.0) * (hi - F))
    return out.reshape(-1, M)


def err_mor(q_mor, q_ref):
    """Relative L2 MOR error (Sec. 3.1)."""
    q_mor = np.asarray(q_mor, dtype=np.float64)
    q_ref = np.asarray(q_ref, dtype=np.float64)
    return np.linalg.norm(q_mor - q_ref) / np.linalg.norm(q_ref)


def work_queue(sizes, tile):
    """Batched work items (e, itile) in longest-processing-time order: cost
    N_e descending, then ensemble index, then tile index ascending."""
    items = []
    for e, n in enumerate(sizes):
        for t in range((int(n) + tile - 1) // tile):
            items.append((-int(n), e, t))
    items.sort()
    return np.array([(e, t) for _, e, t in items], dtype=np.int32).reshape(-1, 2)
