"""Thin ctypes binding of the C ABI in include/vds.h.

Argument marshalling only: every computation runs in the CUDA library.  Device
arrays are passed as torch CUDA tensors (PyTorch provides device memory and
streams) or raw integer device addresses.  Importing this module loads the
compiled library and raises if it is missing -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

VDS_OK, VDS_EARG, VDS_ECUDA, VDS_EDOMAIN, VDS_ENOCONV = 0, -1, -2, -3, -4
VDS_ENAN, VDS_ETIMEOUT, VDS_ENOMEM, VDS_ESURROGATE, VDS_ESIZE = -5, -6, -7, -8, -9
VDS_NOALLOC_MAX_N = 8192
BATCH_CONFIGS = 4  # pair-kernel shapes of the batched tile autotuner
TIMING_KINDS = 7  # density, gradient, bandwidth, refresh, POD Gram, POD eigensolve, POD basis


class VdsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def _load():
    path = _build.library_path()
    if not os.path.exists(path):
        raise ImportError(
            f"CUDA library {path} is not built; run paper_2603_12550_gb300.build.build() "
            "(or __graft_entry__.build()) first")
    return ctypes.CDLL(path)


lib = _load()


class VdsParams(ctypes.Structure):
    _fields_ = [("spring", ctypes.c_int), ("nb", ctypes.c_int), ("s", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("H", ctypes.c_double * 8),
                ("b", ctypes.c_double), ("kBT", ctypes.c_double), ("zeta", ctypes.c_double),
                ("h", ctypes.c_double), ("dt", ctypes.c_double),
                ("kappa", ctypes.c_double * 9), ("tol", ctypes.c_double),
                ("jfloor", ctypes.c_double), ("scheme", ctypes.c_int),
                ("reserved", ctypes.c_int)]


def params(nb, s, H=1.0, kBT=1.0, zeta=4.0, h=0.3, dt=0.0, kappa=None, spring=0, b=0.0,
           tol=1e-6, max_iter=50, jfloor=1e-9, scheme=0) -> VdsParams:
    p = VdsParams()
    p.spring, p.nb, p.s, p.max_iter, p.scheme = int(spring), int(nb), int(s), int(max_iter), int(scheme)
    Hs = np.broadcast_to(np.asarray(H, dtype=np.float64), (nb,))
    for j in range(nb):
        p.H[j] = float(Hs[j])
    p.b, p.kBT, p.zeta, p.h, p.dt = float(b), float(kBT), float(zeta), float(h), float(dt)
    p.tol, p.jfloor = float(tol), float(jfloor)
    k = np.zeros((s, s)) if kappa is None else np.asarray(kappa, dtype=np.float64).reshape(s, s)
    for c in range(s * s):
        p.kappa[c] = float(k.flat[c])
    return p


_vp, _i, _l, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_long, ctypes.c_double
_pp = ctypes.POINTER(VdsParams)
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)

_SIGS = {
    "vds_create": ([ctypes.POINTER(_vp), _vp, _i], _i),
    "vds_destroy": ([_vp], None),
    "vds_set_stream": ([_vp, _vp], _i),
    "vds_strerror": ([_i], ctypes.c_char_p),
    "vds_bandwidth": ([_vp, _vp, _i, _i, _i, _dp], _i),
    "vds_energy_grad": ([_vp, _vp, _i, _i, _pp, _vp, _dp, _vp, _vp], _i),
    "vds_step": ([_vp, _vp, _i, _i, _pp, _i, _ip], _i),
    "vds_stress": ([_vp, _vp, _i, _i, _pp, _dp, _dp], _i),
    "vds_density_at": ([_vp, _vp, _i, _i, _pp, _vp, _i, _vp], _i),
    "vds_density_tc": ([_vp, _vp, _i, _i, _pp, _vp], _i),
    "vds_density_rows": ([_vp, _vp, _i, _i, _pp, _i, _i, _vp], _i),
    "vds_grad_rows": ([_vp, _vp, _i, _i, _pp, _vp, _i, _i, _i, _vp], _i),
    "vds_timing": ([_vp, _i], _i),
    "vds_wait_selftest": ([_vp, _d], _i),
    "vds_energy_grad_noalloc": ([_vp, _i, _i, _pp, _dp, _vp, _vp, _vp], _i),
    "vds_timing_read": ([_vp, _dp, ctypes.POINTER(_l), ctypes.POINTER(_l)], _i),
    "pod_build": ([_vp, _vp, _l, _i, _i, _d, _i, _i, _dp, ctypes.POINTER(_vp), _ip], _i),
    "pod_load": ([_vp, _vp, _l, _i, _i, _dp, ctypes.POINTER(_vp)], _i),
    "pod_sweeps": ([_vp], _i),
    "pod_info": ([_vp, _ip, _ip, ctypes.POINTER(_vp), ctypes.POINTER(_l)], _i),
    "pod_eigenvalues": ([_vp, _dp, _i], _i),
    "pod_xh": ([_vp, _dp], _i),
    "pod_project": ([_vp, _vp, _vp, _i, _i, _vp], _i),
    "pod_lift": ([_vp, _vp, _vp, _i, _i, _vp], _i),
    "pod_free": ([_vp], None),
    "vds_batch_create": ([_vp, _i, _ip, _i, _pp, _dp, _dp, ctypes.POINTER(_vp)], _i),
    "vds_batch_free": ([_vp], None),
    "vds_batch_info": ([_vp, ctypes.POINTER(_l), _ip, _ip], _i),
    "vds_batch_queue": ([_vp, _ip, _i], _i),
    "vds_batch_energy_grad": ([_vp, _vp, _vp, _dp, _vp, _vp], _i),
    "vds_batch_step": ([_vp, _vp, _vp, _i, _ip], _i),
    "vds_batch_autotune": ([_vp, _vp, _vp, _i, _ip, _dp], _i),
    "vds_batch_stress": ([_vp, _vp, _vp, _dp], _i),
    "vds_batch_set_kappa": ([_vp, _vp, _dp], _i),
    "vds_convect": ([_vp, _vp, _vp, _i, _i, _i, _l, _vp, _dp, _d, _i], _i),
    "vds_batch_set_config": ([_vp, _vp, _i], _i),
    "vds_batch_get_config": ([_vp, _ip], _i),
    "vds_score_param_count": ([_i, _i], _l),
    "vds_score_create": ([_vp, _i, _i, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_vp)], _i),
    "vds_score_free": ([_vp], None),
    "vds_score_set_params": ([_vp, _vp, ctypes.POINTER(ctypes.c_float)], _i),
    "vds_score_get_params": ([_vp, _vp, ctypes.POINTER(ctypes.c_float)], _i),
    "vds_score_eval": ([_vp, _vp, _vp, _i, _vp], _i),
    "vds_score_loss_grad": ([_vp, _vp, _vp, _vp, _vp, _i, _d, _dp, ctypes.POINTER(ctypes.c_float)], _i),
    "vds_score_train": ([_vp, _vp, _vp, _vp, _vp, _i, _d, _d, _dp], _i),
    "vds_score_fit": ([_vp, _vp, _vp, _vp, _vp, _i, _d, _dp, ctypes.POINTER(ctypes.c_float)], _i),
    "pod_step_score": ([_vp, _vp, _vp, _vp, _i, _i, _pp, _i, _i, _i, _d, _dp, _ip], _i),
    "pod_brownian": ([_vp, _vp, _vp, _i, _i, _pp, _dp, _dp], _i),
    "pod_step": ([_vp, _vp, _vp, _i, _i, _pp, _i, _i, _i], _i),
}
for _name, (_args, _res) in _SIGS.items():
    if hasattr(lib, _name):
        _f = getattr(lib, _name)
        _f.argtypes = _args
        _f.restype = _res


def exported_symbols():
    return [n for n in _SIGS if hasattr(lib, n)]


def strerror(code) -> str:
    return lib.vds_strerror(int(code)).decode()


def _check(code):
    if code != VDS_OK:
        raise VdsError(code, strerror(code))


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return getattr(stream, "cuda_stream", stream)


def energy_grad_noalloc(q, p: VdsParams, g=None, rho=None, want_energy=True, stream=None):
    """vds_energy_grad_noalloc: the allocation-free evaluation (no context);
    returns E (or None)."""
    N, D = q.shape
    E = ctypes.c_double()
    _check(lib.vds_energy_grad_noalloc(_ptr(q), N, D, ctypes.byref(p),
                                       ctypes.byref(E) if want_energy else None, _ptr(g), _ptr(rho),
                                       _stream_handle(stream)))
    return E.value if want_energy else None


class Context:
    """Owns a vds_ctx bound to a device and stream."""

    def __init__(self, device: int = 0, stream=None):
        h = _vp()
        _check(lib.vds_create(ctypes.byref(h), _stream_handle(stream), int(device)))
        self.h = h

    def close(self):
        if self.h:
            lib.vds_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        _check(lib.vds_set_stream(self.h, _stream_handle(stream)))

    # -- calls (names follow include/vds.h) --------------------------------
    def vds_timing(self, enable=True):
        _check(lib.vds_timing(self.h, 1 if enable else 0))

    def vds_timing_read(self):
        ms = (ctypes.c_double * TIMING_KINDS)()
        n = (ctypes.c_long * TIMING_KINDS)()
        tot = ctypes.c_long()
        _check(lib.vds_timing_read(self.h, ms, n, ctypes.byref(tot)))
        return list(ms), list(n), tot.value

    def vds_wait_selftest(self, limit_s=0.05) -> int:
        """Status of two bounded waits that nothing completes (VDS_ETIMEOUT)."""
        return int(lib.vds_wait_selftest(self.h, float(limit_s)))

    def vds_bandwidth(self, q, rule=0) -> float:
        N, D = q.shape
        h = ctypes.c_double()
        _check(lib.vds_bandwidth(self.h, _ptr(q), N, D, int(rule), ctypes.byref(h)))
        return h.value

    def vds_energy_grad(self, q, p: VdsParams, g=None, rho=None, q_star=None, want_energy=True):
        N, D = q.shape
        E = ctypes.c_double()
        _check(lib.vds_energy_grad(self.h, _ptr(q), N, D, ctypes.byref(p), _ptr(q_star),
                                   ctypes.byref(E) if want_energy else None, _ptr(g), _ptr(rho)))
        return E.value if want_energy else None

    def vds_step(self, q, p: VdsParams, nsteps=1, want_iters=False):
        N, D = q.shape
        it = (ctypes.c_int * max(1, nsteps))() if want_iters else None
        code = lib.vds_step(self.h, _ptr(q), N, D, ctypes.byref(p), int(nsteps), it)
        _check(code)
        return list(it[:nsteps]) if want_iters else None

    def vds_stress(self, q, p: VdsParams):
        N, D = q.shape
        tau = (ctypes.c_double * 9)()
        qq = (ctypes.c_double * (D * D))()
        _check(lib.vds_stress(self.h, _ptr(q), N, D, ctypes.byref(p), tau, qq))
        s = p.s
        return (np.array(tau[:s * s]).reshape(s, s), np.array(qq[:]).reshape(D, D))

    def vds_density_at(self, q, p: VdsParams, y, f):
        """f[J] = kernel density estimate of the cloud q at query point y[J]."""
        N, D = q.shape
        M = int(y.shape[0])
        _check(lib.vds_density_at(self.h, _ptr(q), N, D, ctypes.byref(p), _ptr(y), M, _ptr(f)))

    def vds_density_tc(self, q, p: VdsParams, rho):
        N, D = q.shape
        _check(lib.vds_density_tc(self.h, _ptr(q), N, D, ctypes.byref(p), _ptr(rho)))

    def vds_density_rows(self, q, p: VdsParams, row0, nrows, rho_rows):
        N, D = q.shape
        _check(lib.vds_density_rows(self.h, _ptr(q), N, D, ctypes.byref(p), int(row0), int(nrows),
                                    _ptr(rho_rows)))

    def vds_grad_rows(self, q, p: VdsParams, rho, row0, nrows, out, mode=0):
        N, D = q.shape
        _check(lib.vds_grad_rows(self.h, _ptr(q), N, D, ctypes.byref(p), _ptr(rho), int(row0), int(nrows),
                                 int(mode), _ptr(out)))

    def vds_convect(self, q_in, q_out, shape, u, dx, dt, bc=0):
        """One upwind convection step of a node-major field (include/vds_batch.h)."""
        nx, ny, nz = (int(v) for v in shape)
        M = q_in.numel() // (nx * ny * nz)
        dxs = (ctypes.c_double * 3)(*[float(v) for v in dx])
        _check(lib.vds_convect(self.h, _ptr(q_in), _ptr(q_out), nx, ny, nz, M, _ptr(u), dxs, float(dt), int(bc)))

    def pod_build(self, X, Ns, M, s, energy=0.9999, r_max=64, r_fixed=0, kappa=None):
        kap = np.zeros(9) if kappa is None else np.ascontiguousarray(kappa, dtype=np.float64).ravel()
        kbuf = (ctypes.c_double * 9)(*[float(v) for v in kap[:s * s]] + [0.0] * (9 - s * s))
        out = _vp()
        r = ctypes.c_int()
        _check(lib.pod_build(self.h, _ptr(X), int(Ns), int(M), int(s), float(energy), int(r_max),
                             int(r_fixed), kbuf, ctypes.byref(out), ctypes.byref(r)))
        return PodBasis(out, M), r.value

    def pod_load(self, phi, s, kappa=None):
        """Basis from a device (N s) x r FP32 tensor with orthonormal columns."""
        Ns, r = phi.shape
        kap = np.zeros(9) if kappa is None else np.ascontiguousarray(kappa, dtype=np.float64).ravel()
        kbuf = (ctypes.c_double * 9)(*[float(v) for v in kap[:s * s]] + [0.0] * (9 - s * s))
        out = _vp()
        _check(lib.pod_load(self.h, _ptr(phi), int(Ns), int(r), int(s), kbuf, ctypes.byref(out)))
        return PodBasis(out, 0)

    def pod_project(self, basis: "PodBasis", q, p_out):
        N, D = q.shape
        _check(lib.pod_project(self.h, basis.h, _ptr(q), N, D, _ptr(p_out)))

    def pod_lift(self, basis: "PodBasis", p_in, q_out):
        N, D = q_out.shape
        _check(lib.pod_lift(self.h, basis.h, _ptr(p_in), N, D, _ptr(q_out)))


    def pod_brownian(self, basis: "PodBasis", P, N, D, p: VdsParams):
        r = basis.info()["r"]
        b1 = (ctypes.c_double * (r * r))()
        b2 = (ctypes.c_double * (r * r))()
        _check(lib.pod_brownian(self.h, basis.h, _ptr(P), int(N), int(D), ctypes.byref(p), b1, b2))
        return np.array(b1[:]).reshape(r, r), np.array(b2[:]).reshape(r, r)

    def pod_step_score(self, basis: "PodBasis", score: "Score", P, N, D, p: VdsParams, nsteps=1,
                       check_every=20, check_n=4096, check_tol=0.25):
        err, nf = ctypes.c_double(), ctypes.c_int()
        _check(lib.pod_step_score(self.h, basis.h, score.h, _ptr(P), int(N), int(D), ctypes.byref(p),
                                  int(nsteps), int(check_every), int(check_n), float(check_tol),
                                  ctypes.byref(err), ctypes.byref(nf)))
        return err.value, nf.value

    def pod_step(self, basis: "PodBasis", P, N, D, p: VdsParams, nsteps=1, refresh_every=1, mode=2):
        _check(lib.pod_step(self.h, basis.h, _ptr(P), int(N), int(D), ctypes.byref(p), int(nsteps),
                            int(refresh_every), int(mode)))


class Batch:
    """Owns a vds_batch (include/vds_batch.h)."""

    def __init__(self, ctx: "Context", sizes, D, p: VdsParams, h, kappa):
        sizes = np.ascontiguousarray(sizes, dtype=np.int32)
        h = np.ascontiguousarray(h, dtype=np.float64)
        kappa = np.ascontiguousarray(kappa, dtype=np.float64)
        self.E = len(sizes)
        self.ctx = ctx
        out = _vp()
        _check(lib.vds_batch_create(ctx.h, self.E, sizes.ctypes.data_as(_ip), int(D), ctypes.byref(p),
                                    h.ctypes.data_as(_dp), kappa.ctypes.data_as(_dp), ctypes.byref(out)))
        self.h = out

    def info(self):
        tot, tile, n = ctypes.c_long(), ctypes.c_int(), ctypes.c_int()
        _check(lib.vds_batch_info(self.h, ctypes.byref(tot), ctypes.byref(tile), ctypes.byref(n)))
        return dict(total=tot.value, tile=tile.value, n_items=n.value)

    def queue(self):
        n = self.info()["n_items"]
        buf = (ctypes.c_int * (2 * n))()
        _check(lib.vds_batch_queue(self.h, buf, n))
        return np.array(buf[:], dtype=np.int32).reshape(n, 2)

    def energy_grad(self, q_all, g=None, rho=None, want_energy=True):
        E = (ctypes.c_double * self.E)()
        _check(lib.vds_batch_energy_grad(self.ctx.h, self.h, _ptr(q_all), E if want_energy else None,
                                         _ptr(g), _ptr(rho)))
        return np.array(E[:]) if want_energy else None

    def stress(self, q_all, s):
        """Per-ensemble stress, E x s x s."""
        tau = np.empty((self.E, s, s))
        _check(lib.vds_batch_stress(self.ctx.h, self.h, _ptr(q_all), tau.ctypes.data_as(_dp)))
        return tau

    def set_kappa(self, kappa):
        kappa = np.ascontiguousarray(kappa, dtype=np.float64)
        _check(lib.vds_batch_set_kappa(self.ctx.h, self.h, kappa.ctypes.data_as(_dp)))

    def autotune(self, q_all, reps=3):
        """Times every pair-kernel shape on q_all, keeps the fastest; returns
        (config, milliseconds per config)."""
        cfg = ctypes.c_int()
        ms = (ctypes.c_double * BATCH_CONFIGS)()
        _check(lib.vds_batch_autotune(self.ctx.h, self.h, _ptr(q_all), int(reps), ctypes.byref(cfg), ms))
        return cfg.value, list(ms)

    def set_config(self, config):
        _check(lib.vds_batch_set_config(self.ctx.h, self.h, int(config)))

    def config(self):
        cfg = ctypes.c_int()
        _check(lib.vds_batch_get_config(self.h, ctypes.byref(cfg)))
        return cfg.value

    def step(self, q_all, nsteps=1, want_iters=False):
        it = (ctypes.c_int * max(1, nsteps * self.E))() if want_iters else None
        _check(lib.vds_batch_step(self.ctx.h, self.h, _ptr(q_all), int(nsteps), it))
        return np.array(it[:nsteps * self.E]).reshape(nsteps, self.E) if want_iters else None

    def free(self):
        if self.h:
            lib.vds_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def flatten_layers(layers):
    """[(W, b)] -> flat FP32 parameter vector in the order of vds_score.h."""
    return np.concatenate([np.concatenate([np.asarray(W, np.float32).ravel(), np.asarray(b, np.float32).ravel()])
                           for W, b in layers]).astype(np.float32)


def unflatten(flat, D, width=256):
    shapes = [(width, D), (width, width), (width, width), (D, width)]
    out, k = [], 0
    for r, cc in shapes:
        W = flat[k:k + r * cc].reshape(r, cc)
        k += r * cc
        b = flat[k:k + r]
        k += r
        out.append((W, b))
    return out


class Score:
    """Owns a vds_score network (include/vds_score.h)."""

    def __init__(self, ctx: "Context", D, layers, width=256):
        self.ctx, self.D, self.width = ctx, int(D), int(width)
        flat = flatten_layers(layers)
        n = lib.vds_score_param_count(self.D, self.width)
        assert flat.size == n, (flat.size, n)
        out = _vp()
        _check(lib.vds_score_create(ctx.h, self.D, self.width,
                                    flat.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(out)))
        self.h = out
        self.n = n

    def params(self):
        buf = np.empty(self.n, dtype=np.float32)
        _check(lib.vds_score_get_params(self.ctx.h, self.h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return unflatten(buf, self.D, self.width)

    def set_params(self, layers):
        flat = flatten_layers(layers)
        _check(lib.vds_score_set_params(self.ctx.h, self.h, flat.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def eval(self, x, out):
        _check(lib.vds_score_eval(self.ctx.h, self.h, _ptr(x), int(x.shape[0]), _ptr(out)))

    def loss_grad(self, x, eps, sigma, rows=None):
        loss = ctypes.c_double()
        g = np.empty(self.n, dtype=np.float32)
        M = int(eps.shape[0])
        _check(lib.vds_score_loss_grad(self.ctx.h, self.h, _ptr(x), _ptr(rows), _ptr(eps), M, float(sigma),
                                       ctypes.byref(loss), g.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return loss.value, unflatten(g, self.D, self.width)

    def train_step(self, x, eps, sigma, lr, want_loss=True, rows=None):
        loss = ctypes.c_double()
        M = int(eps.shape[0])
        _check(lib.vds_score_train(self.ctx.h, self.h, _ptr(x), _ptr(rows), _ptr(eps), M, float(sigma),
                                   float(lr), ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def fit_step(self, x, target, lr, rows=None, M=None, want_loss=True, want_grads=False):
        loss = ctypes.c_double()
        M = int(M if M is not None else (rows.shape[0] if rows is not None else x.shape[0]))
        g = np.empty(self.n, dtype=np.float32) if want_grads else None
        _check(lib.vds_score_fit(self.ctx.h, self.h, _ptr(x), _ptr(rows), _ptr(target), M, float(lr),
                                 ctypes.byref(loss) if want_loss else None,
                                 g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if want_grads else None))
        out = loss.value if want_loss else None
        return (out, unflatten(g, self.D, self.width)) if want_grads else out

    def free(self):
        if self.h:
            lib.vds_score_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class PodBasis:
    def __init__(self, h, M):
        self.h = h
        self.M = M

    def info(self):
        r, ld, phi, Ns = ctypes.c_int(), ctypes.c_int(), _vp(), ctypes.c_long()
        _check(lib.pod_info(self.h, ctypes.byref(r), ctypes.byref(ld), ctypes.byref(phi), ctypes.byref(Ns)))
        return dict(r=r.value, ld=ld.value, phi=phi.value, Ns=Ns.value)

    def sweeps(self):
        return lib.pod_sweeps(self.h)

    def eigenvalues(self):
        buf = (ctypes.c_double * self.M)()
        _check(lib.pod_eigenvalues(self.h, buf, self.M))
        return np.array(buf[:])

    def xh(self):
        r = self.info()["r"]
        buf = (ctypes.c_double * (r * r))()
        _check(lib.pod_xh(self.h, buf))
        return np.array(buf[:]).reshape(r, r)

    def phi(self):
        """Copy of Phi as an (N s) x r torch tensor (device)."""
        import torch
        inf = self.info()
        Ns, r, ld = inf["Ns"], inf["r"], inf["ld"]
        buf = torch.empty((Ns, ld), dtype=torch.float32, device="cuda")
        cudart_copy(buf.data_ptr(), inf["phi"], Ns * ld * 4)
        return buf[:, :r].contiguous()

    def free(self):
        if self.h:
            lib.pod_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def cudart_copy(dst, src, nbytes):
    """Device-to-device copy of raw addresses through torch (plumbing only)."""
    import torch
    t_src = torch.as_tensor(_DeviceBuffer(src, nbytes), device="cuda")
    t_dst = torch.as_tensor(_DeviceBuffer(dst, nbytes), device="cuda")
    t_dst.copy_(t_src)
    torch.cuda.current_stream().synchronize()


class _DeviceBuffer:
    """Minimal __cuda_array_interface__ wrapper for a raw device address."""

    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {
            "shape": (int(nbytes),), "typestr": "|u1", "data": (int(ptr), False), "version": 3,
            "strides": None}
