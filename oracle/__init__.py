"""ctypes front end of the FP64 CPU oracle (oracle.h).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the CUDA library never
links or calls it.  It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

FLUX = {"tvdlf": 0, "hll": 1, "hllc": 2}
LIMITER = {"minmod": 0, "vanleer": 1, "koren": 2, "none": 3, "mc": 4, "cada": 5}
BC = {"periodic": 0, "outflow": 1}
MG_BC = {"periodic": 0, "neumann": 1}
RD_MODEL = {"gray-scott": 0, "schnakenberg": 1}
RD_SCHEME = {"imex": 0, "split": 1, "explicit": 2}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class OrcConfig(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("block_nx", C.c_int), ("base", C.c_int * 3), ("max_level", C.c_int),
        ("xmin", C.c_double * 3), ("xmax", C.c_double * 3), ("gamma", C.c_double), ("cfl", C.c_double),
        ("flux", C.c_int), ("limiter", C.c_int), ("rk", C.c_int), ("bc", (C.c_int * 2) * 3),
        ("refine_tol", C.c_double), ("coarsen_frac", C.c_double), ("wavefilter", C.c_double),
        ("var_mask", C.c_uint),
    ]


class OrcMgConfig(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("n", C.c_int), ("L", C.c_double), ("lam", C.c_double),
        ("nu1", C.c_int), ("nu2", C.c_int), ("max_cycles", C.c_int), ("rtol", C.c_double),
        ("coarse_max", C.c_int), ("bc", C.c_int),
    ]


class OrcRdConfig(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("n", C.c_int), ("L", C.c_double), ("Du", C.c_double), ("Dv", C.c_double),
        ("F", C.c_double), ("k", C.c_double), ("dt", C.c_double), ("nu1", C.c_int), ("nu2", C.c_int),
        ("max_cycles", C.c_int), ("rtol", C.c_double), ("coarse_max", C.c_int),
        ("model", C.c_int), ("kappa", C.c_double), ("a", C.c_double), ("b", C.c_double), ("scheme", C.c_int),
        ("bc", C.c_int),
    ]


class OrcAmgConfig(C.Structure):
    _fields_ = [
        ("nbx", C.c_int), ("nby", C.c_int), ("B", C.c_int), ("L", C.c_double), ("lam", C.c_double),
        ("nu1", C.c_int), ("nu2", C.c_int), ("max_cycles", C.c_int), ("rtol", C.c_double),
        ("base_rtol", C.c_double), ("coarse_max", C.c_int),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(OrcConfig)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_num_leaves.argtypes = [C.c_void_p]
        L.orc_leaves.argtypes = [C.c_void_p, _ip, _ip]
        L.orc_set_leaves.argtypes = [C.c_void_p, C.c_int, _ip, _ip]
        for f in ("orc_set_prim", "orc_set_cons", "orc_get_cons", "orc_totals", "orc_lohner"):
            getattr(L, f).argtypes = [C.c_void_p, _dp]
        L.orc_set_time.argtypes = [C.c_void_p, C.c_double]
        L.orc_time.argtypes = [C.c_void_p]
        L.orc_time.restype = C.c_double
        L.orc_dt.argtypes = [C.c_void_p, C.c_double]
        L.orc_dt.restype = C.c_double
        L.orc_step.argtypes = [C.c_void_p, C.c_double]
        L.orc_step.restype = C.c_double
        L.orc_regrid.argtypes = [C.c_void_p]
        L.orc_face_ghosts.argtypes = [C.c_void_p, C.c_int, _dp]
        L.orc_prim_to_cons.argtypes = [C.c_int, C.c_double, _dp, _dp]
        L.orc_cons_to_prim.argtypes = [C.c_int, C.c_double, _dp, _dp]
        L.orc_phys_flux.argtypes = [C.c_int, C.c_int, C.c_double, _dp, _dp]
        L.orc_riemann_flux.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, _dp, _dp, _dp]
        L.orc_limited_slopes.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp]
        L.orc_exact_riemann.argtypes = [C.c_double, _dp, _dp, C.c_int, _dp, _dp, _dp, _dp]
        L.orc_mg_solve.argtypes = [C.POINTER(OrcMgConfig), _dp, _dp, _dp]
        L.orc_mg_vcycle.argtypes = [C.POINTER(OrcMgConfig), _dp, _dp]
        L.orc_mg_apply.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, _dp, _dp]
        L.orc_dense_solve.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, _dp, _dp]
        L.orc_rd_step.argtypes = [C.POINTER(OrcRdConfig), _dp, _dp, _ip]
        L.orc_rd_reaction.argtypes = [C.c_double, C.c_double, C.c_int, _dp, _dp, _dp, _dp]
        L.orc_rd_reaction_schnakenberg.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, _dp, _dp, _dp, _dp]
        L.orc_laplacian.argtypes = [C.c_int, C.c_int, C.c_double, C.c_int, _dp, _dp]
        for f in ("orc_amg_apply", "orc_amg_face_ghosts"):
            getattr(L, f).argtypes = [C.POINTER(OrcAmgConfig), C.c_int, _ip, _ip, _dp, _dp]
        L.orc_amg_solve.argtypes = [C.POINTER(OrcAmgConfig), C.c_int, _ip, _ip, _dp, _dp, C.c_int, _dp]
        L.orc_amg_regrid.argtypes = [C.POINTER(OrcAmgConfig), C.c_int, _ip, _ip, _dp, _dp, C.c_double, C.c_double,
                                     C.c_double, C.c_int, C.c_int, _ip, _ip, _dp, _dp, _dp]
        L.orc_amg_rd_step.argtypes = [C.POINTER(OrcAmgConfig), C.c_int, _ip, _ip] + [C.c_double] * 5 + [_dp, _dp, _ip]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_set_threads.restype = C.c_int
        if hasattr(L, "orc_cnn_forward"):
            _bind_cnn(L)
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_config(ndim, block_nx, base, max_level=1, xmin=(0, 0, 0), xmax=(1, 1, 1), gamma=1.4,
                cfl=0.8, flux="hll", limiter="minmod", rk=2, bc="periodic", refine_tol=0.2,
                coarsen_frac=0.5, wavefilter=0.01, var_mask=None):
    c = OrcConfig()
    c.ndim = ndim
    c.block_nx = block_nx
    base = list(base) + [1] * (3 - len(base))
    for d in range(3):
        c.base[d] = base[d]
        c.xmin[d] = float(xmin[d]) if d < len(xmin) else 0.0
        c.xmax[d] = float(xmax[d]) if d < len(xmax) else 1.0
    c.max_level = max_level
    c.gamma = gamma
    c.cfl = cfl
    c.flux = FLUX[flux] if isinstance(flux, str) else flux
    c.limiter = LIMITER[limiter] if isinstance(limiter, str) else limiter
    c.rk = rk
    if isinstance(bc, str):
        bc = [[bc, bc]] * 3
    for d in range(3):
        for s in range(2):
            b = bc[d][s] if d < len(bc) else "periodic"
            c.bc[d][s] = BC[b] if isinstance(b, str) else b
    c.refine_tol = refine_tol
    c.coarsen_frac = coarsen_frac
    c.wavefilter = wavefilter
    c.var_mask = var_mask if var_mask is not None else (1 | (1 << (ndim + 1)))
    return c


class Grid:
    """A block tree held by the oracle."""

    def __init__(self, **kw):
        self.cfg = make_config(**kw)
        self.ndim = self.cfg.ndim
        self.nv = self.ndim + 2
        self.ncell = self.cfg.block_nx ** self.ndim
        self.h = lib().orc_create(C.byref(self.cfg))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_destroy(self.h)
            self.h = None

    @property
    def nleaves(self):
        return lib().orc_num_leaves(self.h)

    def leaves(self):
        n = self.nleaves
        lev = np.zeros(n, dtype=np.int32)
        crd = np.zeros((n, 3), dtype=np.int32)
        lib().orc_leaves(self.h, _i(lev), _i(crd))
        return lev, crd

    def set_leaves(self, level, coords):
        level = np.ascontiguousarray(level, dtype=np.int32)
        coords = np.ascontiguousarray(coords, dtype=np.int32).reshape(-1, 3)
        if lib().orc_set_leaves(self.h, len(level), _i(level), _i(coords)) != 0:
            raise ValueError("duplicate leaves")

    def set_prim(self, V):
        V = _f64(V).reshape(self.nleaves, self.nv, self.ncell)
        lib().orc_set_prim(self.h, _d(V))

    def set_cons(self, U):
        U = _f64(U).reshape(self.nleaves, self.nv, self.ncell)
        lib().orc_set_cons(self.h, _d(U))

    def get_cons(self):
        U = np.zeros((self.nleaves, self.nv, self.ncell))
        lib().orc_get_cons(self.h, _d(U))
        return U

    @property
    def t(self):
        return lib().orc_time(self.h)

    @t.setter
    def t(self, v):
        lib().orc_set_time(self.h, v)

    def dt(self, t_end=np.inf):
        return lib().orc_dt(self.h, t_end)

    def step(self, t_end=np.inf):
        return lib().orc_step(self.h, t_end)

    def run(self, nsteps=None, t_end=np.inf):
        k = 0
        while (nsteps is None or k < nsteps) and self.t < t_end:
            if self.step(t_end) <= 0:
                break
            k += 1
        return k

    def totals(self):
        t = np.zeros(self.nv)
        lib().orc_totals(self.h, _d(t))
        return t

    def lohner(self):
        e = np.zeros(self.nleaves)
        lib().orc_lohner(self.h, _d(e))
        return e

    def regrid(self):
        return lib().orc_regrid(self.h)

    def face_ghosts(self, leaf):
        nt = self.cfg.block_nx ** (self.ndim - 1)
        out = np.zeros((self.nv, 2 * self.ndim, 2, nt))
        lib().orc_face_ghosts(self.h, leaf, _d(out))
        return out


def set_threads(n=0):
    """Threads of the oracle's OpenMP loops (n <= 0 keeps the current setting); returns the count."""
    return lib().orc_set_threads(int(n))


def prim_to_cons(ndim, gamma, V):
    V = _f64(V)
    U = np.zeros(ndim + 2)
    lib().orc_prim_to_cons(ndim, gamma, _d(V), _d(U))
    return U


def cons_to_prim(ndim, gamma, U):
    U = _f64(U)
    V = np.zeros(ndim + 2)
    lib().orc_cons_to_prim(ndim, gamma, _d(U), _d(V))
    return V


def phys_flux(ndim, direction, gamma, V):
    V = _f64(V)
    F = np.zeros(ndim + 2)
    lib().orc_phys_flux(ndim, direction, gamma, _d(V), _d(F))
    return F


def riemann_flux(ndim, direction, flux, gamma, VL, VR):
    VL, VR = _f64(VL), _f64(VR)
    F = np.zeros(ndim + 2)
    lib().orc_riemann_flux(ndim, direction, FLUX.get(flux, flux) if isinstance(flux, str) else flux,
                           gamma, _d(VL), _d(VR), _d(F))
    return F


def limited_slopes(limiter, a, b):
    sm, sp = C.c_double(), C.c_double()
    lim = LIMITER[limiter] if isinstance(limiter, str) else limiter
    lib().orc_limited_slopes(lim, float(a), float(b), C.byref(sm), C.byref(sp))
    return sm.value, sp.value


def exact_riemann(gamma, left, right, xi):
    xi = _f64(xi)
    out = np.zeros((len(xi), 3))
    ps, us = C.c_double(), C.c_double()
    rc = lib().orc_exact_riemann(gamma, _d(_f64(left)), _d(_f64(right)), len(xi), _d(xi), _d(out),
                                 C.byref(ps), C.byref(us))
    if rc != 0:
        raise ValueError("vacuum")
    return out, ps.value, us.value


def mg_config(ndim, n, L, lam, nu1=2, nu2=2, max_cycles=50, rtol=1e-10, coarse_max=8, bc="periodic"):
    return OrcMgConfig(ndim, n, L, lam, nu1, nu2, max_cycles, rtol, coarse_max, MG_BC[bc])


def mg_solve(b, x0, L, lam, **kw):
    b = _f64(b)
    x = _f64(x0).copy()
    ndim, n = b.ndim, b.shape[0]
    c = mg_config(ndim, n, L, lam, **kw)
    rr = C.c_double()
    cyc = lib().orc_mg_solve(C.byref(c), _d(b), _d(x), C.byref(rr))
    return x, cyc, rr.value


def mg_vcycle(r, L, lam, **kw):
    r = _f64(r)
    e = np.zeros_like(r)
    c = mg_config(r.ndim, r.shape[0], L, lam, **kw)
    lib().orc_mg_vcycle(C.byref(c), _d(r), _d(e))
    return e


def mg_apply(x, L, lam, bc="periodic"):
    x = _f64(x)
    out = np.zeros_like(x)
    lib().orc_mg_apply(x.ndim, x.shape[0], L, lam, MG_BC[bc], _d(x), _d(out))
    return out


def dense_solve(b, L, lam, bc="periodic"):
    b = _f64(b)
    x = np.zeros_like(b)
    if lib().orc_dense_solve(b.ndim, b.shape[0], L, lam, MG_BC[bc], _d(b), _d(x)) != 0:
        raise ValueError("singular")
    return x


def laplacian(x, L, bc="periodic"):
    x = _f64(x)
    out = np.zeros_like(x)
    lib().orc_laplacian(x.ndim, x.shape[0], L, MG_BC[bc], _d(x), _d(out))
    return out


def rd_reaction(F, k, u, v):
    u, v = _f64(u), _f64(v)
    fu, fv = np.zeros_like(u), np.zeros_like(v)
    lib().orc_rd_reaction(F, k, u.size, _d(u), _d(v), _d(fu), _d(fv))
    return fu, fv


def rd_reaction_schnakenberg(kappa, a, b, u, v):
    u, v = _f64(u), _f64(v)
    fu, fv = np.zeros_like(u), np.zeros_like(v)
    lib().orc_rd_reaction_schnakenberg(kappa, a, b, u.size, _d(u), _d(v), _d(fu), _d(fv))
    return fu, fv


def rd_step(u, v, L, Du, Dv, dt, F=0.0, k=0.0, nu1=2, nu2=2, max_cycles=50, rtol=1e-10, coarse_max=8,
            model="gray-scott", kappa=0.0, a=0.0, b=0.0, scheme="imex", bc="periodic"):
    """One reaction-diffusion step of `scheme` ("imex", "split", "explicit") for `model`
    ("gray-scott": F, k; "schnakenberg": kappa, a, b) with `bc` ("periodic", "neumann")."""
    u, v = _f64(u).copy(), _f64(v).copy()
    c = OrcRdConfig(u.ndim, u.shape[0], L, Du, Dv, F, k, dt, nu1, nu2, max_cycles, rtol, coarse_max,
                    RD_MODEL[model], kappa, a, b, RD_SCHEME[scheme], MG_BC[bc])
    cyc = np.zeros(2, dtype=np.int32)
    st = lib().orc_rd_step(C.byref(c), _d(u), _d(v), _i(cyc))
    if st != 0:
        raise RuntimeError("multigrid did not converge")
    return u, v, cyc


def _bind_cnn(L):
    L.orc_cnn_num_params.argtypes = [C.c_int]
    L.orc_cnn_num_params.restype = C.c_longlong
    L.orc_cnn_forward.argtypes = [C.c_int, _dp, C.c_int, C.c_int, C.c_int, C.c_int, _dp, _dp]
    L.orc_cnn_loss_grad.argtypes = [C.c_int, _dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _dp, _dp, _dp]
    L.orc_cnn_loss_grad.restype = C.c_double
    L.orc_cnn_loss_grad_kind.argtypes = [C.c_int, _dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _dp,
                                         _dp, _dp, _dp]
    L.orc_cnn_loss_grad_kind.restype = C.c_double
    L.orc_cnn_output_loss.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _dp, _dp, _dp,
                                      _dp]
    L.orc_cnn_output_loss.restype = C.c_double
    L.orc_cnn_adam.argtypes = [C.c_longlong, _dp, _dp, _dp, _dp, C.c_int, C.c_double, C.c_double, C.c_double,
                               C.c_double]
    L.orc_gelu.argtypes = [C.c_double]
    L.orc_gelu.restype = C.c_double
    L.orc_gelu_d.argtypes = [C.c_double]
    L.orc_gelu_d.restype = C.c_double


CNN_CHANNELS = (5, 16, 16, 16, 2)


def cnn_num_params(ndim):
    return lib().orc_cnn_num_params(ndim)


def _shape(x, ndim):
    x = _f64(x)
    N = x.shape[0]
    if ndim == 2:
        return x, N, 1, x.shape[2], x.shape[3]
    return x, N, x.shape[2], x.shape[3], x.shape[4]


def cnn_forward(params, x, ndim=2):
    """x: [N][5][H][W] (2D) or [N][5][D][H][W]; returns [N][2][...]"""
    x, N, D, H, W = _shape(x, ndim)
    out = np.zeros((N, 2) + x.shape[2:])
    lib().orc_cnn_forward(ndim, _d(_f64(params)), N, D, H, W, _d(x), _d(out))
    return out


CNN_LOSS = {"mse": 0, "operator": 1}


def cnn_loss_grad(params, x, target, margin=0, ndim=2, loss="mse", kappa=(0.0, 0.0)):
    """Loss and its gradient over the flat parameters.  loss="operator": the mean of q^2,
    q = (1 + kappa_c) e - (1/(2 ndim)) sum_faces e, e = out - target (margin >= 1)."""
    x, N, D, H, W = _shape(x, ndim)
    target = _f64(target)
    g = np.zeros(cnn_num_params(ndim))
    kap = _f64(np.asarray(kappa, dtype=np.float64).reshape(2))
    val = lib().orc_cnn_loss_grad_kind(ndim, _d(_f64(params)), N, D, H, W, margin, CNN_LOSS[loss], _d(kap), _d(x),
                                       _d(target), _d(g))
    if val < 0:
        raise ValueError("the operator-weighted loss needs margin >= 1")
    return val, g


def cnn_output_loss(out, target, margin=0, ndim=2, loss="mse", kappa=(0.0, 0.0)):
    """The loss alone on network outputs [N][2][...]: (loss, dL/d(out))."""
    out, N, D, H, W = _shape(out, ndim)
    target = _f64(target)
    dout = np.zeros_like(out)
    kap = _f64(np.asarray(kappa, dtype=np.float64).reshape(2))
    val = lib().orc_cnn_output_loss(ndim, N, D, H, W, margin, CNN_LOSS[loss], _d(kap), _d(out), _d(target),
                                    _d(dout))
    if val < 0:
        raise ValueError("the operator-weighted loss needs margin >= 1")
    return val, dout


def cnn_adam(params, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """in place on params, m, v (float64 arrays)"""
    lib().orc_cnn_adam(len(params), _d(params), _d(_f64(grad)), _d(m), _d(v), t, lr, b1, b2, eps)


def gelu(z):
    return lib().orc_gelu(float(z))


def gelu_d(z):
    return lib().orc_gelu_d(float(z))


def cnn_layer_slices(ndim):
    """(W slice, b slice, cin, cout) per layer in the flat parameter vector"""
    T = 27 if ndim == 3 else 9
    out, o = [], 0
    for l in range(4):
        ci, co = CNN_CHANNELS[l], CNN_CHANNELS[l + 1]
        out.append((slice(o, o + co * ci * T), slice(o + co * ci * T, o + co * ci * T + co), ci, co))
        o += co * ci * T + co
    return out


# ------------------------------------------------------------------ AMR multigrid --
def amg_config(nb, B, L, lam, nu1=2, nu2=2, max_cycles=50, rtol=1e-10, base_rtol=1e-3, coarse_max=8):
    return OrcAmgConfig(nb, nb, B, L, lam, nu1, nu2, max_cycles, rtol, base_rtol, coarse_max)


def _tree(level, coords):
    level = np.ascontiguousarray(level, dtype=np.int32)
    coords = np.ascontiguousarray(coords, dtype=np.int32).reshape(-1, 2)
    return level, coords


def amg_solve(level, coords, b, x0, nb, B, L, lam, fixed_cycles=0, **kw):
    """Multigrid on a 2D block quadtree: leaves (level, (bx, by)); b, x0 [leaf][B*B].
    Returns (x, cycles, relres); cycles -1 if rtol was not reached."""
    level, coords = _tree(level, coords)
    b = _f64(b)
    x = _f64(x0).copy()
    c = amg_config(nb, B, L, lam, **kw)
    rr = C.c_double()
    cyc = lib().orc_amg_solve(C.byref(c), len(level), _i(level), _i(coords), _d(b), _d(x), fixed_cycles,
                              C.byref(rr))
    if cyc == -2:
        raise ValueError("invalid tree")
    return x, cyc, rr.value


def amg_apply(level, coords, x, nb, B, L, lam):
    level, coords = _tree(level, coords)
    x = _f64(x)
    out = np.zeros_like(x)
    if lib().orc_amg_apply(C.byref(amg_config(nb, B, L, lam)), len(level), _i(level), _i(coords), _d(x), _d(out)):
        raise ValueError("invalid tree")
    return out


def amg_face_ghosts(level, coords, x, nb, B, L):
    level, coords = _tree(level, coords)
    x = _f64(x)
    g = np.zeros((len(level), 4, B))
    if lib().orc_amg_face_ghosts(C.byref(amg_config(nb, B, L, 1.0)), len(level), _i(level), _i(coords), _d(x),
                                 _d(g)):
        raise ValueError("invalid tree")
    return g


def amg_rd_step(level, coords, u, v, nb, B, L, Du, Dv, F, k, dt, **kw):
    """Gray-Scott IMEX step on the quadtree leaves; returns (u, v, cycles[2])."""
    level, coords = _tree(level, coords)
    u, v = _f64(u).copy(), _f64(v).copy()
    cyc = np.zeros(2, dtype=np.int32)
    st = lib().orc_amg_rd_step(C.byref(amg_config(nb, B, L, 0.0, **kw)), len(level), _i(level), _i(coords),
                               Du, Dv, F, k, dt, _d(u), _d(v), _i(cyc))
    if st == -2:
        raise ValueError("invalid tree")
    if st != 0:
        raise RuntimeError("tree multigrid did not converge")
    return u, v, cyc


def amg_regrid(level, coords, u, v, nb, B, L, refine_tol, coarsen_frac=0.5, eps=0.01, max_level=3):
    """Regrid of the reaction-diffusion quadtree; returns (level, coords, u, v, err_of_old_leaves)."""
    level, coords = _tree(level, coords)
    u, v = _f64(u), _f64(v)
    n = len(level)
    cap = 4 * n
    nl, nc = np.zeros(cap, np.int32), np.zeros((cap, 2), np.int32)
    nu, nv = np.zeros((cap, B * B)), np.zeros((cap, B * B))
    err = np.zeros(n)
    m = lib().orc_amg_regrid(C.byref(amg_config(nb, B, L, 0.0)), n, _i(level), _i(coords), _d(u), _d(v), refine_tol,
                             coarsen_frac, eps, max_level, cap, _i(nl), _i(nc), _d(nu), _d(nv), _d(err))
    if m < 0:
        raise ValueError("invalid tree" if m == -2 else "capacity")
    return nl[:m].copy(), nc[:m].copy(), nu[:m].copy(), nv[:m].copy(), err
