"""Python binding of the amrvac_gb300 C ABI (include/amrvac_gb300.h).

Argument marshalling only: every step of the method runs in the CUDA library.
Loading fails loudly if the library has not been built; there is no CPU path.
Arrays may be numpy (host) or torch CUDA tensors (device, float64, contiguous).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

AMR_OK = 0
STATUS = {0: "AMR_OK", -1: "AMR_ERR_INVALID_ARG", -2: "AMR_ERR_OOM", -3: "AMR_ERR_CUDA",
          -4: "AMR_ERR_NONPHYSICAL", -5: "AMR_ERR_TIMEOUT", -6: "MG_ERR_NOT_CONVERGED",
          -7: "AMR_ERR_CAPACITY", -8: "AMR_ERR_UNBALANCED"}
FLUX = {"tvdlf": 0, "hll": 1, "hllc": 2}
LIMITER = {"minmod": 0, "vanleer": 1, "koren": 2, "none": 3, "mc": 4, "cada": 5}
BC = {"periodic": 0, "outflow": 1}
PRECISION = {"fp64": 0, "fp32": 1}


class AmrError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__(f"{STATUS.get(code, code)}: {msg}")


class AmrConfig(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("block_nx", C.c_int), ("base_nblocks", C.c_int * 3), ("max_level", C.c_int),
        ("xmin", C.c_double * 3), ("xmax", C.c_double * 3), ("gamma", C.c_double),
        ("flux", C.c_int), ("limiter", C.c_int), ("rk", C.c_int), ("cfl", C.c_double),
        ("bc", (C.c_int * 2) * 3), ("precision", C.c_int), ("refine_tol", C.c_double),
        ("coarsen_frac", C.c_double), ("wavefilter", C.c_double), ("refine_var_mask", C.c_uint),
        ("max_blocks", C.c_longlong), ("stream", C.c_void_p),
    ]


class MgConfig(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("n_inst", C.c_int), ("n_cells", C.POINTER(C.c_int)),
        ("lam", C.POINTER(C.c_double)), ("L", C.c_double), ("nu1", C.c_int), ("nu2", C.c_int),
        ("max_cycles", C.c_int), ("rtol", C.c_double), ("coarse_max", C.c_int), ("precision", C.c_int),
        ("stream", C.c_void_p), ("bc", C.c_int),
    ]


class MgtConfig(C.Structure):
    _fields_ = [
        ("nbx", C.c_int), ("nby", C.c_int), ("B", C.c_int), ("L", C.c_double), ("lam", C.c_double),
        ("nu1", C.c_int), ("nu2", C.c_int), ("max_cycles", C.c_int), ("rtol", C.c_double),
        ("base_rtol", C.c_double), ("coarse_max", C.c_int), ("stream", C.c_void_p),
    ]


class RdtConfig(C.Structure):
    _fields_ = [("mg", MgtConfig), ("Du", C.c_double), ("Dv", C.c_double), ("F", C.c_double), ("k", C.c_double),
                ("dt", C.c_double)]


MG_BC = {"periodic": 0, "neumann": 1}
RD_MODEL = {"gray-scott": 0, "schnakenberg": 1}
RD_SCHEME = {"imex": 0, "split": 1, "explicit": 2}


class RdConfig(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("n_inst", C.c_int), ("n_cells", C.POINTER(C.c_int)), ("L", C.c_double),
        ("Du", C.c_double), ("Dv", C.c_double), ("F", C.c_double), ("k", C.c_double), ("dt", C.c_double),
        ("nu1", C.c_int), ("nu2", C.c_int), ("max_cycles", C.c_int), ("rtol", C.c_double),
        ("coarse_max", C.c_int), ("precision", C.c_int), ("stream", C.c_void_p),
        ("model", C.c_int), ("kappa", C.c_double), ("a", C.c_double), ("b", C.c_double), ("scheme", C.c_int),
        ("bc", C.c_int),
    ]


_vp, _dp, _ip, _llp = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_longlong)
# amr_prim_fn: void (*)(const double x[3], double* V, void* user)
_PRIM_FN = C.CFUNCTYPE(None, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p)

_SIGS = {
    "amr_create": ([C.POINTER(AmrConfig), C.POINTER(_vp)], C.c_int),
    "amr_destroy": ([_vp], C.c_int),
    "amr_last_error": ([_vp], C.c_char_p),
    "amr_num_leaves": ([_vp, _llp], C.c_int),
    "amr_leaf_info": ([_vp, _ip, _ip, C.c_longlong], C.c_int),
    "amr_set_leaves": ([_vp, C.c_longlong, _ip, _ip], C.c_int),
    "amr_set_state": ([_vp, _vp, C.c_longlong, C.c_int, C.c_int], C.c_int),
    "amr_set_state_fn": ([_vp, _PRIM_FN, _vp], C.c_int),
    "amr_read_state": ([_vp, _vp, C.c_longlong, C.c_int], C.c_int),
    "amr_set_time": ([_vp, C.c_double], C.c_int),
    "amr_step": ([_vp, C.c_double, _dp, _dp], C.c_int),
    "amr_run": ([_vp, C.c_int, C.c_double], C.c_int),
    "amr_sync": ([_vp, _dp, _dp], C.c_int),
    "amr_estimate": ([_vp, _dp, C.c_longlong], C.c_int),
    "amr_regrid": ([_vp], C.c_int),
    "amr_conserved_totals": ([_vp, _dp], C.c_int),
    "amr_face_neighbors": ([_vp, _ip, _ip, C.c_longlong], C.c_int),
    "amr_face_ghosts": ([_vp, C.c_longlong, _dp, C.c_longlong], C.c_int),
    "amr_kernel_launches": ([_vp, _llp], C.c_int),
    "amr_profile_step": ([_vp, C.c_double, C.POINTER(C.c_float), _ip, C.c_int, _ip], C.c_int),
    "amr_march_tuning": ([_vp, _ip, C.POINTER(C.c_float)], C.c_int),
    "amr_set_march_tuning": ([_vp, _ip], C.c_int),
    "amr_reduce_noalloc": ([C.POINTER(AmrConfig), _vp, C.c_longlong, _dp, _dp], C.c_int),
    "mg_create": ([C.POINTER(MgConfig), C.POINTER(_vp)], C.c_int),
    "mg_destroy": ([_vp], C.c_int),
    "mg_last_error": ([_vp], C.c_char_p),
    "mg_solve": ([_vp, _vp, _vp, C.c_int, _ip, _dp], C.c_int),
    "mg_num_unknowns": ([_vp, _llp], C.c_int),
    "rd_create": ([C.POINTER(RdConfig), C.POINTER(_vp)], C.c_int),
    "rd_destroy": ([_vp], C.c_int),
    "rd_last_error": ([_vp], C.c_char_p),
    "rd_set_state": ([_vp, _vp, _vp, C.c_int], C.c_int),
    "rd_read_state": ([_vp, _vp, _vp, C.c_int], C.c_int),
    "rd_step": ([_vp, C.c_int, _ip], C.c_int),
    "cnn_create": ([C.c_int, C.c_ulonglong, _vp, C.POINTER(_vp)], C.c_int),
    "cnn_destroy": ([_vp], C.c_int),
    "cnn_last_error": ([_vp], C.c_char_p),
    "cnn_num_params": ([_vp, _llp], C.c_int),
    "cnn_set_params": ([_vp, C.POINTER(C.c_float), C.c_longlong], C.c_int),
    "cnn_get_params": ([_vp, C.POINTER(C.c_float), C.c_longlong], C.c_int),
    "cnn_forward": ([_vp, _vp, C.c_int, C.c_int, C.c_int, C.c_int, _vp], C.c_int),
    "cnn_gradient": ([_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_float),
                      C.POINTER(C.c_float)], C.c_int),
    "cnn_train_step": ([_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float,
                        C.POINTER(C.c_float)], C.c_int),
    "cnn_set_loss": ([_vp, C.c_int, C.POINTER(C.c_double)], C.c_int),
    "cnn_infer": ([_vp, _vp, C.c_int, C.c_int, C.c_int, C.c_int, _vp], C.c_int),
    "cnn_save": ([_vp, C.c_char_p], C.c_int),
    "cnn_load": ([_vp, C.c_char_p], C.c_int),
    "cnn_kernel_launches": ([_vp, _llp], C.c_int),
    "rd_set_guess": ([_vp, _vp, C.c_double], C.c_int),
    "rd_set_guess_inputs": ([_vp, C.c_int], C.c_int),
    "rd_last_residuals": ([_vp, _dp, _dp], C.c_int),
    "rd_extract_crops": ([_vp, C.c_int, _ip, _ip, C.c_int, C.c_double, _vp, _vp], C.c_int),
    "mg_kernel_launches": ([_vp, _llp], C.c_int),
    "mg_strip_height": ([_vp, C.c_int, _ip], C.c_int),
    "mg_profile_vcycle": ([_vp, _ip, C.POINTER(C.c_float), C.c_int, _ip], C.c_int),
    "rd_kernel_launches": ([_vp, _llp], C.c_int),
    "mgt_create": ([C.POINTER(MgtConfig), C.c_int, _ip, _ip, C.POINTER(_vp)], C.c_int),
    "mgt_destroy": ([_vp], C.c_int),
    "mgt_last_error": ([_vp], C.c_char_p),
    "mgt_num_leaves": ([_vp, _llp], C.c_int),
    "mgt_solve": ([_vp, _vp, _vp, C.c_int, C.c_int, _ip, _dp], C.c_int),
    "mgt_apply": ([_vp, _vp, _vp, C.c_int], C.c_int),
    "mgt_kernel_launches": ([_vp, _llp], C.c_int),
    "rdt_create": ([C.POINTER(RdtConfig), C.c_int, _ip, _ip, C.POINTER(_vp)], C.c_int),
    "rdt_destroy": ([_vp], C.c_int),
    "rdt_last_error": ([_vp], C.c_char_p),
    "rdt_set_state": ([_vp, _vp, _vp, C.c_int], C.c_int),
    "rdt_read_state": ([_vp, _vp, _vp, C.c_int], C.c_int),
    "rdt_step": ([_vp, C.c_int, _ip], C.c_int),
    "rdt_kernel_launches": ([_vp, _llp], C.c_int),
    "rdt_num_leaves": ([_vp, _llp], C.c_int),
    "rdt_leaves": ([_vp, _ip, _ip, C.c_longlong], C.c_int),
    "rdt_regrid": ([_vp, C.c_double, C.c_double, C.c_double, C.c_int, _dp, _llp], C.c_int),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load the CUDA library; raises if it is missing (no fallback)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
            _build.build()
        L = C.CDLL(path)
        for name, (args, res) in _SIGS.items():
            if hasattr(L, name):
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _ptr(a):
    """(address, on_device) of a numpy array or a torch tensor."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data, 0


def _check(rc, h, errfn="amr_last_error"):
    if rc != AMR_OK:
        msg = ""
        if h:
            m = getattr(load(), errfn)(h)
            msg = m.decode() if m else ""
        raise AmrError(rc, msg)


def make_amr_config(ndim, block_nx, base, max_level=1, xmin=(0, 0, 0), xmax=(1, 1, 1), gamma=1.4,
                    flux="hllc", limiter="vanleer", rk=3, cfl=0.8, bc="periodic", precision="fp64",
                    refine_tol=0.2, coarsen_frac=0.5, wavefilter=0.01, var_mask=None, max_blocks=None,
                    stream=None):
    c = AmrConfig()
    c.ndim = ndim
    c.block_nx = block_nx
    base = list(base) + [1] * (3 - len(base))
    for d in range(3):
        c.base_nblocks[d] = base[d]
        c.xmin[d] = float(xmin[d]) if d < len(xmin) else 0.0
        c.xmax[d] = float(xmax[d]) if d < len(xmax) else 1.0
    c.max_level = max_level
    c.gamma = gamma
    c.flux = FLUX[flux] if isinstance(flux, str) else flux
    c.limiter = LIMITER[limiter] if isinstance(limiter, str) else limiter
    c.rk = rk
    c.cfl = cfl
    if isinstance(bc, str):
        bc = [[bc, bc]] * 3
    for d in range(3):
        for s in range(2):
            b = bc[d][s] if d < len(bc) else "periodic"
            c.bc[d][s] = BC[b] if isinstance(b, str) else b
    c.precision = PRECISION[precision] if isinstance(precision, str) else precision
    c.refine_tol = refine_tol
    c.coarsen_frac = coarsen_frac
    c.wavefilter = wavefilter
    c.refine_var_mask = var_mask if var_mask is not None else (1 | (1 << (ndim + 1)))
    nbase = int(np.prod(base[:ndim]))
    c.max_blocks = max_blocks if max_blocks is not None else nbase * (2 ** ndim) ** (max_level - 1)
    c.stream = stream
    return c


CHECKPOINT_KIND = "amrvac-gb300 block-tree checkpoint v2"


def _update_fields(cfg):
    """Every amr_config field that changes the update or the regrid (the stream and the
    capacity do not), as plain Python values in a fixed order."""
    return {
        "ndim": int(cfg.ndim), "block_nx": int(cfg.block_nx),
        "base": [int(cfg.base_nblocks[d]) for d in range(3)], "max_level": int(cfg.max_level),
        "xmin": [float(cfg.xmin[d]) for d in range(3)], "xmax": [float(cfg.xmax[d]) for d in range(3)],
        "gamma": float(cfg.gamma), "flux": int(cfg.flux), "limiter": int(cfg.limiter), "rk": int(cfg.rk),
        "cfl": float(cfg.cfl), "bc": [[int(cfg.bc[d][s]) for s in range(2)] for d in range(3)],
        "precision": int(cfg.precision), "refine_tol": float(cfg.refine_tol),
        "coarsen_frac": float(cfg.coarsen_frac), "wavefilter": float(cfg.wavefilter),
        "refine_var_mask": int(cfg.refine_var_mask),
    }


def save_checkpoint(solver, path, steps=0):
    """Writes a solver's tree (leaf levels and block coordinates, Morton order), time, step
    count and float64 conserved state to an .npz file, with every configuration field that
    affects the update.  Works on any object with the AmrSolver calls used here."""
    import json
    lev, crd = solver.leaves()
    np.savez(path, kind=CHECKPOINT_KIND, config=json.dumps(_update_fields(solver.cfg)),
             level=np.asarray(lev, dtype=np.int32), coords=np.asarray(crd, dtype=np.int32), t=float(solver.t),
             steps=int(steps), U=np.asarray(solver.read_state()))


def load_checkpoint(solver, path):
    """Restores a checkpoint into a solver created with the same configuration (geometry,
    domain, physics, scheme, precision and refinement fields): tree, then conserved state,
    then time.  Returns the saved step count.  A continuation from it repeats the saved
    run's steps.  ValueError if the file does not match the solver."""
    import json
    with np.load(path, allow_pickle=False) as d:
        if "kind" not in d.files or str(d["kind"]) != CHECKPOINT_KIND:
            raise ValueError(f"{path}: not a block-tree checkpoint")
        want, got = _update_fields(solver.cfg), json.loads(str(d["config"]))
        diff = sorted(k for k in want if want[k] != got.get(k))
        if diff:
            raise ValueError(f"{path}: configuration differs from the solver's in {diff}")
        solver.set_leaves(d["level"], d["coords"])
        solver.set_state(np.ascontiguousarray(d["U"]), primitive=False)
        solver.set_time(float(d["t"]))
        return int(d["steps"])


class AmrSolver:
    """Owns one amr_handle.  Methods map one to one onto the C calls."""

    def __init__(self, **kw):
        self.lib = load()
        self.cfg = make_amr_config(**kw)
        self.ndim = self.cfg.ndim
        self.nv = self.ndim + 2
        self.ncell = self.cfg.block_nx ** self.ndim
        h = _vp()
        rc = self.lib.amr_create(C.byref(self.cfg), C.byref(h))
        if rc != AMR_OK:
            raise AmrError(rc, "amr_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.amr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nleaves(self):
        n = C.c_longlong()
        _check(self.lib.amr_num_leaves(self.h, C.byref(n)), self.h)
        return n.value

    def leaves(self):
        n = self.nleaves
        lev = np.zeros(n, dtype=np.int32)
        crd = np.zeros((n, 3), dtype=np.int32)
        _check(self.lib.amr_leaf_info(self.h, lev.ctypes.data_as(_ip), crd.ctypes.data_as(_ip), n), self.h)
        return lev, crd

    def set_leaves(self, level, coords):
        level = np.ascontiguousarray(level, dtype=np.int32)
        coords = np.ascontiguousarray(coords, dtype=np.int32).reshape(-1, 3)
        _check(self.lib.amr_set_leaves(self.h, len(level), level.ctypes.data_as(_ip), coords.ctypes.data_as(_ip)),
               self.h)

    def set_state(self, W, primitive=True):
        if not hasattr(W, "data_ptr"):
            W = np.ascontiguousarray(W, dtype=np.float64)
        p, dev = _ptr(W)
        n = W.numel() if hasattr(W, "numel") else W.size
        _check(self.lib.amr_set_state(self.h, p, n, dev, 1 if primitive else 0), self.h)

    def set_state_fn(self, prim_at):
        """Initial condition from a Python callable prim_at(x) -> ndim + 2 primitive values at the
        cell centre x (3 floats; unused dimensions 0): the tree is sampled and regridded
        max_level - 1 times (amr_set_state_fn).  One call per cell, so meant for moderate grids."""
        nv, failure = self.nv, []

        def cb(xp, vp, _user):
            try:
                vals = prim_at((xp[0], xp[1], xp[2]))
                for k in range(nv):
                    vp[k] = float(vals[k])
            except Exception as e:  # noqa: BLE001 -- re-raised after the C call returns
                if not failure:
                    failure.append(e)
                for k in range(nv):
                    vp[k] = float("nan")

        fn = _PRIM_FN(cb)
        rc = self.lib.amr_set_state_fn(self.h, fn, None)
        if failure:
            raise failure[0]
        _check(rc, self.h)

    def set_prim(self, V):
        self.set_state(V, primitive=True)

    def set_cons(self, U):
        self.set_state(U, primitive=False)

    def read_state(self, out=None):
        n = self.nleaves * self.nv * self.ncell
        if out is None:
            out = np.zeros((self.nleaves, self.nv, self.ncell))
        p, dev = _ptr(out)
        _check(self.lib.amr_read_state(self.h, p, n, dev), self.h)
        return out

    get_cons = read_state

    def set_time(self, t):
        _check(self.lib.amr_set_time(self.h, t), self.h)

    def step(self, t_end=1e300):
        dt, t = C.c_double(), C.c_double()
        _check(self.lib.amr_step(self.h, t_end, C.byref(dt), C.byref(t)), self.h)
        return dt.value

    def run(self, nsteps, t_end=1e300):
        _check(self.lib.amr_run(self.h, nsteps, t_end), self.h)

    def sync(self):
        t, dt = C.c_double(), C.c_double()
        _check(self.lib.amr_sync(self.h, C.byref(t), C.byref(dt)), self.h)
        return t.value, dt.value

    @property
    def t(self):
        return self.sync()[0]

    def totals(self):
        out = np.zeros(self.nv)
        _check(self.lib.amr_conserved_totals(self.h, out.ctypes.data_as(_dp)), self.h)
        return out

    def estimate(self):
        e = np.zeros(self.nleaves)
        _check(self.lib.amr_estimate(self.h, e.ctypes.data_as(_dp), len(e)), self.h)
        return e

    lohner = estimate

    def regrid(self):
        _check(self.lib.amr_regrid(self.h), self.h)
        return self.nleaves

    def face_neighbors(self):
        n = self.nleaves * 2 * self.ndim
        kind = np.zeros(n, dtype=np.int32)
        nbr = np.zeros(n, dtype=np.int32)
        _check(self.lib.amr_face_neighbors(self.h, kind.ctypes.data_as(_ip), nbr.ctypes.data_as(_ip), n), self.h)
        return kind.reshape(-1, 2 * self.ndim), nbr.reshape(-1, 2 * self.ndim)

    def face_ghosts(self, leaf):
        nt = self.cfg.block_nx ** (self.ndim - 1)
        out = np.zeros((self.nv, 2 * self.ndim, 2, nt))
        _check(self.lib.amr_face_ghosts(self.h, leaf, out.ctypes.data_as(_dp), out.size), self.h)
        return out

    def profile_step(self, t_end=1e300):
        """One step kernel by kernel; returns [(kind, ms)] (kind 0 stage, 1 ghost, 2 reflux, 3 reduce)."""
        cap = 64
        ms = (C.c_float * cap)()
        kind = (C.c_int * cap)()
        n = C.c_int()
        _check(self.lib.amr_profile_step(self.h, t_end, ms, kind, cap, C.byref(n)), self.h)
        return [(kind[i], ms[i]) for i in range(n.value)]

    def kernel_launches(self):
        n = C.c_longlong()
        _check(self.lib.amr_kernel_launches(self.h, C.byref(n)), self.h)
        return n.value

    def march_tuning(self):
        """amr_march_tuning: ([(warps per CTA, persistent)] per stage kind, [us per kind])."""
        ch = np.zeros(6, dtype=np.int32)
        us = (C.c_float * 3)()
        _check(self.lib.amr_march_tuning(self.h, ch.ctypes.data_as(_ip), us), self.h)
        return [(int(ch[2 * k]), int(ch[2 * k + 1])) for k in range(3)], [float(us[k]) for k in range(3)]

    def set_march_tuning(self, choice):
        """amr_set_march_tuning: choice = [(warps per CTA, persistent)] for the three stage kinds."""
        ch = np.ascontiguousarray(np.array(choice, dtype=np.int32).ravel())
        _check(self.lib.amr_set_march_tuning(self.h, ch.ctypes.data_as(_ip)), self.h)


NOALLOC_MAX_LEAVES = 16384


def reduce_noalloc(U, stream=None, **kw):
    """amr_reduce_noalloc: (dt_cfl, totals) of a uniform block grid whose float64
    conserved state U ([leaf][var][cell], a CUDA tensor) is already on the device.
    Allocates no device memory; see include/amrvac_gb300.h for the shared scratch."""
    lib = load()
    cfg = make_amr_config(stream=stream, **kw)
    p, dev = _ptr(U)
    if not dev:
        raise ValueError("U must be device memory")
    nleaves = int(np.prod(list(cfg.base_nblocks)[:cfg.ndim]))
    # the kernel reads nleaves * (ndim + 2) * block_nx^ndim float64 values from the bare pointer
    need = nleaves * (cfg.ndim + 2) * cfg.block_nx ** cfg.ndim
    if str(getattr(U, "dtype", "")) != "torch.float64":
        raise ValueError(f"U must be a float64 CUDA tensor, got {getattr(U, 'dtype', type(U))}")
    if nleaves <= NOALLOC_MAX_LEAVES and U.numel() < need:
        raise ValueError(f"U holds {U.numel()} values, the grid needs {need}")
    dt = C.c_double()
    tot = np.zeros(cfg.ndim + 2)
    rc = lib.amr_reduce_noalloc(C.byref(cfg), p, nleaves, C.byref(dt), tot.ctypes.data_as(_dp))
    if rc != AMR_OK:
        raise AmrError(rc, "amr_reduce_noalloc")
    return dt.value, tot


class MgSolver:
    """Owns one mg_handle: batched Helmholtz multigrid (lambda_i - lap) x = b."""

    def __init__(self, ndim, n_cells, lam, L, nu1=2, nu2=2, max_cycles=50, rtol=1e-10, coarse_max=8,
                 precision="fp32", stream=None, bc="periodic"):
        self.lib = load()
        self.n_cells = np.ascontiguousarray(n_cells, dtype=np.int32)
        self.lam = np.ascontiguousarray(np.broadcast_to(np.asarray(lam, dtype=np.float64), self.n_cells.shape))
        c = MgConfig()
        c.ndim = ndim
        c.n_inst = len(self.n_cells)
        c.n_cells = self.n_cells.ctypes.data_as(_ip)
        c.lam = self.lam.ctypes.data_as(_dp)
        c.L = L
        c.nu1, c.nu2, c.max_cycles, c.rtol, c.coarse_max = nu1, nu2, max_cycles, rtol, coarse_max
        c.precision = PRECISION[precision] if isinstance(precision, str) else precision
        c.stream = stream
        c.bc = MG_BC[bc]
        self.ndim = ndim
        h = _vp()
        rc = self.lib.mg_create(C.byref(c), C.byref(h))
        if rc != AMR_OK:
            raise AmrError(rc, "mg_create")
        self.h = h
        n = C.c_longlong()
        _check(self.lib.mg_num_unknowns(self.h, C.byref(n)), self.h, "mg_last_error")
        self.n = n.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.mg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def strip_height(self, side):
        """2D: the autotuned strip height of the sweep for levels of this side."""
        h = C.c_int()
        _check(self.lib.mg_strip_height(self.h, side, C.byref(h)), self.h, "mg_last_error")
        return h.value

    def solve(self, b, x):
        """b, x: packed float64 arrays (numpy host or torch CUDA); x is updated in place.
        Returns (cycles per instance, relative residual per instance)."""
        if not hasattr(b, "data_ptr"):
            b = np.ascontiguousarray(b, dtype=np.float64)
        pb, db = _ptr(b)
        px, dx = _ptr(x)
        if db != dx:
            raise ValueError("b and x must both be host or both be device arrays")
        cyc = np.zeros(len(self.n_cells), dtype=np.int32)
        rr = np.zeros(len(self.n_cells))
        rc = self.lib.mg_solve(self.h, pb, px, db, cyc.ctypes.data_as(_ip), rr.ctypes.data_as(_dp))
        if rc != AMR_OK:
            e = AmrError(rc, self.lib.mg_last_error(self.h).decode())
            e.cycles, e.relres = cyc, rr
            raise e
        return cyc, rr

    MG_KINDS = ("sweep", "copy", "smooth3d", "resrestrict", "coarse", "prolong", "update", "zero", "correct64",
                "residual64", "coarse_cycle")

    def profile_vcycle(self, cap=4096):
        """One more V-cycle (after a solve), kernel by kernel: [(kind name, microseconds)]."""
        kind = np.zeros(cap, dtype=np.int32)
        us = np.zeros(cap, dtype=np.float32)
        n = C.c_int()
        _check(self.lib.mg_profile_vcycle(self.h, kind.ctypes.data_as(_ip), us.ctypes.data_as(C.POINTER(C.c_float)),
                                          cap, C.byref(n)), self.h, "mg_last_error")
        m = min(n.value, cap)
        return [(self.MG_KINDS[k], float(t)) for k, t in zip(kind[:m], us[:m])]


class RdSolver:
    """Owns one rd_handle: reaction-diffusion steps for a batch of instances.  model
    "gray-scott" (F, k) or "schnakenberg" (kappa, a, b); scheme "imex", "split" or "explicit";
    bc "periodic" or "neumann"."""

    def __init__(self, ndim, n_cells, L, Du, Dv, dt, F=0.0, k=0.0, nu1=2, nu2=2, max_cycles=50, rtol=1e-10,
                 coarse_max=8, precision="fp32", stream=None, model="gray-scott", kappa=0.0, a=0.0, b=0.0,
                 scheme="imex", bc="periodic"):
        self.lib = load()
        self.n_cells = np.ascontiguousarray(n_cells, dtype=np.int32)
        c = RdConfig()
        c.ndim, c.n_inst = ndim, len(self.n_cells)
        c.n_cells = self.n_cells.ctypes.data_as(_ip)
        c.L, c.Du, c.Dv, c.F, c.k, c.dt = L, Du, Dv, F, k, dt
        c.nu1, c.nu2, c.max_cycles, c.rtol, c.coarse_max = nu1, nu2, max_cycles, rtol, coarse_max
        c.precision = PRECISION[precision] if isinstance(precision, str) else precision
        c.stream = stream
        c.model, c.kappa, c.a, c.b = RD_MODEL[model], kappa, a, b
        c.scheme, c.bc = RD_SCHEME[scheme], MG_BC[bc]
        self.ndim = ndim
        h = _vp()
        rc = self.lib.rd_create(C.byref(c), C.byref(h))
        if rc != AMR_OK:
            raise AmrError(rc, "rd_create")
        self.h = h
        self.ncells = int(sum(int(n) ** ndim for n in self.n_cells))

    def close(self):
        if getattr(self, "h", None):
            self.lib.rd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, u, v):
        if not hasattr(u, "data_ptr"):
            u = np.ascontiguousarray(u, dtype=np.float64)
            v = np.ascontiguousarray(v, dtype=np.float64)
        pu, du = _ptr(u)
        pv, dv = _ptr(v)
        _check(self.lib.rd_set_state(self.h, pu, pv, du), self.h, "rd_last_error")

    def read_state(self, u=None, v=None):
        if u is None:
            u, v = np.zeros(self.ncells), np.zeros(self.ncells)
        pu, du = _ptr(u)
        pv, dv = _ptr(v)
        _check(self.lib.rd_read_state(self.h, pu, pv, du), self.h, "rd_last_error")
        return u, v

    def set_guess_inputs(self, kind="prev"):
        """Network input channels 2, 3: "prev" = (u*_prev, v*_prev); "residual" = the normalised
        residual of the previous-step guess per species."""
        _check(self.lib.rd_set_guess_inputs(self.h, {"prev": 0, "residual": 1}[kind]), self.h, "rd_last_error")

    def set_guess(self, net=None, scale=1.0):
        """Multigrid initial guess: None -> previous-step guess w_n; a CnnNet -> w_n + scale * net(...)."""
        _check(self.lib.rd_set_guess(self.h, net.h if net is not None else None, scale), self.h, "rd_last_error")
        self._guess = net  # keep the network alive while the handle points to it

    def last_residuals(self):
        """(initial, final) max-norm relative residuals of the last solve, shape [2, n_inst]."""
        a = np.zeros(2 * len(self.n_cells))
        b = np.zeros(2 * len(self.n_cells))
        _check(self.lib.rd_last_residuals(self.h, a.ctypes.data_as(_dp), b.ctypes.data_as(_dp)), self.h,
               "rd_last_error")
        return a.reshape(2, -1), b.reshape(2, -1)

    def extract_crops(self, inst, corners, crop, scale, out_in, out_tgt):
        """Training pairs of the last step into device float tensors [n][5][...], [n][2][...]."""
        inst = np.ascontiguousarray(inst, dtype=np.int32)
        corners = np.ascontiguousarray(corners, dtype=np.int32).reshape(-1, 3)
        _check(self.lib.rd_extract_crops(self.h, len(inst), inst.ctypes.data_as(_ip), corners.ctypes.data_as(_ip),
                                         crop, scale, out_in.data_ptr(), out_tgt.data_ptr()), self.h,
               "rd_last_error")

    def step(self, nsteps=1):
        """Returns V-cycles per step, shape [nsteps, 2, n_inst] (species-major)."""
        cyc = np.zeros((nsteps, 2, len(self.n_cells)), dtype=np.int32)
        _check(self.lib.rd_step(self.h, nsteps, cyc.ctypes.data_as(_ip)), self.h, "rd_last_error")
        return cyc


class TreeMgSolver:
    """Owns one mgt_handle: multigrid on the leaves of a 2D block quadtree (float64).
    level[k] >= 1, coords[k] = (bx, by) block coordinates at that level; leaf data
    [leaf][B*B] in the same order."""

    def __init__(self, level, coords, nb, B, L, lam, nu1=2, nu2=2, max_cycles=50, rtol=1e-10, base_rtol=1e-3,
                 coarse_max=8, stream=None):
        self.lib = load()
        self.level = np.ascontiguousarray(level, dtype=np.int32)
        self.coords = np.ascontiguousarray(coords, dtype=np.int32).reshape(-1, 2)
        c = MgtConfig(nb, nb, B, L, lam, nu1, nu2, max_cycles, rtol, base_rtol, coarse_max, stream)
        h = _vp()
        rc = self.lib.mgt_create(C.byref(c), len(self.level), self.level.ctypes.data_as(_ip),
                                 self.coords.ctypes.data_as(_ip), C.byref(h))
        if rc != AMR_OK:
            raise AmrError(rc, "mgt_create")
        self.h = h
        self.B = B
        self.n = len(self.level) * B * B

    def close(self):
        if getattr(self, "h", None):
            self.lib.mgt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, b, x, fixed_cycles=0):
        """b, x: [leaf][B*B] float64 (numpy host or torch CUDA); x updated in place.
        Returns (cycles, relative residual)."""
        if not hasattr(b, "data_ptr"):
            b = np.ascontiguousarray(b, dtype=np.float64)
        pb, db = _ptr(b)
        px, dx = _ptr(x)
        if db != dx:
            raise ValueError("b and x must both be host or both be device arrays")
        cyc = C.c_int()
        rr = C.c_double()
        rc = self.lib.mgt_solve(self.h, pb, px, db, fixed_cycles, C.byref(cyc), C.byref(rr))
        if rc != AMR_OK:
            raise AmrError(rc, self.lib.mgt_last_error(self.h).decode())
        return cyc.value, rr.value

    def apply(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.zeros_like(x)
        _check(self.lib.mgt_apply(self.h, x.ctypes.data_as(_vp), out.ctypes.data_as(_vp), 0), self.h,
               "mgt_last_error")
        return out

    def kernel_launches(self):
        n = C.c_longlong()
        _check(self.lib.mgt_kernel_launches(self.h, C.byref(n)), self.h, "mgt_last_error")
        return n.value


class TreeRdSolver:
    """Owns one rdt_handle: Gray-Scott IMEX steps on the leaves of a fixed 2D block quadtree."""

    def __init__(self, level, coords, nb, B, L, Du, Dv, F, k, dt, nu1=2, nu2=2, max_cycles=50, rtol=1e-10,
                 base_rtol=1e-3, coarse_max=8, stream=None):
        self.lib = load()
        self.level = np.ascontiguousarray(level, dtype=np.int32)
        self.coords = np.ascontiguousarray(coords, dtype=np.int32).reshape(-1, 2)
        mg = MgtConfig(nb, nb, B, L, 0.0, nu1, nu2, max_cycles, rtol, base_rtol, coarse_max, stream)
        c = RdtConfig(mg, Du, Dv, F, k, dt)
        h = _vp()
        rc = self.lib.rdt_create(C.byref(c), len(self.level), self.level.ctypes.data_as(_ip),
                                 self.coords.ctypes.data_as(_ip), C.byref(h))
        if rc != AMR_OK:
            raise AmrError(rc, "rdt_create")
        self.h = h
        self.B2 = B * B
        self.n = len(self.level) * B * B

    def close(self):
        if getattr(self, "h", None):
            self.lib.rdt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, u, v):
        u = np.ascontiguousarray(u, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        _check(self.lib.rdt_set_state(self.h, u.ctypes.data_as(_vp), v.ctypes.data_as(_vp), 0), self.h,
               "rdt_last_error")

    def read_state(self):
        u, v = np.zeros(self.n), np.zeros(self.n)
        _check(self.lib.rdt_read_state(self.h, u.ctypes.data_as(_vp), v.ctypes.data_as(_vp), 0), self.h,
               "rdt_last_error")
        return u, v

    def step(self, nsteps=1):
        cyc = np.zeros((nsteps, 2), dtype=np.int32)
        _check(self.lib.rdt_step(self.h, nsteps, cyc.ctypes.data_as(_ip)), self.h, "rdt_last_error")
        return cyc

    def leaves(self):
        n = C.c_longlong()
        _check(self.lib.rdt_num_leaves(self.h, C.byref(n)), self.h, "rdt_last_error")
        lev = np.zeros(n.value, np.int32)
        crd = np.zeros((n.value, 2), np.int32)
        _check(self.lib.rdt_leaves(self.h, lev.ctypes.data_as(_ip), crd.ctypes.data_as(_ip), n.value), self.h,
               "rdt_last_error")
        return lev, crd

    def regrid(self, refine_tol, coarsen_frac=0.5, eps=0.01, max_level=3):
        """Adapt the tree; returns the old leaves' estimator."""
        err = np.zeros(self.n // self.B2)
        n = C.c_longlong()
        _check(self.lib.rdt_regrid(self.h, refine_tol, coarsen_frac, eps, max_level, err.ctypes.data_as(_dp),
                                   C.byref(n)), self.h, "rdt_last_error")
        self.n = n.value * self.B2
        return err

    def kernel_launches(self):
        n = C.c_longlong()
        _check(self.lib.rdt_kernel_launches(self.h, C.byref(n)), self.h, "rdt_last_error")
        return n.value


class CnnNet:
    """Owns one cnn_handle (learned multigrid guess).  Images are CUDA float32
    tensors [N][C][H][W] (2D) or [N][C][D][H][W] (3D)."""

    def __init__(self, ndim=2, seed=0, stream=None):
        self.lib = load()
        self.ndim = ndim
        h = _vp()
        rc = self.lib.cnn_create(ndim, seed, stream, C.byref(h))
        if rc != AMR_OK:
            raise AmrError(rc, "cnn_create")
        self.h = h
        n = C.c_longlong()
        _check(self.lib.cnn_num_params(self.h, C.byref(n)), self.h, "cnn_last_error")
        self.nparams = n.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.cnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dims(self, x):
        if self.ndim == 2:
            N, _, H, W = x.shape
            return N, 1, H, W
        N, _, D, H, W = x.shape
        return N, D, H, W

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(self.lib.cnn_set_params(self.h, p.ctypes.data_as(C.POINTER(C.c_float)), len(p)), self.h,
               "cnn_last_error")

    def get_params(self):
        p = np.zeros(self.nparams, dtype=np.float32)
        _check(self.lib.cnn_get_params(self.h, p.ctypes.data_as(C.POINTER(C.c_float)), len(p)), self.h,
               "cnn_last_error")
        return p

    def forward(self, x, out=None):
        import torch
        N, D, H, W = self._dims(x)
        if out is None:
            out = torch.empty((x.shape[0], 2) + tuple(x.shape[2:]), dtype=torch.float32, device=x.device)
        _check(self.lib.cnn_forward(self.h, x.data_ptr(), N, D, H, W, out.data_ptr()), self.h, "cnn_last_error")
        return out

    def infer(self, x, out=None):
        """cnn_infer: the forward pass under the inference call's name."""
        import torch
        N, D, H, W = self._dims(x)
        if out is None:
            out = torch.empty((x.shape[0], 2) + tuple(x.shape[2:]), dtype=torch.float32, device=x.device)
        _check(self.lib.cnn_infer(self.h, x.data_ptr(), N, D, H, W, out.data_ptr()), self.h, "cnn_last_error")
        return out

    def gradient(self, x, target, margin=0):
        N, D, H, W = self._dims(x)
        g = np.zeros(self.nparams, dtype=np.float32)
        loss = C.c_float()
        _check(self.lib.cnn_gradient(self.h, x.data_ptr(), target.data_ptr(), N, D, H, W, margin,
                                     g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss)), self.h, "cnn_last_error")
        return loss.value, g

    def train_step(self, x, target, lr=1e-3, margin=0, want_loss=True):
        N, D, H, W = self._dims(x)
        loss = C.c_float()
        _check(self.lib.cnn_train_step(self.h, x.data_ptr(), target.data_ptr(), N, D, H, W, margin, lr,
                                       C.byref(loss) if want_loss else None), self.h, "cnn_last_error")
        return loss.value if want_loss else None

    def save(self, path):
        """Parameters to a file (cnn_save)."""
        _check(self.lib.cnn_save(self.h, os.fsencode(path)), self.h, "cnn_last_error")

    def load(self, path):
        """Parameters from a file written by save (cnn_load); resets Adam."""
        _check(self.lib.cnn_load(self.h, os.fsencode(path)), self.h, "cnn_last_error")

    def set_loss(self, kind="mse", kappa=None):
        """kind "mse" or "operator" (kappa: two values, one per output channel)."""
        k = {"mse": 0, "operator": 1}[kind]
        arr = None
        if kappa is not None:
            arr = (C.c_double * 2)(*[float(v) for v in kappa])
        _check(self.lib.cnn_set_loss(self.h, k, arr), self.h, "cnn_last_error")

    def kernel_launches(self):
        n = C.c_longlong()
        _check(self.lib.cnn_kernel_launches(self.h, C.byref(n)), self.h, "cnn_last_error")
        return n.value
