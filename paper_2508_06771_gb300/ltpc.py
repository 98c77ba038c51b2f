"""Thin ctypes binding of the C ABI in ``include/ltpc.h``.

Argument marshalling only: every step of the collision path runs in the CUDA
library ``_lib/libltpc.so``.  PyTorch provides the device buffers and the
stream.  There is no CPU fallback: importing works without a GPU, but creating
a ``Collider`` needs the library and a CUDA device and raises otherwise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libltpc.so")

OK, EINVAL, ECAPACITY, ECUDA, ETIMEOUT, ENONFINITE, EUNSUPPORTED, EINTERNAL = 0, -1, -2, -3, -4, -5, -6, -7
F32, F64 = 0, 1
LOAD_SRC_DEVICE, LOAD_ASYNC = 1, 2   # flags of ltpc_load_particles
LNL_CONST, LNL_NRL = 0, 1
PAIR_KEY, PAIR_BIJECTION = 0, 1      # ltpc_config.pairing_mode
WALL_PERIODIC, WALL_ABSORB = 0, 1    # ltpc_set_field
SELECT_NULL, SELECT_PER_PARTICLE = 0, 1   # ltpc_set_cross_sections
XS_MAX_PIECES = 256

_lock = threading.Lock()
_lib = None


class LtpcError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        msg = f"{where}: {strerror(code) if _lib else code} ({code})"
        if detail:
            msg += f" [{detail}]"
        super().__init__(msg)


class Config(C.Structure):
    _fields_ = [
        ("precision", C.c_int32), ("n_cells", C.c_int32), ("capacity", C.c_int64), ("seed", C.c_uint64),
        ("mass", C.c_double), ("charge", C.c_double), ("eps0", C.c_double), ("weight", C.c_double),
        ("n_neutral", C.c_double), ("mass_neutral", C.c_double), ("sigma_el", C.c_double),
        ("sigma_ion", C.c_double), ("e_ion", C.c_double),
        ("lnlambda_mode", C.c_int32), ("correction", C.c_int32), ("has_position", C.c_int32),
        ("use_graph", C.c_int32),
        ("inv_volume", C.POINTER(C.c_double)), ("dt_factor", C.POINTER(C.c_double)),
        ("lnlambda", C.POINTER(C.c_double)), ("cache_grouping", C.c_int32), ("pairing_mode", C.c_int32),
        ("reserved", C.c_int32 * 6),
    ]


class Xsec(C.Structure):
    """One tabulated cross section (ltpc_xsec): piecewise cubic in ln E."""
    _fields_ = [("pieces", C.c_int32), ("zero_below", C.c_int32), ("lnE0", C.c_double), ("h", C.c_double),
                ("coef", C.c_void_p)]


def load_library(path: str = LIB_PATH):
    """Load libltpc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise FileNotFoundError(f"{path} not built; run paper_2508_06771_gb300/build.py")
        L = C.CDLL(path)
        vp, i32, i64, u32p, f64p = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_uint32), C.POINTER(C.c_double)
        cfgp = C.POINTER(Config)
        sig = {
            "ltpc_required_bytes": (C.c_int, [cfgp, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
            "ltpc_create": (C.c_int, [C.POINTER(vp), cfgp, vp, vp, vp]),
            "ltpc_destroy": (None, [vp]),
            "ltpc_load_particles": (C.c_int, [vp, i64, vp, vp, vp, vp, vp, C.c_int]),
            "ltpc_set_field": (C.c_int, [vp, C.c_double, vp, i32]),
            "ltpc_push": (C.c_int, [vp, C.c_double, i64]),
            "ltpc_set_recombination": (C.c_int, [vp, C.c_double, C.c_double]),
            "ltpc_set_cross_sections": (C.c_int, [vp, vp, vp, C.c_double, i32]),
            "ltpc_compact": (C.c_int, [vp]),
            "ltpc_collide_coulomb": (C.c_int, [vp, C.c_double, i64]),
            "ltpc_collide_neutral": (C.c_int, [vp, C.c_double, i64]),
            "ltpc_step": (C.c_int, [vp, C.c_double, i64]),
            "ltpc_run": (C.c_int, [vp, C.c_double, i64, i64]),
            "ltpc_profile_step": (C.c_int, [vp, C.c_double, i64, C.POINTER(C.c_float), i32, C.POINTER(i32)]),
            "ltpc_profile_phases": (C.c_int, [vp, C.c_double, i64, vp]),
            "ltpc_moments": (C.c_int, [vp, vp, vp, C.c_int]),
            "ltpc_set_moments": (C.c_int, [vp, vp, vp, C.c_int]),
            "ltpc_read_particles": (C.c_int, [vp, vp, vp, vp, vp, vp, C.POINTER(i64), C.c_int]),
            "ltpc_sync": (C.c_int, [vp]),
            "ltpc_pair_order": (C.c_int, [vp, i64, vp, vp]),
            "ltpc_grouping": (C.c_int, [vp, vp, vp, vp]),
            "ltpc_classes": (C.c_int, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32),
                                       C.POINTER(i32)]),
            "ltpc_autotune": (C.c_int, [vp, C.c_double, C.POINTER(i32)]),
            "ltpc_set_class_table": (C.c_int, [vp, i32]),
            "ltpc_group_cells_noalloc": (C.c_int, [vp, i64, i32, vp, vp, vp]),
            "ltpc_mlp_param_count": (C.c_int, []),
            "ltpc_mlp_required_bytes": (C.c_int, [i32, i32, C.POINTER(C.c_size_t)]),
            "ltpc_mlp_create": (C.c_int, [C.POINTER(vp), vp, i32, i32, C.c_uint64, vp]),
            "ltpc_mlp_destroy": (None, [vp]),
            "ltpc_mlp_set_params": (C.c_int, [vp, vp, C.c_int]),
            "ltpc_mlp_get_params": (C.c_int, [vp, vp, C.c_int]),
            "ltpc_mlp_set_norm": (C.c_int, [vp, vp, vp, vp]),
            "ltpc_mlp_forward": (C.c_int, [vp, vp, i32, vp]),
            "ltpc_mlp_gradients": (C.c_int, [vp, vp, vp, i32, vp, vp]),
            "ltpc_mlp_train_step": (C.c_int, [vp, vp, vp, i32, C.c_float, vp]),
            "ltpc_mlp_features": (C.c_int, [vp, vp, vp, vp, C.c_int]),
            "ltpc_mlp_infer": (C.c_int, [vp, vp, vp]),
            "ltpc_mlp_subsample_features": (C.c_int, [vp, vp, i32, C.c_uint32, vp, vp]),
            "ltpc_strerror": (C.c_char_p, [C.c_int]),
            "ltpc_last_cuda_error": (C.c_char_p, [vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def strerror(code: int) -> str:
    return load_library().ltpc_strerror(code).decode()


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _f64p(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Collider:
    """One collision context on the current CUDA device (see include/ltpc.h)."""

    def __init__(self, *, n_cells: int, capacity: int, inv_volume, precision: int = F32, seed: int = 0,
                 mass: float, charge: float, eps0: float, weight: float = 1.0, n_neutral: float = 0.0,
                 mass_neutral: float = 1.0, sigma_el: float = 0.0, sigma_ion: float = 0.0, e_ion: float = 1e30,
                 lnlambda_mode: int = LNL_CONST, correction: int = -1, has_position: bool = False,
                 use_graph: bool = True, dt_factor=None, lnlambda=None, device=None, stream=None,
                 cache_grouping: bool = False, pairing_mode: int = PAIR_KEY):
        import torch

        self.torch = torch
        self.L = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("ltpc needs a CUDA device")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.precision = precision
        self.dtype = torch.float32 if precision == F32 else torch.float64
        self.np_dtype = np.float32 if precision == F32 else np.float64
        self.M = int(n_cells)
        self.capacity = int(capacity)
        self._inv = np.ascontiguousarray(inv_volume, dtype=np.float64)
        self._dtf = None if dt_factor is None else np.ascontiguousarray(dt_factor, dtype=np.float64)
        self._lnl = None if lnlambda is None else np.ascontiguousarray(lnlambda, dtype=np.float64)
        cfg = Config()
        cfg.precision, cfg.n_cells, cfg.capacity, cfg.seed = precision, self.M, self.capacity, int(seed)
        cfg.mass, cfg.charge, cfg.eps0, cfg.weight = mass, charge, eps0, weight
        cfg.n_neutral, cfg.mass_neutral, cfg.sigma_el, cfg.sigma_ion, cfg.e_ion = (
            n_neutral, mass_neutral, sigma_el, sigma_ion, e_ion)
        cfg.lnlambda_mode, cfg.correction = lnlambda_mode, correction
        cfg.has_position, cfg.use_graph = int(bool(has_position)), int(bool(use_graph))
        cfg.cache_grouping = int(bool(cache_grouping))
        cfg.pairing_mode = int(pairing_mode)
        self.pairing_mode = int(pairing_mode)
        cfg.inv_volume = _f64p(self._inv)
        cfg.dt_factor = _f64p(self._dtf) if self._dtf is not None else None
        cfg.lnlambda = _f64p(self._lnl) if self._lnl is not None else None
        self.cfg = cfg
        sb, wb = C.c_size_t(), C.c_size_t()
        self._check(self.L.ltpc_required_bytes(C.byref(cfg), C.byref(sb), C.byref(wb)), "required_bytes")
        self.state_bytes, self.work_bytes = sb.value, wb.value
        with torch.cuda.device(self.device):
            self.d_state = torch.empty(self.state_bytes, dtype=torch.uint8, device=self.device)
            self.d_work = torch.empty(self.work_bytes, dtype=torch.uint8, device=self.device)
        ctx = C.c_void_p()
        rc = self.L.ltpc_create(C.byref(ctx), C.byref(cfg), _ptr(self.d_state), _ptr(self.d_work),
                                self.stream.cuda_stream)
        self._check(rc, "create")
        self.ctx = ctx

    @classmethod
    def from_workload(cls, wl: dict, precision: int | None = None, correction: int = -1, use_graph=True,
                      capacity: int | None = None, **kw):
        prec = precision if precision is not None else (F32 if wl.get("precision") == "f32" else F64)
        dt = float(np.max(wl["dt_cell"]))
        c = cls(n_cells=wl["M"], capacity=int(capacity or wl["capacity"]), inv_volume=wl["inv_vol"],
                precision=prec, seed=wl["seed"], mass=wl["mass"], charge=wl["charge"], eps0=wl["eps0"],
                weight=wl["weight"], n_neutral=wl["n_neutral"] if wl.get("neutral", True) else 0.0,
                mass_neutral=wl["mass_neutral"], sigma_el=wl["sigma_el"], sigma_ion=wl["sigma_ion"],
                e_ion=wl["e_ion"], lnlambda_mode=wl.get("lnlam_mode", 0), correction=correction,
                pairing_mode=kw.pop("pairing_mode", wl.get("pairing_mode", PAIR_KEY)),
                has_position=wl.get("x") is not None, use_graph=use_graph,
                dt_factor=np.asarray(wl["dt_cell"]) / dt, lnlambda=wl["lnlam_cell"], **kw)
        c.dt = dt
        xs, sel = wl.get("xs"), int(wl.get("selection", SELECT_NULL))
        if xs is not None or sel != SELECT_NULL:      # (elastic table, ionization table, sigma_max)
            el, ion, smax = xs if xs is not None else (None, None, 0.0)
            c.set_cross_sections(el, ion, smax, sel)
        return c

    # ------------------------------------------------------------------ plumbing
    def _check(self, rc, where):
        if rc != OK:
            detail = ""
            if rc == ECUDA and getattr(self, "ctx", None):
                detail = self.L.ltpc_last_cuda_error(self.ctx).decode()
            raise LtpcError(rc, where, detail)

    def close(self):
        if getattr(self, "ctx", None):
            self.L.ltpc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, a, dtype):
        t = self.torch
        if isinstance(a, t.Tensor):
            return a.to(device=self.device, dtype=dtype).contiguous()
        return t.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=self.device)

    # ------------------------------------------------------------------ API
    def set_field(self, dx: float, accel, boundary: int = WALL_PERIODIC):
        """Steps S2b/S2c: cells of width dx along z, per-cell acceleration accel [M] (m/s^2)."""
        self._accel = np.ascontiguousarray(accel, dtype=np.float64)
        self._check(self.L.ltpc_set_field(self.ctx, float(dx), self._accel.ctypes.data, int(boundary)), "set_field")

    def set_recombination(self, k_rec: float, de_rec: float):
        """Recombination C5: three-body rate k_rec [m^6/s], energy de_rec [eV] to the catalyte."""
        self._check(self.L.ltpc_set_recombination(self.ctx, float(k_rec), float(de_rec)), "set_recombination")

    def set_cross_sections(self, el=None, ion=None, sigma_max: float = 0.0, selection: int = SELECT_NULL):
        """Tabulated sigma_el(E) / sigma_ion(E) (dicts with pieces, zero_below, lnE0, h, coef [pieces, 4])
        and the selection method (SELECT_NULL or SELECT_PER_PARTICLE)."""
        keep, refs = [], []
        for t in (el, ion):
            if t is None:
                refs.append(None)
                continue
            coef = np.ascontiguousarray(t["coef"], dtype=np.float64)
            x = Xsec(int(t["pieces"]), int(t["zero_below"]), float(t["lnE0"]), float(t["h"]), coef.ctypes.data)
            keep.append((coef, x))
            refs.append(C.addressof(x))
        self._check(self.L.ltpc_set_cross_sections(self.ctx, refs[0], refs[1], float(sigma_max), int(selection)),
                    "set_cross_sections")

    def compact(self):
        """Rewrite the storage grouped by cell (appended particles into their cell's run, removed
        ones dropped); ids become the new storage indices."""
        self._check(self.L.ltpc_compact(self.ctx), "compact")

    def push(self, dt, step):
        self._check(self.L.ltpc_push(self.ctx, float(dt), int(step)), "push")

    def load(self, vx, vy, vz, cell, x=None):
        """Load particles from numpy arrays or tensors (copied to the device first); cell=None
        bins the positions (needs a field, see set_field)."""
        t = self.torch
        n = int(len(vx))
        vxd, vyd, vzd = (self._dev(v, self.dtype) for v in (vx, vy, vz))
        cd = self._dev(cell, t.int32) if cell is not None else None
        xd = self._dev(x, self.dtype) if x is not None else None
        self._check(self.L.ltpc_load_particles(self.ctx, n, _ptr(cd), _ptr(xd), _ptr(vxd), _ptr(vyd), _ptr(vzd),
                                               LOAD_SRC_DEVICE),
                    "load_particles")
        self._keep = (vxd, vyd, vzd, cd, xd)
        return self

    def load_host(self, vx, vy, vz, cell, x=None, asynchronous=False):
        """Load from host arrays (numpy views of pinned tensors for full bandwidth) through the
        C ABI's host path.  With `asynchronous`, the call does not wait on the stream (the arrays
        must stay alive and unchanged until the stream has copied them; errors surface at `sync`)."""
        arrs = [np.ascontiguousarray(v, dtype=self.np_dtype) for v in (vx, vy, vz)]
        c = np.ascontiguousarray(cell, dtype=np.int32)
        xa = np.ascontiguousarray(x, dtype=self.np_dtype) if x is not None else None
        p = lambda a: a.ctypes.data if a is not None else None
        flags = LOAD_ASYNC if asynchronous else 0
        self._check(self.L.ltpc_load_particles(self.ctx, c.size, p(c), p(xa), p(arrs[0]), p(arrs[1]), p(arrs[2]),
                                               flags), "load_particles")
        return self

    def load_workload(self, wl):
        return self.load(wl["vx"], wl["vy"], wl["vz"], wl["cell"], wl.get("x"))

    def collide_coulomb(self, dt, step):
        self._check(self.L.ltpc_collide_coulomb(self.ctx, float(dt), int(step)), "collide_coulomb")

    def collide_neutral(self, dt, step):
        self._check(self.L.ltpc_collide_neutral(self.ctx, float(dt), int(step)), "collide_neutral")

    def step(self, dt, step):
        self._check(self.L.ltpc_step(self.ctx, float(dt), int(step)), "step")

    def run(self, dt, step0, nsteps):
        self._check(self.L.ltpc_run(self.ctx, float(dt), int(step0), int(nsteps)), "run")

    def profile_step(self, dt, step):
        """Device milliseconds of each kernel of one (non-graph) step, in launch order."""
        ms = (C.c_float * 16)()
        n = C.c_int32()
        self._check(self.L.ltpc_profile_step(self.ctx, float(dt), int(step), ms, 16, C.byref(n)), "profile_step")
        return [ms[k] for k in range(n.value)]

    PHASES = ["fetch", "keys", "bucket_scan", "place", "rank", "pos_lookup", "gather", "coulomb", "neutral",
              "moments", "writeback"]

    def profile_phases(self, dt, step):
        """SM cycles per cell-kernel phase (summed over CTAs) for one step."""
        t = self.torch
        buf = t.zeros(16, dtype=t.int64, device=self.device)
        self._check(self.L.ltpc_profile_phases(self.ctx, float(dt), int(step), _ptr(buf)), "profile_phases")
        self.sync()
        v = buf.cpu().numpy()
        return dict(zip(self.PHASES, v[:len(self.PHASES)].tolist()))

    def sync(self):
        self._check(self.L.ltpc_sync(self.ctx), "sync")

    def sync_code(self) -> int:
        return int(self.L.ltpc_sync(self.ctx))

    def moments(self, as_numpy=True):
        t = self.torch
        mom = t.empty((self.M, 10), dtype=t.float64, device=self.device)
        hist = t.empty((self.M, 64), dtype=t.int32, device=self.device)
        self._check(self.L.ltpc_moments(self.ctx, _ptr(mom), _ptr(hist), 1), "moments")
        if as_numpy:
            self.stream.synchronize()
            return mom.cpu().numpy(), hist.cpu().numpy().view(np.uint32)
        return mom, hist

    def moments_host(self, mom: np.ndarray, hist: np.ndarray | None = None):
        """Moments straight into host arrays (synchronizing)."""
        self._check(self.L.ltpc_moments(self.ctx, mom.ctypes.data, hist.ctypes.data if hist is not None else None, 0),
                    "moments")

    def set_moments(self, mom: np.ndarray, hist: np.ndarray | None = None):
        """Restore the per-cell moments from host arrays (a checkpoint's), after a load."""
        m = np.ascontiguousarray(mom, dtype=np.float64)
        h = None if hist is None else np.ascontiguousarray(hist, dtype=np.uint32)
        self._check(self.L.ltpc_set_moments(self.ctx, m.ctypes.data, None if h is None else h.ctypes.data, 0),
                    "set_moments")

    def count(self) -> int:
        n = C.c_int64()
        self._check(self.L.ltpc_read_particles(self.ctx, None, None, None, None, None, C.byref(n), 1), "count")
        return n.value

    def read(self):
        """(vx, vy, vz, cell, x) as numpy arrays of the current particles."""
        t = self.torch
        n = self.count()
        vx, vy, vz = (t.empty(max(n, 1), dtype=self.dtype, device=self.device) for _ in range(3))
        cell = t.empty(max(n, 1), dtype=t.int32, device=self.device)
        x = t.empty(max(n, 1), dtype=self.dtype, device=self.device) if self.cfg.has_position else None
        nn = C.c_int64()
        self._check(self.L.ltpc_read_particles(self.ctx, _ptr(vx), _ptr(vy), _ptr(vz), _ptr(cell), _ptr(x),
                                               C.byref(nn), 1), "read_particles")
        out = [a[:n].cpu().numpy() for a in (vx, vy, vz, cell)]
        out.append(x[:n].cpu().numpy() if x is not None else None)
        return tuple(out)

    def pair_order(self, step):
        t = self.torch
        n = self.count()
        order = t.zeros(max(n, 1), dtype=t.int32, device=self.device)
        cs = t.zeros(self.M + 1, dtype=t.int32, device=self.device)
        self._check(self.L.ltpc_pair_order(self.ctx, int(step), _ptr(order), _ptr(cs)), "pair_order")
        self.sync()
        return cs.cpu().numpy().view(np.uint32), order[:n].cpu().numpy().view(np.uint32)

    def grouping(self):
        t = self.torch
        n = self.count()
        perm = t.zeros(max(n, 1), dtype=t.int32, device=self.device)
        cs = t.zeros(self.M + 1, dtype=t.int32, device=self.device)
        counts = t.zeros(self.M, dtype=t.int32, device=self.device)
        self._check(self.L.ltpc_grouping(self.ctx, _ptr(cs), _ptr(perm), _ptr(counts)), "grouping")
        self.sync()
        return (cs.cpu().numpy().view(np.uint32), perm[:n].cpu().numpy().view(np.uint32),
                counts.cpu().numpy().view(np.uint32))

    def classes(self):
        n = C.c_int32()
        arrs = [(C.c_int32 * 8)() for _ in range(4)]
        self._check(self.L.ltpc_classes(self.ctx, C.byref(n), *arrs), "classes")
        return [dict(cluster=arrs[0][k], threads=arrs[1][k], per_cta=arrs[2][k], max_n=arrs[3][k])
                for k in range(n.value)]

    def set_class_table(self, table: int):
        self._check(self.L.ltpc_set_class_table(self.ctx, int(table)), "set_class_table")

    def autotune(self, dt=0.0) -> int:
        ch = C.c_int32()
        self._check(self.L.ltpc_autotune(self.ctx, float(dt), C.byref(ch)), "autotune")
        return ch.value


class Surrogate:
    """Rate-coefficient network (see include/ltpc.h): features -> (k_ion, k_el)."""

    DIN, H, DOUT = 66, 128, 2

    def __init__(self, batch_max=4096, n_cells_max=4096, seed=0, device=None, stream=None):
        import torch
        self.torch = torch
        self.L = load_library()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.batch_max = int(batch_max)
        nb = C.c_size_t()
        rc = self.L.ltpc_mlp_required_bytes(self.batch_max, int(n_cells_max), C.byref(nb))
        if rc != OK:
            raise LtpcError(rc, "mlp_required_bytes")
        self.buf = torch.empty(nb.value, dtype=torch.uint8, device=self.device)
        h = C.c_void_p()
        rc = self.L.ltpc_mlp_create(C.byref(h), _ptr(self.buf), self.batch_max, int(n_cells_max), int(seed),
                                    self.stream.cuda_stream)
        if rc != OK:
            raise LtpcError(rc, "mlp_create")
        self.h = h
        self.nparam = int(self.L.ltpc_mlp_param_count())
        # the library starts with the identity normalisation (mean 0, std 1, target scale 1)
        self.norm = (np.zeros(self.DIN, np.float32), np.ones(self.DIN, np.float32), np.ones(self.DOUT, np.float32))
        self.loss_buf = torch.zeros(1, dtype=torch.float32, device=self.device)

    def _chk(self, rc, where):
        if rc != OK:
            raise LtpcError(rc, where)

    def close(self):
        if getattr(self, "h", None):
            self.L.ltpc_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # packed parameter vector <-> dict of float64 arrays (oracle layout: W1 [128][66])
    def get_params(self) -> np.ndarray:
        out = np.zeros(self.nparam, np.float32)
        self._chk(self.L.ltpc_mlp_get_params(self.h, out.ctypes.data, 0), "mlp_get_params")
        return out

    def set_params(self, flat: np.ndarray):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        self._chk(self.L.ltpc_mlp_set_params(self.h, flat.ctypes.data, 0), "mlp_set_params")

    def unpack(self, flat):
        H, D = self.H, self.DIN
        o = 0
        W1 = flat[o:o + H * 80].reshape(H, 80)[:, :D]; o += H * 80
        b1 = flat[o:o + H]; o += H
        W2 = flat[o:o + H * H].reshape(H, H); o += H * H
        b2 = flat[o:o + H]; o += H
        W3 = flat[o:o + 2 * H].reshape(2, H); o += 2 * H
        b3 = flat[o:o + 2]
        return {k: np.asarray(v, np.float64) for k, v in
                dict(W1=W1, b1=b1, W2=W2, b2=b2, W3=W3, b3=b3).items()}

    def set_norm(self, mean, std, tscale):
        m = np.ascontiguousarray(mean, np.float32)
        s_ = np.ascontiguousarray(std, np.float32)
        t = np.ascontiguousarray(tscale, np.float32)
        self._chk(self.L.ltpc_mlp_set_norm(self.h, m.ctypes.data, s_.ctypes.data, t.ctypes.data), "mlp_set_norm")
        self.norm = (m, s_, t)

    def forward(self, X):
        B = int(X.shape[0])
        Y = self.torch.empty((B, 2), dtype=self.torch.float32, device=self.device)
        self._chk(self.L.ltpc_mlp_forward(self.h, _ptr(X), B, _ptr(Y)), "mlp_forward")
        return Y

    def gradients(self, X, T):
        g = self.torch.empty(self.nparam, dtype=self.torch.float32, device=self.device)
        self._chk(self.L.ltpc_mlp_gradients(self.h, _ptr(X), _ptr(T), int(X.shape[0]), _ptr(g), _ptr(self.loss_buf)),
                  "mlp_gradients")
        return g, self.loss_buf

    def train_step(self, X, T, lr=1e-3):
        self._chk(self.L.ltpc_mlp_train_step(self.h, _ptr(X), _ptr(T), int(X.shape[0]), float(lr),
                                             _ptr(self.loss_buf)), "mlp_train_step")
        return self.loss_buf

    def features(self, col, normalize=True):
        X = self.torch.empty((col.M, 66), dtype=self.torch.float32, device=self.device)
        T = self.torch.empty((col.M, 2), dtype=self.torch.float32, device=self.device)
        self._chk(self.L.ltpc_mlp_features(col.ctx, self.h, _ptr(X), _ptr(T), int(bool(normalize))), "mlp_features")
        return X, T

    def subsample_features(self, col, per_cell, salt):
        X = self.torch.empty((col.M, 66), dtype=self.torch.float32, device=self.device)
        R = self.torch.empty((col.M, 2), dtype=self.torch.float32, device=self.device)
        self._chk(self.L.ltpc_mlp_subsample_features(col.ctx, self.h, int(per_cell), int(salt) & 0xFFFFFFFF,
                                                     _ptr(X), _ptr(R)), "mlp_subsample_features")
        return X, R

    def infer(self, col, out=None):
        R = out if out is not None else self.torch.empty((col.M, 2), dtype=self.torch.float32, device=self.device)
        self._chk(self.L.ltpc_mlp_infer(col.ctx, self.h, _ptr(R)), "mlp_infer")
        return R


NOALLOC_MAX_CELLS = 131072


def group_cells_noalloc(cell, n_cells: int, stream=None):
    """Group particle ids by cell without any device allocation by the library.

    For callers that may not allocate device memory themselves (the library keeps
    its counters in a fixed device array).  ``cell`` is a CUDA int32 tensor; the
    outputs are allocated here by the caller side (torch) and returned as
    (cell_start[n_cells + 1], perm[n]) uint32 numpy arrays.  Raises LtpcError.
    """
    import torch
    L = load_library()
    n = int(cell.numel())
    cs = torch.empty(n_cells + 1, dtype=torch.int32, device=cell.device)
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=cell.device)
    st = stream if stream is not None else torch.cuda.current_stream(cell.device)
    rc = L.ltpc_group_cells_noalloc(_ptr(cell), n, int(n_cells), _ptr(cs), _ptr(perm), st.cuda_stream)
    if rc != OK:
        raise LtpcError(rc, "group_cells_noalloc")
    return cs.cpu().numpy().view(np.uint32), perm[:n].cpu().numpy().view(np.uint32)


def header_symbols(header: str | None = None):
    """Function names declared in include/ltpc.h."""
    import re
    header = header or os.path.join(os.path.dirname(_HERE), "include", "ltpc.h")
    txt = open(header).read()
    return sorted(set(re.findall(r"\b(ltpc_[a-z0-9_]+)\s*\(", txt)))
