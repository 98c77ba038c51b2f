"""FP64 CPU oracle for the collision hot path of arXiv 2508.06771.

Test infrastructure only: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may load it.  The product (the CUDA library in
``paper_2508_06771_gb300``) never imports this module and shares no code with
it.  The arithmetic lives in ``ltpc_oracle.c`` (plain sequential C, FP64,
compiled without floating-point contraction); this file only builds that
library and marshals numpy arrays through ctypes.

Pinning status: every function is pinned by a ``-m "not gpu"`` test against
something other than itself (known-answer vectors, numpy routines, closed-form
physics, brute force); see the header of ``ltpc_oracle.c`` and
``mlp_oracle.c`` for the list.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["ltpc_oracle.c", "mlp_oracle.c"]
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

TAG_PARTICLE, TAG_PAIR, TAG_SCATTER, TAG_SECONDARY, TAG_PERM = 1, 2, 3, 4, 5
OK, EINVAL, ECAPACITY = 0, -1, -2
PAIR_KEY, PAIR_BIJECTION = 0, 1
BIJ_MIN_N = 4097          # in the bijection mode, cells of at least this many particles use it


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, no FP contraction)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIB_PATH):
        mt = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= mt for s in srcs):
            return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, *srcs, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [
        ("mass", C.c_double), ("charge", C.c_double), ("eps0", C.c_double),
        ("weight", C.c_double), ("n_neutral", C.c_double), ("mass_neutral", C.c_double),
        ("sigma_el", C.c_double), ("sigma_ion", C.c_double), ("e_ion", C.c_double),
        ("seed", C.c_uint64), ("odd_mode", C.c_int32), ("correction", C.c_int32),
        ("pairing_mode", C.c_int32), ("selection", C.c_int32), ("cell_ids", C.c_void_p),
        ("xs_el", C.c_void_p), ("xs_ion", C.c_void_p), ("sigma_max", C.c_double),
    ]


class Xs(C.Structure):
    """A tabulated cross section (orc_xs): piecewise cubic on a uniform ln E grid."""
    _fields_ = [("pieces", C.c_int32), ("zero_below", C.c_int32), ("lnE0", C.c_double), ("h", C.c_double),
                ("coef", C.c_void_p)]


def _xs(table):
    coef = np.ascontiguousarray(table["coef"], dtype=np.float64)
    x = Xs(int(table["pieces"]), int(table["zero_below"]), float(table["lnE0"]), float(table["h"]), coef.ctypes.data)
    x._coef = coef
    return x


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            u32p, u64p, i32p, f64p, i64p = (C.POINTER(C.c_uint32), C.POINTER(C.c_uint64),
                                           C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                           C.POINTER(C.c_int64))
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_uniform.argtypes = [C.c_uint32]
            L.orc_uniform.restype = C.c_double
            L.orc_group.argtypes = [C.c_int64, C.c_int32, i32p, u32p, u64p, u32p]
            L.orc_pair_order.argtypes = [C.c_int64, C.c_int32, i32p, C.c_uint64, C.c_uint32, u64p, u32p]
            L.orc_ta_pair.argtypes = [f64p, f64p, C.c_double, u32p]
            L.orc_ta_coefficient.argtypes = [C.POINTER(Params), C.c_double, C.c_double, C.c_double]
            L.orc_ta_coefficient.restype = C.c_double
            L.orc_nrl_lnlambda.argtypes = [C.c_double, C.c_double]
            L.orc_nrl_lnlambda.restype = C.c_double
            L.orc_coulomb.argtypes = [C.c_int64, C.c_int32, i32p, f64p, f64p, f64p, f64p, f64p, f64p,
                                      C.POINTER(Params), C.c_uint32]
            L.orc_coulomb_ids.argtypes = [C.c_int64, C.c_int32, i32p, u32p, f64p, f64p, f64p, f64p, f64p, f64p,
                                          C.POINTER(Params), C.c_uint32]
            L.orc_pair_order_ids.argtypes = [C.c_int64, C.c_int32, i32p, u32p, C.c_uint64, C.c_uint32, u64p, u32p]
            L.orc_neutral.argtypes = [i64p, C.c_int64, C.c_int32, i32p, f64p, f64p, f64p, f64p, f64p,
                                      C.POINTER(Params), C.c_uint32, i64p, C.POINTER(C.c_int8), f64p]
            L.orc_neutral_ids.argtypes = [i64p, C.c_int64, C.c_int32, i32p, u32p, f64p, f64p, f64p, f64p, f64p,
                                          C.POINTER(Params), C.c_uint32, i64p, C.POINTER(C.c_int8), f64p]
            L.orc_energy_bin.argtypes = [C.c_double]
            L.orc_energy_bin.restype = C.c_int
            L.orc_moments.argtypes = [C.c_int64, C.c_int32, i32p, f64p, f64p, f64p, C.POINTER(Params),
                                      f64p, u32p]
            L.orc_step.argtypes = [i64p, C.c_int64, C.c_int32, i32p, f64p, f64p, f64p, f64p, f64p, f64p,
                                   f64p, C.POINTER(Params), C.c_uint32, C.c_int, C.c_int, f64p, u32p, i64p]
            L.orc_bij_table.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, u32p, u32p]
            L.orc_push.argtypes = [C.c_int64, C.c_int32, i32p, f64p, f64p, f64p, f64p, C.c_double, C.c_int, i64p]
            L.orc_recombine.argtypes = [C.c_int64, C.c_int32, i32p, u32p, f64p, f64p, f64p, f64p, f64p,
                                        C.POINTER(Params), C.c_uint32, C.c_double, C.c_double, i64p]
            L.orc_bin.argtypes = [C.c_double, C.c_double, C.c_int32]
            L.orc_xs_eval.argtypes = [C.c_void_p, C.c_double]
            L.orc_xs_eval.restype = C.c_double
            L.orc_bin.restype = C.c_int
            L.orc_pair_order_mode.argtypes = [C.c_int64, C.c_int32, i32p, u32p, C.POINTER(Params), C.c_uint32,
                                              u64p, u32p]
            _mlp_argtypes(L)
        return _lib


def _check(rc):
    if rc != OK:
        raise RuntimeError(f"oracle call failed with code {rc}")


# ----------------------------------------------------------------------------- RNG
def philox(ctr, key):
    """Philox4x32-10 block: ``ctr`` 4 words, ``key`` 2 words -> 4 words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def draw(seed: int, ident: int, step: int, tag: int):
    """The block a stream uses: counter (id lo, step, tag, id hi), key = seed."""
    return philox([ident & 0xFFFFFFFF, step & 0xFFFFFFFF, tag, ident >> 32],
                  [seed & 0xFFFFFFFF, seed >> 32])


def uniform(w: int) -> float:
    return lib().orc_uniform(int(w))


# ----------------------------------------------------------------------------- grouping
def group(cell: np.ndarray, M: int):
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    n = cell.size
    counts = np.zeros(M, dtype=np.uint32)
    cs = np.zeros(M + 1, dtype=np.uint64)
    perm = np.zeros(max(n, 1), dtype=np.uint32)
    _check(lib().orc_group(n, M, _p(cell, C.c_int32), _p(counts, C.c_uint32), _p(cs, C.c_uint64),
                           _p(perm, C.c_uint32)))
    return counts, cs, perm[:n]


def pair_order(cell: np.ndarray, M: int, seed: int, step: int):
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    n = cell.size
    cs = np.zeros(M + 1, dtype=np.uint64)
    order = np.zeros(max(n, 1), dtype=np.uint32)
    _check(lib().orc_pair_order(n, M, _p(cell, C.c_int32), seed, step, _p(cs, C.c_uint64),
                                _p(order, C.c_uint32)))
    return cs, order[:n]


def bij_table(seed: int, cell: int, step: int, n: int, inverse: bool = False):
    """The pairing bijection of a cell of n particles (bijection mode): pi(r) for r in [0, n)
    (or its inverse), and the parameters (a, b, six round keys, candidate-count word)."""
    out = np.zeros(max(n, 1), np.uint32)
    prm = np.zeros(9, np.uint32)
    _check(lib().orc_bij_table(int(seed), int(cell), int(step) & 0xFFFFFFFF, int(n), 1 if inverse else 0,
                               _p(out, C.c_uint32), _p(prm, C.c_uint32)))
    return out[:n], prm


def pair_order_mode(cell: np.ndarray, M: int, params: "Params", step: int, ids: np.ndarray | None = None):
    """Pairing order under the params' pairing mode (key sort, or bijection for large cells)."""
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    n = cell.size
    cs = np.zeros(M + 1, dtype=np.uint64)
    order = np.zeros(max(n, 1), dtype=np.uint32)
    idp = None if ids is None else np.ascontiguousarray(ids, dtype=np.uint32)
    _check(lib().orc_pair_order_mode(n, M, _p(cell, C.c_int32), _p(idp, C.c_uint32), C.byref(params), step,
                                     _p(cs, C.c_uint64), _p(order, C.c_uint32)))
    return cs, order[:n]


# ----------------------------------------------------------------------------- physics
def make_params(cfg: dict, correction: bool = False, pairing_mode: int | None = None) -> Params:
    """Oracle parameters of a workload; the pairing mode defaults to the workload's
    ``pairing_mode`` (key sort when absent) and ``cell_ids`` (a subset's original cell
    indices) address the per-cell random streams."""
    mode = int(cfg.get("pairing_mode", PAIR_KEY) if pairing_mode is None else pairing_mode)
    P = Params(cfg["mass"], cfg["charge"], cfg["eps0"], cfg["weight"],
               cfg.get("n_neutral", 0.0), cfg.get("mass_neutral", 1.0),
               cfg.get("sigma_el", 0.0), cfg.get("sigma_ion", 0.0), cfg.get("e_ion", 1e30),
               int(cfg["seed"]), int(cfg.get("odd_mode", 0)), 1 if correction else 0, mode,
               int(cfg.get("selection", 0)), None, None, None, 0.0)
    xs = cfg.get("xs")                  # (elastic table, ionization table, bound on their sum)
    if xs is not None:
        P._xs = (_xs(xs[0]), _xs(xs[1]))
        P.xs_el, P.xs_ion = C.addressof(P._xs[0]), C.addressof(P._xs[1])
        P.sigma_max = float(xs[2])
    cid = cfg.get("cell_ids")
    if cid is not None:
        P._cell_ids = np.ascontiguousarray(cid, dtype=np.uint32)    # kept alive with the struct
        P.cell_ids = P._cell_ids.ctypes.data
    return P


def ta_pair(va, vb, A: float, words):
    va = np.array(va, dtype=np.float64)
    vb = np.array(vb, dtype=np.float64)
    w = np.ascontiguousarray(words, dtype=np.uint32)
    lib().orc_ta_pair(_p(va, C.c_double), _p(vb, C.c_double), float(A), _p(w, C.c_uint32))
    return va, vb


def ta_coefficient(params: Params, n_j: float, lnlam: float, dt: float) -> float:
    return lib().orc_ta_coefficient(C.byref(params), n_j, lnlam, dt)


def nrl_lnlambda(n_m3: float, T_eV: float) -> float:
    return lib().orc_nrl_lnlambda(float(n_m3), float(T_eV))


def energy_bin(E_eV: float) -> int:
    return lib().orc_energy_bin(float(E_eV))


class State:
    """Particle state held by the oracle: FP64 SoA arrays with spare capacity."""

    def __init__(self, wl: dict, capacity: int | None = None):
        n = int(wl["vx"].size)
        cap = int(capacity if capacity is not None else wl.get("capacity", n))
        self.M = int(wl["M"])
        self.n = n
        self.capacity = cap
        self.vx = np.zeros(cap, np.float64); self.vx[:n] = wl["vx"]
        self.vy = np.zeros(cap, np.float64); self.vy[:n] = wl["vy"]
        self.vz = np.zeros(cap, np.float64); self.vz[:n] = wl["vz"]
        self.cell = np.zeros(cap, np.int32); self.cell[:n] = wl["cell"]
        self.x = np.zeros(cap, np.float64)
        if wl.get("x") is not None:
            self.x[:n] = wl["x"]
        self.ids = None if wl.get("ids") is None else np.ascontiguousarray(wl["ids"], dtype=np.uint32)
        self.inv_vol = np.ascontiguousarray(wl["inv_vol"], dtype=np.float64)
        self.dt = np.ascontiguousarray(wl["dt_cell"], dtype=np.float64)
        self.lnlam = np.ascontiguousarray(wl["lnlam_cell"], dtype=np.float64)

    def views(self):
        n = self.n
        return self.vx[:n], self.vy[:n], self.vz[:n], self.cell[:n]


def coulomb(st: State, params: Params, step: int, lnlam: np.ndarray | None = None):
    """Step S1 on the oracle state; st.ids (if set) are the particles' random-stream ids."""
    ln = st.lnlam if lnlam is None else np.ascontiguousarray(lnlam, dtype=np.float64)
    ids = getattr(st, "ids", None)
    _check(lib().orc_coulomb_ids(st.n, st.M, _p(st.cell, C.c_int32), _p(ids, C.c_uint32), _p(st.vx, C.c_double),
                                 _p(st.vy, C.c_double), _p(st.vz, C.c_double), _p(st.inv_vol, C.c_double),
                                 _p(ln, C.c_double), _p(st.dt, C.c_double), C.byref(params), step))


def neutral(st: State, params: Params, step: int, with_decisions: bool = False):
    n = C.c_int64(st.n)
    counts = np.zeros(3, np.int64)
    dec = np.zeros(max(st.n, 1), np.int8) if with_decisions else None
    mar = np.zeros(max(st.n, 1), np.float64) if with_decisions else None
    ids = getattr(st, "ids", None)
    rc = lib().orc_neutral_ids(C.byref(n), st.capacity, st.M, _p(st.cell, C.c_int32), _p(ids, C.c_uint32),
                               _p(st.x, C.c_double), _p(st.vx, C.c_double), _p(st.vy, C.c_double),
                               _p(st.vz, C.c_double), _p(st.dt, C.c_double), C.byref(params), step,
                               _p(counts, C.c_int64), _p(dec, C.c_int8), _p(mar, C.c_double))
    if rc == ECAPACITY:
        raise OverflowError("oracle: particle capacity exceeded")
    _check(rc)
    old = st.n
    st.n = int(n.value)
    out = {"candidates": int(counts[0]), "elastic": int(counts[1]), "ionization": int(counts[2])}
    if with_decisions:
        out["decision"] = dec[:old]
        out["margin"] = mar[:old]
    return out


BOUNDARY_PERIODIC, BOUNDARY_ABSORB = 0, 1


def push(st: State, accel: np.ndarray, dx: float, boundary: int = BOUNDARY_PERIODIC) -> int:
    """Steps S2b/S2c on the oracle state (x along the grid axis, v_z accelerated by the
    particle's cell field); re-bins the cells; returns how many particles a wall absorbed."""
    a = np.ascontiguousarray(accel, dtype=np.float64)
    gone = C.c_int64(0)
    _check(lib().orc_push(st.n, st.M, _p(st.cell, C.c_int32), _p(st.x, C.c_double), _p(st.vz, C.c_double),
                          _p(a, C.c_double), _p(st.dt, C.c_double), float(dx), int(boundary), C.byref(gone)))
    return int(gone.value)


def recombine(st: State, params: Params, step: int, k_rec: float, de_rec: float, n_start: int | None = None) -> int:
    """Recombination C5 (RS0-RS5) on the oracle state after the neutral step of `step`, over the
    particles present at the start of the step (`n_start`, default all: the secondaries the
    neutral step appended are not in this step's pairing order); returns how many primaries
    were removed."""
    gone = C.c_int64(0)
    ids = getattr(st, "ids", None)
    n0 = st.n if n_start is None else int(n_start)
    _check(lib().orc_recombine(n0, st.M, _p(st.cell, C.c_int32), _p(ids, C.c_uint32), _p(st.vx, C.c_double),
                               _p(st.vy, C.c_double), _p(st.vz, C.c_double), _p(st.inv_vol, C.c_double),
                               _p(st.dt, C.c_double), C.byref(params), step, float(k_rec), float(de_rec),
                               C.byref(gone)))
    return int(gone.value)


def xs_eval(table: dict, E: float) -> float:
    """The oracle's value of a tabulated cross section at E [eV]."""
    x = _xs(table)
    return lib().orc_xs_eval(C.addressof(x), float(E))


def bin_position(x: float, dx: float, M: int) -> int:
    return lib().orc_bin(float(x), float(dx), int(M))


def moments(st: State, params: Params):
    mom = np.zeros((st.M, 10), np.float64)
    hist = np.zeros((st.M, 64), np.uint32)
    _check(lib().orc_moments(st.n, st.M, _p(st.cell, C.c_int32), _p(st.vx, C.c_double),
                             _p(st.vy, C.c_double), _p(st.vz, C.c_double), C.byref(params),
                             _p(mom, C.c_double), _p(hist, C.c_uint32)))
    return mom, hist


def step(st: State, params: Params, step_no: int, coulomb_on=True, neutral_on=True,
         lnlam: np.ndarray | None = None):
    """One full oracle step (S1 Coulomb, S2a neutral, S3 moments); returns (mom, hist, counts)."""
    if coulomb_on:
        coulomb(st, params, step_no, lnlam)
    counts = {"candidates": 0, "elastic": 0, "ionization": 0}
    if neutral_on:
        counts = neutral(st, params, step_no)
    mom, hist = moments(st, params)
    return mom, hist, counts


def lnlambda_from_moments(mom: np.ndarray, inv_vol: np.ndarray, weight: float, mass: float,
                          charge: float) -> np.ndarray:
    """Per-cell NRL Coulomb logarithm from a moments array (density-dependent mode)."""
    out = np.empty(mom.shape[0])
    for j in range(mom.shape[0]):
        N = mom[j, 0]
        if N < 2:
            out[j] = 2.0
            continue
        mean = mom[j, 2:5] / N
        msq = mom[j, 5:8].sum() / N
        T = mass * (msq - float(mean @ mean)) / 3.0 / charge
        out[j] = nrl_lnlambda(weight * N * inv_vol[j], T)
    return out


# ----------------------------------------------------------------------------- MLP
def _mlp_argtypes(L):
    f64p, i32p = C.POINTER(C.c_double), C.POINTER(C.c_int32)
    L.orc_bf16_round.argtypes = [C.c_double]
    L.orc_bf16_round.restype = C.c_double
    L.orc_mlp_forward.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, f64p, f64p, f64p, f64p,
                                  f64p, f64p, f64p, f64p, C.c_int32]
    L.orc_mlp_loss_backward.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, f64p, f64p, f64p,
                                        f64p, f64p, f64p, f64p, f64p, f64p, f64p, f64p, f64p, f64p,
                                        f64p, f64p, f64p, C.c_int32]
    L.orc_mlp_loss_backward.restype = C.c_double
    L.orc_adam_update.argtypes = [C.c_int64, f64p, f64p, f64p, f64p, C.c_double, C.c_double,
                                  C.c_double, C.c_double, C.c_int32]
    L.orc_gelu.argtypes = [C.c_double]
    L.orc_gelu.restype = C.c_double


def bf16_round(x: float) -> float:
    return lib().orc_bf16_round(float(x))


def gelu(z: float) -> float:
    return lib().orc_gelu(float(z))


def _dims(P):
    h, din = P["W1"].shape
    dout = P["W3"].shape[0]
    return din, h, dout


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def mlp_forward(X: np.ndarray, P: dict, bf16: bool = True) -> np.ndarray:
    """Surrogate forward pass; P holds W1 (h,din), b1, W2 (h,h), b2, W3 (dout,h), b3."""
    din, h, dout = _dims(P)
    X = _c64(X)
    B = X.shape[0]
    Y = np.zeros((B, dout), np.float64)
    ar = [_c64(P[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]
    lib().orc_mlp_forward(B, din, h, dout, _p(X, C.c_double), *[_p(a, C.c_double) for a in ar],
                          _p(Y, C.c_double), 1 if bf16 else 0)
    return Y


def mlp_loss_backward(X: np.ndarray, T: np.ndarray, P: dict, bf16: bool = True):
    """MSE loss and parameter gradients (dict with the same keys as P)."""
    din, h, dout = _dims(P)
    X = _c64(X)
    T = _c64(T)
    B = X.shape[0]
    ar = [_c64(P[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3")]
    grads = {k: np.zeros_like(a) for k, a in zip(("W1", "b1", "W2", "b2", "W3", "b3"), ar)}
    Y = np.zeros((B, dout), np.float64)
    loss = lib().orc_mlp_loss_backward(
        B, din, h, dout, _p(X, C.c_double), _p(T, C.c_double), *[_p(a, C.c_double) for a in ar],
        *[_p(grads[k], C.c_double) for k in ("W1", "b1", "W2", "b2", "W3", "b3")],
        _p(Y, C.c_double), None, 1 if bf16 else 0)
    return float(loss), grads, Y


def adam_update(w: np.ndarray, g: np.ndarray, m: np.ndarray, v: np.ndarray, t: int, lr=1e-3,
                beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam update of float64 arrays w, m, v with gradient g at step t (1-based)."""
    for a in (w, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _c64(g)
    lib().orc_adam_update(w.size, _p(w, C.c_double), _p(g, C.c_double), _p(m, C.c_double),
                          _p(v, C.c_double), lr, beta1, beta2, eps, int(t))
