"""Python binding of the C ABI declared in include/tl.h (argument marshalling
only; every step of the solve runs in the CUDA library).

The functions keep the C names (tl_create_problem, tl_coarse_step, ...).
``Problem`` is a thin convenience wrapper around one handle.  Loading fails
loudly if libtl.so has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtl.so")

TL_OK, TL_EINVAL, TL_ENOMEM, TL_ENOCONV, TL_ESTATE, TL_ECUDA, TL_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
TL_FP64, TL_FP32_REFINED = 0, 1
TL_PREDICT, TL_CORRECT = 0, 1
TL_COARSE, TL_FINE = 0, 1
POWDER, SOLID, MELTED = 0, 1, 2


class tl_track(C.Structure):
    _fields_ = [("x0", C.c_double), ("y0", C.c_double), ("x1", C.c_double), ("y1", C.c_double),
                ("speed", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class tl_config(C.Structure):
    _fields_ = [
        ("Lx", C.c_double), ("Ly", C.c_double), ("Lz", C.c_double),
        ("NXc", C.c_int), ("NYc", C.c_int), ("NZc", C.c_int),
        ("pNXc", C.c_int), ("pNYc", C.c_int), ("pNZc", C.c_int),
        ("r", C.c_int), ("m", C.c_int),
        ("dt_coarse", C.c_double), ("T0", C.c_double), ("T_bottom", C.c_double),
        ("rho", C.c_double), ("c0", C.c_double), ("c1", C.c_double),
        ("k0", C.c_double), ("k1", C.c_double), ("Tref", C.c_double),
        ("powder_depth", C.c_double), ("powder_factor", C.c_double), ("T_melt", C.c_double),
        ("P", C.c_double), ("eta", C.c_double), ("radius", C.c_double),
        ("path", C.POINTER(tl_track)), ("ntracks", C.c_int),
        ("coarse_source", C.c_int), ("bc_weight_literal", C.c_int), ("energy", C.c_int),
        ("precision", C.c_int), ("tol", C.c_double), ("tol_inner", C.c_double),
        ("max_iter", C.c_int), ("inner_tiles", C.c_int),
        ("coupling_sweeps", C.c_int), ("coupling_tol", C.c_double), ("precond", C.c_int),
        ("latent", C.c_double), ("T_solidus", C.c_double), ("T_liquidus", C.c_double),
        ("pc_sharpness", C.c_double), ("picard_iters", C.c_int),
        ("h_conv", C.c_double), ("emissivity", C.c_double), ("T_amb", C.c_double),
        ("barrier_timeout", C.c_double), ("autotune", C.c_int), ("interface_coupling", C.c_int),
        ("stream", C.c_void_p),
        ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p),
    ]


class tl_stats(C.Structure):
    _fields_ = [
        ("macro_steps", C.c_int64), ("substeps", C.c_int64),
        ("cg_iters_fine", C.c_int64), ("cg_iters_coarse", C.c_int64),
        ("outer_iters_fine", C.c_int64), ("outer_iters_coarse", C.c_int64),
        ("solves_fine", C.c_int64), ("solves_coarse", C.c_int64),
        ("max_iters_fine", C.c_int32), ("max_iters_coarse", C.c_int32),
        ("origin", C.c_int32 * 3),
        ("patch_moves", C.c_int64),
        ("launches", C.c_int64),
        ("energy_fine_stored", C.c_double), ("energy_fine_laser", C.c_double),
        ("energy_fine_flux", C.c_double),
        ("energy_coarse_stored", C.c_double), ("energy_coarse_laser", C.c_double),
        ("energy_coarse_flux", C.c_double),
        ("time", C.c_double),
        ("coupling_resolves", C.c_int64),
        ("energy_fine_loss", C.c_double), ("energy_coarse_loss", C.c_double),
    ]


class tl_box_step_desc(C.Structure):
    _fields_ = [
        ("Lx", C.c_double), ("Ly", C.c_double), ("Lz", C.c_double),
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dt", C.c_double), ("T_bottom", C.c_double),
        ("rho", C.c_double), ("c0", C.c_double), ("c1", C.c_double),
        ("k0", C.c_double), ("k1", C.c_double), ("Tref", C.c_double),
        ("powder_factor", C.c_double), ("T_melt", C.c_double),
        ("P", C.c_double), ("eta", C.c_double), ("radius", C.c_double),
        ("xc", C.c_double), ("yc", C.c_double), ("laser_on", C.c_int),
        ("tol", C.c_double), ("max_iter", C.c_int),
    ]


TL_NOALLOC_MAX_NODES = 65536

EXPORTS = [
    "tl_create_problem", "tl_coarse_step", "tl_fine_substeps", "tl_restrict", "tl_macro_steps",
    "tl_sync", "tl_node_count", "tl_get_temperature", "tl_get_state", "tl_get_stats",
    "tl_destroy_problem", "tl_status_string", "tl_box_step_noalloc", "tl_trace_last_solve",
    "tl_batch_create", "tl_batch_add", "tl_batch_round", "tl_batch_poll", "tl_batch_info", "tl_batch_destroy",
    "tl_checkpoint_size", "tl_checkpoint_save", "tl_checkpoint_load", "tl_get_tiling",
]

_lib = None


def load(path=LIB_PATH):
    """Load libtl.so and declare the signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2110_12932_gb300.build.build()")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.tl_create_problem.argtypes = [C.POINTER(tl_config), C.POINTER(P)]
    lib.tl_create_problem.restype = C.c_int
    lib.tl_coarse_step.argtypes = [P, C.c_int]
    lib.tl_coarse_step.restype = C.c_int
    lib.tl_fine_substeps.argtypes = [P, C.c_int]
    lib.tl_fine_substeps.restype = C.c_int
    lib.tl_restrict.argtypes = [P]
    lib.tl_restrict.restype = C.c_int
    lib.tl_macro_steps.argtypes = [P, C.c_int]
    lib.tl_macro_steps.restype = C.c_int
    lib.tl_sync.argtypes = [P]
    lib.tl_sync.restype = C.c_int
    lib.tl_node_count.argtypes = [P, C.c_int]
    lib.tl_node_count.restype = C.c_size_t
    lib.tl_get_temperature.argtypes = [P, C.c_int, C.POINTER(C.c_double), C.c_size_t, C.POINTER(C.c_int)]
    lib.tl_get_temperature.restype = C.c_int
    lib.tl_get_state.argtypes = [P, C.c_int, C.POINTER(C.c_uint8), C.c_size_t]
    lib.tl_get_state.restype = C.c_int
    lib.tl_get_stats.argtypes = [P, C.POINTER(tl_stats)]
    lib.tl_get_stats.restype = C.c_int
    lib.tl_destroy_problem.argtypes = [P]
    lib.tl_destroy_problem.restype = None
    lib.tl_status_string.argtypes = [C.c_int]
    lib.tl_status_string.restype = C.c_char_p
    lib.tl_box_step_noalloc.argtypes = [C.POINTER(tl_box_step_desc), C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p]
    lib.tl_box_step_noalloc.restype = C.c_int
    lib.tl_trace_last_solve.argtypes = [P, C.c_int, C.POINTER(C.c_uint64), C.c_size_t, C.POINTER(C.c_size_t)]
    lib.tl_checkpoint_size.argtypes = [P, C.POINTER(C.c_size_t)]
    lib.tl_checkpoint_save.argtypes = [P, C.c_void_p, C.c_size_t]
    lib.tl_checkpoint_load.argtypes = [P, C.c_void_p, C.c_size_t]
    lib.tl_trace_last_solve.restype = C.c_int
    lib.tl_batch_create.argtypes = [C.c_void_p, C.c_int, C.c_int, C.POINTER(P)]
    lib.tl_batch_create.restype = C.c_int
    lib.tl_batch_add.argtypes = [P, P, C.c_int, C.POINTER(C.c_int)]
    lib.tl_batch_add.restype = C.c_int
    lib.tl_batch_round.argtypes = [P, C.POINTER(C.c_int)]
    lib.tl_batch_round.restype = C.c_int
    lib.tl_batch_poll.argtypes = [P, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int)]
    lib.tl_batch_poll.restype = C.c_int
    lib.tl_batch_info.argtypes = [P, C.POINTER(C.c_int), C.POINTER(C.c_longlong)]
    lib.tl_batch_info.restype = C.c_int
    lib.tl_get_tiling.argtypes = [P, C.c_int, C.POINTER(C.c_int32)]
    lib.tl_get_tiling.restype = C.c_int
    lib.tl_batch_destroy.argtypes = [P]
    lib.tl_batch_destroy.restype = None
    _lib = lib
    return lib


class TLError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {tl_status_string(status)} ({status})")


def tl_status_string(status):
    return load().tl_status_string(int(status)).decode()


def make_config(cfg, stream=None):
    """tl_config from a workload dict (keys = tl_config fields + tracks).
    Returns (config, keep-alive objects)."""
    c = tl_config()
    for name, _ in tl_config._fields_:
        if name in ("path", "ntracks", "stream", "alloc", "free", "alloc_ctx"):
            continue
        if name in cfg:
            setattr(c, name, cfg[name])
    tracks = list(cfg.get("tracks", []))
    arr = (tl_track * max(1, len(tracks)))()
    for j, t in enumerate(tracks):
        arr[j] = tl_track(*[float(v) for v in t])
    c.path = C.cast(arr, C.POINTER(tl_track))
    c.ntracks = len(tracks)
    c.stream = stream
    return c, [arr]


def tl_create_problem(cfg, stream=None):
    """Create a problem from a workload dict; returns (status, handle)."""
    lib = load()
    c, keep = make_config(cfg, stream)
    h = C.c_void_p()
    st = lib.tl_create_problem(C.byref(c), C.byref(h))
    return st, h


def tl_coarse_step(h, phase):
    return load().tl_coarse_step(h, int(phase))


def tl_fine_substeps(h, nsub):
    return load().tl_fine_substeps(h, int(nsub))


def tl_restrict(h):
    return load().tl_restrict(h)


def tl_macro_steps(h, n):
    return load().tl_macro_steps(h, int(n))


def tl_sync(h):
    return load().tl_sync(h)


def tl_node_count(h, level):
    return int(load().tl_node_count(h, int(level)))


def tl_get_temperature(h, level, out=None):
    """Returns (status, array, origin)."""
    lib = load()
    n = tl_node_count(h, level)
    if out is None:
        out = np.empty(n, dtype=np.float64)
    org = (C.c_int * 3)()
    st = lib.tl_get_temperature(h, int(level), out.ctypes.data_as(C.POINTER(C.c_double)), out.size, org)
    return st, out, tuple(org)


def tl_get_state(h, level, n):
    out = np.empty(n, dtype=np.uint8)
    st = load().tl_get_state(h, int(level), out.ctypes.data_as(C.POINTER(C.c_uint8)), n)
    return st, out


def tl_get_stats(h):
    s = tl_stats()
    st = load().tl_get_stats(h, C.byref(s))
    return st, s


def tl_destroy_problem(h):
    load().tl_destroy_problem(h)


def tl_box_step_noalloc(desc, T_in_ptr, T_out_ptr, state_ptr, stream=None):
    """One allocation-free backward-Euler step (see include/tl.h); the
    pointers are device addresses (ints), desc a tl_box_step_desc."""
    return load().tl_box_step_noalloc(C.byref(desc), C.c_void_p(T_in_ptr), C.c_void_p(T_out_ptr),
                                      C.c_void_p(state_ptr), C.c_void_p(stream))


TRACE_MARKS = {0: "start", 1: "phase0", 2: "rhs", 3: "resid", 4: "cg_pass", 5: "outer_init",
               6: "outer_apply", 7: "outer_end", 8: "update", 9: "end", 10: "cg_apply",
               11: "rr_value", 12: "breakdown_value", 13: "cg_update", 14: "cg_u_start", 15: "cg_u_end",
               16: "cg_precond", 17: "p0_elems", 18: "p0_dirichlet", 19: "p0_load", 20: "end_elems",
               21: "end_dirichlet"}


def tl_checkpoint_size(h):
    n = C.c_size_t()
    st = load().tl_checkpoint_size(h, C.byref(n))
    return st, n.value


def tl_checkpoint_save(h):
    """Returns (status, numpy uint8 buffer)."""
    st, n = tl_checkpoint_size(h)
    if st != TL_OK:
        return st, None
    buf = np.empty(n, dtype=np.uint8)
    st = load().tl_checkpoint_save(h, buf.ctypes.data_as(C.c_void_p), n)
    return st, buf


def tl_checkpoint_load(h, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    return load().tl_checkpoint_load(h, buf.ctypes.data_as(C.c_void_p), buf.size)


def tl_trace_last_solve(h, level, cap=1024):
    """Returns (status, [(marker, ns), ...]) of the level's most recent solve."""
    buf = (C.c_uint64 * (2 * cap))()
    n = C.c_size_t()
    st = load().tl_trace_last_solve(h, int(level), buf, cap, C.byref(n))
    m = min(n.value, cap)
    return st, [(int(buf[2 * i]), int(buf[2 * i + 1])) for i in range(m)]


def _check(st, what):
    if st != TL_OK:
        raise TLError(st, what)


class Problem:
    """One two-level problem on the GPU (see include/tl.h)."""

    def __init__(self, cfg, stream=None):
        self.cfg = dict(cfg)
        st, self.h = tl_create_problem(self.cfg, stream)
        _check(st, "tl_create_problem")
        r = self.cfg["r"]
        self.fine_elems = (self.cfg["pNXc"] * r) * (self.cfg["pNYc"] * r) * (self.cfg["pNZc"] * r)
        self.coarse_elems = self.cfg["NXc"] * self.cfg["NYc"] * self.cfg["NZc"]

    def predict(self):
        _check(tl_coarse_step(self.h, TL_PREDICT), "tl_coarse_step(PREDICT)")

    def fine_substeps(self, nsub):
        _check(tl_fine_substeps(self.h, nsub), "tl_fine_substeps")

    def restrict(self):
        _check(tl_restrict(self.h), "tl_restrict")

    def correct(self):
        _check(tl_coarse_step(self.h, TL_CORRECT), "tl_coarse_step(CORRECT)")

    def macro_steps(self, n):
        _check(tl_macro_steps(self.h, n), "tl_macro_steps")

    def sync(self):
        return tl_sync(self.h)

    def temperature(self, level):
        st, arr, org = tl_get_temperature(self.h, level)
        _check(st, "tl_get_temperature")
        return arr, org

    def state(self, level):
        n = self.fine_elems if level == TL_FINE else self.coarse_elems
        st, arr = tl_get_state(self.h, level, n)
        _check(st, "tl_get_state")
        return arr

    def stats(self):
        st, s = tl_get_stats(self.h)
        _check(st, "tl_get_stats")
        return {name: (list(getattr(s, name)) if name == "origin" else getattr(s, name))
                for name, _ in tl_stats._fields_}

    def tiling(self, level):
        """The level's tilings (see tl_get_tiling)."""
        out = (C.c_int32 * 11)()
        _check(load().tl_get_tiling(self.h, int(level), out), "tl_get_tiling")
        v = list(out)
        return {"element": v[0:3], "wide": v[3:6], "precond": v[6:9], "grid": v[9], "tuned": bool(v[10])}

    def trace(self, level):
        st, ev = tl_trace_last_solve(self.h, level)
        _check(st, "tl_trace_last_solve")
        return ev

    def checkpoint(self):
        """The problem's state between macro steps as an opaque byte buffer."""
        st, buf = tl_checkpoint_save(self.h)
        _check(st, "tl_checkpoint_save")
        return buf

    def restore(self, buf):
        _check(tl_checkpoint_load(self.h, buf), "tl_checkpoint_load")

    def close(self):
        if self.h:
            tl_destroy_problem(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many problems advanced together by one persistent kernel per launch
    (see include/tl.h, batched jobs)."""

    def __init__(self, launches_per_round=10, max_jobs=256, stream=None):
        lib = load()
        h = C.c_void_p()
        _check(lib.tl_batch_create(C.c_void_p(stream), int(launches_per_round), int(max_jobs), C.byref(h)),
               "tl_batch_create")
        self.h = h
        self.jobs = {}

    def add(self, prob, macro_steps):
        jid = C.c_int()
        _check(load().tl_batch_add(self.h, prob.h, int(macro_steps), C.byref(jid)), "tl_batch_add")
        self.jobs[jid.value] = prob
        return jid.value

    def round(self):
        act = C.c_int()
        _check(load().tl_batch_round(self.h, C.byref(act)), "tl_batch_round")
        return act.value

    def poll(self, cap=512):
        ids = (C.c_int * cap)()
        n = C.c_int()
        _check(load().tl_batch_poll(self.h, ids, cap, C.byref(n)), "tl_batch_poll")
        return [self.jobs.pop(ids[i]) for i in range(n.value)]

    def info(self):
        a, l = C.c_int(), C.c_longlong()
        _check(load().tl_batch_info(self.h, C.byref(a), C.byref(l)), "tl_batch_info")
        return {"active": a.value, "launches": l.value}

    def run(self):
        """Rounds until every job finished; returns the problems in finishing order."""
        done = []
        while self.jobs:
            self.round()
            done += self.poll()
        return done

    def close(self):
        if self.h:
            load().tl_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
