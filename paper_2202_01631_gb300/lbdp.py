"""ctypes binding of ``liblbdp.so`` (see ``include/lbdp.h``).

Argument marshalling only: every step of the lattice update runs in the CUDA
kernels of the library.  The functions keep the C names (``lb_create``,
``lb_set_fields``, ``lb_add_particle``, ``lb_step``, ``lb_read_fields``,
``lb_read_particles`` ...); :class:`Box` wraps a handle for convenience.

Importing this module raises if the library has not been built: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Dict, List, Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "liblbdp.so")

LB_FP64, LB_FP32, LB_FP16_SHIFT, LB_BF16_SHIFT = 0, 1, 2, 3
PRECISIONS = {"fp64": LB_FP64, "fp32": LB_FP32, "fp16": LB_FP16_SHIFT, "bf16": LB_BF16_SHIFT}
LB_OK = 0
STATUS = {0: "LB_OK", -1: "LB_ERR_PARAM", -2: "LB_ERR_NOMEM", -3: "LB_ERR_NONFINITE",
          -4: "LB_ERR_OVERLAP", -5: "LB_ERR_CUDA", -6: "LB_ERR_TIMEOUT", -7: "LB_ERR_STATE"}


class LbParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("periodic", C.c_int * 3),
        ("precision", C.c_int), ("thermo_force", C.c_int),
        ("tau", C.c_double), ("rho0", C.c_double),
        ("body_force", C.c_double * 3),
        ("A", C.c_double), ("kappa", C.c_double), ("M_psi", C.c_double),
        ("C", C.c_double), ("M_phi", C.c_double),
        ("E", C.c_double), ("phi_b", C.c_double),
        ("k_d", C.c_double),
        ("cuda_stream", C.c_void_p),
        ("scalar_scheme", C.c_int),
    ]


class LbParticleDesc(C.Structure):
    _fields_ = [
        ("pos", C.c_double * 3), ("m_hat", C.c_double * 3),
        ("R", C.c_double), ("rho_p", C.c_double), ("alpha", C.c_double),
        ("mu_plus", C.c_double), ("mu_minus", C.c_double),
        ("theta_c_deg", C.c_double), ("H", C.c_double),
        ("vel", C.c_double * 3), ("omega", C.c_double * 3),
        ("ext_force", C.c_double * 3), ("ext_torque", C.c_double * 3),
        ("fixed", C.c_int),
    ]


class LbParticleState(C.Structure):
    _fields_ = [(k, C.c_double * 3) for k in ("pos", "vel", "omega", "m_hat", "force", "torque")]


class LbbParams(C.Structure):
    _fields_ = [("precision", C.c_int), ("arena_bytes", C.c_size_t), ("graph_steps", C.c_int),
                ("cuda_stream", C.c_void_p)]


class LbsParams(C.Structure):
    _fields_ = [("precision", C.c_int), ("arena_bytes", C.c_size_t), ("chunk_steps", C.c_int),
                ("max_boxes", C.c_int), ("cuda_stream", C.c_void_p)]


class LbsRequest(C.Structure):
    _fields_ = [("box", LbParams), ("n_particles", C.c_int), ("particles", LbParticleDesc * 4),
                ("psi", C.POINTER(C.c_double)), ("phi", C.POINTER(C.c_double)),
                ("steps", C.c_longlong), ("arrival", C.c_double),
                ("out_psi", C.POINTER(C.c_double)), ("out_phi", C.POINTER(C.c_double))]


class LbsResult(C.Structure):
    _fields_ = [("id", C.c_longlong), ("status", C.c_int),
                ("arrival", C.c_double), ("admitted", C.c_double), ("done", C.c_double),
                ("n_particles", C.c_int), ("particles", LbParticleState * 4), ("sums", C.c_double * 3)]


class LbError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__("%s: %s (%s)" % (where, STATUS.get(status, status), _err_string(status)))
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("liblbdp.so is not built (%s); run paper_2202_01631_gb300/build.py" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    P = C.POINTER
    dp = P(C.c_double)
    h = C.c_void_p
    sig = {
        "lb_create": (C.c_int, [P(LbParams), P(h)]),
        "lb_destroy": (None, [h]),
        "lb_set_fields": (C.c_int, [h, dp, dp, dp, dp]),
        "lb_add_particle": (C.c_int, [h, P(LbParticleDesc), P(C.c_int)]),
        "lb_step": (C.c_int, [h, C.c_int]),
        "lb_sync": (C.c_int, [h]),
        "lb_profile_step": (C.c_int, [h, C.c_int, dp, P(C.c_int)]),
        "lb_step_launches": (C.c_int, [h, C.c_int]),
        "lb_tune": (C.c_int, [h, C.c_int, P(C.c_int), dp]),
        "lb_set_planes": (C.c_int, [h, P(C.c_int)]),
        "lb_get_planes": (C.c_int, [h, P(C.c_int)]),
        "lb_read_fields": (C.c_int, [h, dp, dp, dp, dp]),
        "lb_read_mu": (C.c_int, [h, dp, dp]),
        "lb_read_populations": (C.c_int, [h, dp]),
        "lb_read_mask": (C.c_int, [h, P(C.c_ubyte)]),
        "lb_read_particles": (C.c_int, [h, P(LbParticleState), C.c_int, P(C.c_int)]),
        "lb_conservation": (C.c_int, [h, dp]),
        "lb_state_bytes": (C.c_int, [h, P(C.c_size_t)]),
        "lb_save_state": (C.c_int, [h, C.c_void_p, C.c_size_t]),
        "lb_load_state": (C.c_int, [h, C.c_void_p, C.c_size_t]),
        "lb_totals_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
        "lb_device_bytes": (C.c_int, [P(LbParams), P(C.c_size_t)]),
        "lb_wetting_h": (C.c_double, [C.c_double]),
        "lb_solubility_E": (C.c_double, [C.c_double, C.c_double]),
        "lb_error_string": (C.c_char_p, [C.c_int]),
        # batches, arena, server (include/lbdp_batch.h)
        "lb_arena_create": (C.c_int, [C.c_size_t, P(h)]),
        "lb_arena_alloc": (C.c_int, [h, C.c_size_t, P(C.c_size_t)]),
        "lb_arena_free": (C.c_int, [h, C.c_size_t]),
        "lb_arena_stats": (C.c_int, [h, P(C.c_size_t), P(C.c_size_t), P(C.c_int)]),
        "lb_arena_destroy": (None, [h]),
        "lbb_create": (C.c_int, [P(LbbParams), P(h)]),
        "lbb_destroy": (None, [h]),
        "lbb_box_bytes": (C.c_int, [h, P(LbParams), P(C.c_size_t)]),
        "lbb_memory": (C.c_int, [h, P(C.c_size_t), P(C.c_size_t), P(C.c_size_t)]),
        "lbb_add_box": (C.c_int, [h, P(LbParams), P(h)]),
        "lbb_num_boxes": (C.c_int, [h]),
        "lbb_set_steps": (C.c_int, [h, h, C.c_longlong]),
        "lbb_get_steps": (C.c_int, [h, h, P(C.c_longlong)]),
        "lbb_run": (C.c_int, [h, C.c_int, P(C.c_longlong)]),
        "lbb_tune": (C.c_int, [h, C.c_int, P(C.c_int), dp]),
        "lbb_set_config": (C.c_int, [h, P(C.c_int)]),
        "lbb_num_configs": (C.c_int, []),
        "lbb_config_shape": (C.c_int, [C.c_int, P(C.c_int), P(C.c_int)]),
        "lbb_sync": (C.c_int, [h]),
        "lbs_create": (C.c_int, [P(LbsParams), P(h)]),
        "lbs_destroy": (None, [h]),
        "lbs_submit": (C.c_int, [h, P(LbsRequest), P(C.c_longlong)]),
        "lbs_pump": (C.c_int, [h, C.c_double, P(C.c_int), P(C.c_int)]),
        "lbs_poll": (C.c_int, [h, P(LbsResult), C.c_int, P(C.c_int)]),
        "lbs_cancel": (C.c_int, [h, C.c_longlong, C.c_double]),
        "lbs_batch": (h, [h]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def _err_string(status: int) -> str:
    return _lib.lb_error_string(int(status)).decode()


def _check(status: int, where: str):
    if status != LB_OK:
        raise LbError(status, where)


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ---------------------------------------------------------------------------
# thin C-named wrappers
# ---------------------------------------------------------------------------

def lb_params(**kw) -> LbParams:
    """Build an :class:`LbParams` from keyword arguments (names as in C);
    ``precision`` may also be one of ``"fp64" "fp32" "fp16" "bf16"``."""
    p = LbParams()
    p.nx, p.ny, p.nz = int(kw["nx"]), int(kw["ny"]), int(kw["nz"])
    p.periodic = (C.c_int * 3)(*[int(v) for v in kw.get("periodic", (1, 1, 1))])
    prec = kw.get("precision", LB_FP64)
    p.precision = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    p.thermo_force = int(kw.get("thermo_force", 1))
    p.tau = float(kw.get("tau", 1.0))
    p.rho0 = float(kw.get("rho0", 1.0))
    p.body_force = (C.c_double * 3)(*[float(v) for v in kw.get("body_force", (0.0, 0.0, 0.0))])
    for k, d in (("A", 0.0625), ("kappa", 0.04), ("M_psi", 0.1), ("C", 0.0625), ("M_phi", 1.6),
                 ("E", 0.0), ("phi_b", 0.0), ("k_d", 0.0)):
        setattr(p, k, float(kw.get(k, d)))
    p.cuda_stream = kw.get("cuda_stream", None)
    p.scalar_scheme = int(kw.get("scalar_scheme", 0))
    return p


def lb_create(params: LbParams) -> int:
    h = C.c_void_p()
    _check(_lib.lb_create(C.byref(params), C.byref(h)), "lb_create")
    return h.value


def lb_destroy(h: int) -> None:
    _lib.lb_destroy(h)


def lb_set_fields(h, rho=None, u=None, psi=None, phi=None) -> None:
    _check(_lib.lb_set_fields(h, _dptr(rho), _dptr(u), _dptr(psi), _dptr(phi)), "lb_set_fields")


def lb_add_particle(h, desc: LbParticleDesc) -> int:
    k = C.c_int(-1)
    _check(_lib.lb_add_particle(h, C.byref(desc), C.byref(k)), "lb_add_particle")
    return k.value


def lb_step(h, nsteps: int) -> None:
    _check(_lib.lb_step(h, int(nsteps)), "lb_step")


# kernel classes of lb_profile_step, in its sequential order: the particle
# kernels before the bulk (pressure tensor and force next to the particles,
# link sums and particle update, boundary collide-stream), the fused bulk
# kernel (chemical potentials, force, collide-stream), the bulk transport,
# the boundary transport, covering
KERNEL_CLASSES = ("k_particles", "k_fused", "k_scalars", "k_scalars_particles", "k_cover")


def lb_profile_step(h, nsteps: int):
    """Run nsteps with per-kernel CUDA events; returns ({kernel: ms}, launches)."""
    ms = np.zeros(5)
    n = C.c_int(0)
    _check(_lib.lb_profile_step(h, int(nsteps), _dptr(ms), C.byref(n)), "lb_profile_step")
    return dict(zip(KERNEL_CLASSES, ms.tolist())), n.value


def lb_tune(h, reps: int = 10):
    """Time the two bulk kernels over z chunk lengths and keep the fastest;
    returns ({kernel: planes}, {kernel: ms per launch}) for k_fused, k_scalars."""
    planes = (C.c_int * 2)()
    ms = np.zeros(2)
    _check(_lib.lb_tune(h, int(reps), planes, _dptr(ms)), "lb_tune")
    return (dict(zip(("k_fused", "k_scalars"), list(planes))), dict(zip(("k_fused", "k_scalars"), ms.tolist())))


def lb_set_planes(h, fused: int, scalars: int) -> None:
    """Chunk lengths of the two bulk kernels (0 = size heuristic)."""
    planes = (C.c_int * 2)(int(fused), int(scalars))
    _check(_lib.lb_set_planes(h, planes), "lb_set_planes")


def lb_get_planes(h):
    planes = (C.c_int * 2)()
    _check(_lib.lb_get_planes(h, planes), "lb_get_planes")
    return {"k_fused": planes[0], "k_scalars": planes[1]}


def lb_step_launches(h, nsteps: int) -> int:
    n = _lib.lb_step_launches(h, int(nsteps))
    if n < 0:
        raise LbError(n, "lb_step_launches")
    return n


def lb_sync(h) -> None:
    _check(_lib.lb_sync(h), "lb_sync")


def lb_read_fields(h, rho=None, u=None, psi=None, phi=None) -> None:
    _check(_lib.lb_read_fields(h, _dptr(rho), _dptr(u), _dptr(psi), _dptr(phi)), "lb_read_fields")


def lb_read_particles(h, cap: int) -> List[LbParticleState]:
    out = (LbParticleState * max(cap, 1))()
    n = C.c_int(0)
    _check(_lib.lb_read_particles(h, out, int(cap), C.byref(n)), "lb_read_particles")
    return [out[k] for k in range(min(n.value, cap))]


def lb_conservation(h) -> np.ndarray:
    s = np.zeros(3)
    _check(_lib.lb_conservation(h, _dptr(s)), "lb_conservation")
    return s


def lb_totals_noalloc(precision, nx, ny, nz, f_ptr, psi_ptr, phi_ptr, mask_ptr, sums_ptr, stream=None) -> None:
    """FP64 totals (sum rho, psi, phi) of caller-owned device arrays into the
    device buffer ``sums_ptr``, without any device allocation (for callers
    whose device memory is owned by their own allocator).  Pointers are raw
    device addresses (ints); ``mask_ptr`` may be None."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check(_lib.lb_totals_noalloc(prec, int(nx), int(ny), int(nz), f_ptr, psi_ptr, phi_ptr, mask_ptr,
                                  sums_ptr, stream), "lb_totals_noalloc")


def lb_device_bytes(params: LbParams) -> int:
    b = C.c_size_t(0)
    _check(_lib.lb_device_bytes(C.byref(params), C.byref(b)), "lb_device_bytes")
    return int(b.value)


def lb_wetting_h(theta_c_deg: float) -> float:
    return float(_lib.lb_wetting_h(float(theta_c_deg)))


def lb_solubility_E(ratio: float, phi_b: float) -> float:
    return float(_lib.lb_solubility_E(float(ratio), float(phi_b)))


def particle_desc(**kw) -> LbParticleDesc:
    d = LbParticleDesc()
    for k in ("pos", "m_hat", "vel", "omega", "ext_force", "ext_torque"):
        v = kw.get(k, (1.0, 0.0, 0.0) if k == "m_hat" else (0.0, 0.0, 0.0))
        setattr(d, k, (C.c_double * 3)(*[float(x) for x in v]))
    d.R = float(kw["R"])
    d.rho_p = float(kw.get("rho_p", 1.0))
    d.alpha = float(kw.get("alpha", 0.0))
    d.mu_plus = float(kw.get("mu_plus", 0.0))
    d.mu_minus = float(kw.get("mu_minus", 0.0))
    if "H" in kw:
        d.theta_c_deg = math.nan
        d.H = float(kw["H"])
    else:
        d.theta_c_deg = float(kw.get("theta_c_deg", 90.0))
        d.H = 0.0
    d.fixed = int(kw.get("fixed", 0))
    return d


def box_params(precision="fp64", stream=None, **params) -> LbParams:
    """:class:`LbParams` from keyword parameters; ``solubility_ratio`` (if
    present and ``E`` absent) is mapped to ``E`` by :func:`lb_solubility_E`."""
    q = dict(params)
    if "E" not in q and "solubility_ratio" in q:
        q["E"] = lb_solubility_E(q["solubility_ratio"], q.get("phi_b", 0.0))
    q.pop("solubility_ratio", None)
    q["precision"] = precision
    if stream is not None:
        q["cuda_stream"] = stream
    return lb_params(**q)


# ---------------------------------------------------------------------------
# arena, batches, server (include/lbdp_batch.h)
# ---------------------------------------------------------------------------

def lb_arena_create(capacity: int) -> int:
    a = C.c_void_p()
    _check(_lib.lb_arena_create(int(capacity), C.byref(a)), "lb_arena_create")
    return a.value


def lb_arena_alloc(a, nbytes: int) -> int:
    off = C.c_size_t(0)
    _check(_lib.lb_arena_alloc(a, int(nbytes), C.byref(off)), "lb_arena_alloc")
    return int(off.value)


def lb_arena_free(a, offset: int) -> None:
    _check(_lib.lb_arena_free(a, int(offset)), "lb_arena_free")


def lb_arena_stats(a):
    """(used, largest_free, free_ranges)"""
    u, big, n = C.c_size_t(0), C.c_size_t(0), C.c_int(0)
    _check(_lib.lb_arena_stats(a, C.byref(u), C.byref(big), C.byref(n)), "lb_arena_stats")
    return int(u.value), int(big.value), n.value


def lb_arena_destroy(a) -> None:
    _lib.lb_arena_destroy(a)


def lbb_create(precision="fp32", arena_bytes=0, graph_steps=0, stream=None) -> int:
    p = LbbParams()
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.arena_bytes = int(arena_bytes)
    p.graph_steps = int(graph_steps)
    p.cuda_stream = stream
    b = C.c_void_p()
    _check(_lib.lbb_create(C.byref(p), C.byref(b)), "lbb_create")
    return b.value


def lbb_destroy(b) -> None:
    _lib.lbb_destroy(b)


def lbb_add_box(b, params: LbParams) -> int:
    h = C.c_void_p()
    _check(_lib.lbb_add_box(b, C.byref(params), C.byref(h)), "lbb_add_box")
    return h.value


def lbb_box_bytes(b, params: LbParams) -> int:
    n = C.c_size_t(0)
    _check(_lib.lbb_box_bytes(b, C.byref(params), C.byref(n)), "lbb_box_bytes")
    return int(n.value)


def lbb_memory(b):
    """(capacity, used, largest_free)"""
    c, u, big = C.c_size_t(0), C.c_size_t(0), C.c_size_t(0)
    _check(_lib.lbb_memory(b, C.byref(c), C.byref(u), C.byref(big)), "lbb_memory")
    return int(c.value), int(u.value), int(big.value)


def lbb_set_steps(b, h, nsteps: int) -> None:
    _check(_lib.lbb_set_steps(b, h, int(nsteps)), "lbb_set_steps")


def lbb_get_steps(b, h) -> int:
    n = C.c_longlong(0)
    _check(_lib.lbb_get_steps(b, h, C.byref(n)), "lbb_get_steps")
    return int(n.value)


def lbb_run(b, nsteps: int) -> int:
    """Queue nsteps batch steps; returns the number of kernel launches queued."""
    n = C.c_longlong(0)
    _check(_lib.lbb_run(b, int(nsteps), C.byref(n)), "lbb_run")
    return int(n.value)


# bulk kernel classes the batch autotuner times (include/lbdp_batch.h)
BATCH_KERNEL_CLASSES = ("fused", "transport")


def lbb_tune(b, reps: int = 10):
    """Autotune the z chunk of the two bulk kernels; returns the chosen
    candidate per kernel class and its time in ms."""
    k = len(BATCH_KERNEL_CLASSES)
    cfg = (C.c_int * k)()
    ms = np.zeros(k)
    _check(_lib.lbb_tune(b, int(reps), cfg, _dptr(ms)), "lbb_tune")
    return list(cfg), ms.tolist()


def lbb_set_config(b, cfg) -> None:
    k = len(BATCH_KERNEL_CLASSES)
    if len(cfg) != k:
        raise ValueError("one candidate per bulk kernel class (%d)" % k)
    _check(_lib.lbb_set_config(b, (C.c_int * k)(*[int(c) for c in cfg])), "lbb_set_config")


def lbb_num_configs() -> int:
    return int(_lib.lbb_num_configs())


def lbb_config_shape(k: int):
    """(threads per block, planes per block) of candidate k."""
    t, z = C.c_int(0), C.c_int(0)
    _check(_lib.lbb_config_shape(int(k), C.byref(t), C.byref(z)), "lbb_config_shape")
    return t.value, z.value


def lbb_sync(b) -> None:
    _check(_lib.lbb_sync(b), "lbb_sync")


class Batch:
    """Boxes of one precision mode advanced together (:func:`lbb_run`)."""

    def __init__(self, precision="fp32", arena_bytes=0, graph_steps=0, stream=None, _handle=None):
        self.precision = precision
        self.own = _handle is None
        self.h = _handle if _handle is not None else lbb_create(precision, arena_bytes, graph_steps, stream)
        self.boxes = set()

    def add_box(self, **params) -> Box:
        b = Box(precision=self.precision, _batch=self, **params)
        self.boxes.add(b)
        return b

    def box_bytes(self, **params) -> int:
        return lbb_box_bytes(self.h, box_params(self.precision, None, **params))

    def memory(self):
        return lbb_memory(self.h)

    def set_steps(self, box: Box, nsteps: int):
        lbb_set_steps(self.h, box.h, nsteps)

    def steps_left(self, box: Box) -> int:
        return lbb_get_steps(self.h, box.h)

    def run(self, nsteps: int) -> int:
        return lbb_run(self.h, nsteps)

    def tune(self, reps: int = 10):
        return lbb_tune(self.h, reps)

    def set_config(self, cfg):
        lbb_set_config(self.h, cfg)

    def sync(self):
        lbb_sync(self.h)

    def close(self):
        if getattr(self, "h", None):
            for b in list(self.boxes):
                b.h = None   # lbb_destroy destroys the member boxes
            self.boxes.clear()
            if self.own:
                lbb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous batching (:func:`lbs_pump`): requests are admitted into a
    batch as memory frees up and leave when their steps are done."""

    def __init__(self, precision="fp32", arena_bytes=0, chunk_steps=0, max_boxes=0, stream=None):
        p = LbsParams()
        p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        p.arena_bytes = int(arena_bytes)
        p.chunk_steps = int(chunk_steps)
        p.max_boxes = int(max_boxes)
        p.cuda_stream = stream
        self.precision = precision
        h = C.c_void_p()
        _check(_lib.lbs_create(C.byref(p), C.byref(h)), "lbs_create")
        self.h = h.value
        self.batch = Batch(precision, _handle=_lib.lbs_batch(self.h))
        self._keep = {}

    def submit(self, box: Dict, particles=(), psi=None, phi=None, steps=1, arrival=0.0,
               out_psi=None, out_phi=None) -> int:
        r = LbsRequest()
        r.box = box_params(self.precision, None, **box)
        r.n_particles = len(particles)
        for k, d in enumerate(particles):
            r.particles[k] = particle_desc(**d)
        keep = []
        for name, a in (("psi", psi), ("phi", phi)):
            if a is not None:
                a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
                keep.append(a)
                setattr(r, name, _dptr(a))
        for name, a in (("out_psi", out_psi), ("out_phi", out_phi)):
            if a is not None:
                if not (a.flags.c_contiguous and a.dtype == np.float64):
                    raise ValueError("%s must be a C-contiguous float64 array" % name)
                setattr(r, name, _dptr(a))
        r.steps = int(steps)
        r.arrival = float(arrival)
        rid = C.c_longlong(-1)
        _check(_lib.lbs_submit(self.h, C.byref(r), C.byref(rid)), "lbs_submit")
        self._keep[rid.value] = (out_psi, out_phi)   # output buffers stay alive until polled
        return rid.value

    def pump(self, now: float):
        """One round; returns (active, queued)."""
        a, q = C.c_int(0), C.c_int(0)
        _check(_lib.lbs_pump(self.h, float(now), C.byref(a), C.byref(q)), "lbs_pump")
        return a.value, q.value

    def cancel(self, rid: int, now: float = 0.0):
        """Cancel a queued or resident request (:func:`lbs_cancel`)."""
        _check(_lib.lbs_cancel(self.h, int(rid), float(now)), "lbs_cancel")

    def poll(self, cap: int = 64) -> List[Dict]:
        out = (LbsResult * cap)()
        n = C.c_int(0)
        _check(_lib.lbs_poll(self.h, out, cap, C.byref(n)), "lbs_poll")
        res = []
        for k in range(n.value):
            r = out[k]
            self._keep.pop(r.id, None)
            res.append(dict(id=r.id, status=r.status, arrival=r.arrival, admitted=r.admitted, done=r.done,
                            particles=[{f: np.array(getattr(r.particles[j], f)[:])
                                        for f in ("pos", "vel", "omega", "m_hat", "force", "torque")}
                                       for j in range(r.n_particles)],
                            sums=np.array(r.sums[:])))
        return res

    def close(self):
        if getattr(self, "h", None):
            self.batch.h = None
            _lib.lbs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------

class Box:
    """One simulation box on the current CUDA device.

    ``params`` take the :class:`LbParams` names; ``solubility_ratio`` (if
    present and ``E`` absent) is mapped to ``E`` by :func:`lb_solubility_E`.
    Arrays use the [nz, ny, nx] shape of the node index x + nx (y + ny z).
    """

    def __init__(self, precision="fp64", stream=None, _batch=None, **params):
        self.params = box_params(precision, stream, **params)
        self.batch = _batch
        self.h = lbb_add_box(_batch.h, self.params) if _batch is not None else lb_create(self.params)
        self.shape = (self.params.nz, self.params.ny, self.params.nx)
        self.N = self.params.nx * self.params.ny * self.params.nz
        self.np = 0

    def close(self):
        if getattr(self, "h", None):
            lb_destroy(self.h)
            self.h = None
            if self.batch is not None:
                self.batch.boxes.discard(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, rho=None, u=None, psi=None, phi=None):
        def prep(a, n):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
            if a.size != n:
                raise ValueError("field has %d values, expected %d" % (a.size, n))
            return a
        lb_set_fields(self.h, prep(rho, self.N), prep(u, 3 * self.N), prep(psi, self.N), prep(phi, self.N))

    def add_particle(self, **kw) -> int:
        k = lb_add_particle(self.h, particle_desc(**kw))
        self.np += 1
        return k

    def step(self, n: int = 1):
        lb_step(self.h, n)

    def tune(self, reps: int = 10):
        """Pick the z chunk length of each bulk kernel by timing (lb_tune)."""
        return lb_tune(self.h, reps)

    def set_planes(self, fused: int = 0, scalars: int = 0):
        lb_set_planes(self.h, fused, scalars)

    def planes(self):
        return lb_get_planes(self.h)

    def sync(self):
        lb_sync(self.h)

    def fields(self) -> Dict[str, np.ndarray]:
        N = self.N
        rho, u, psi, phi = np.empty(N), np.empty(3 * N), np.empty(N), np.empty(N)
        lb_read_fields(self.h, rho, u, psi, phi)
        s = self.shape
        return dict(rho=rho.reshape(s), u=u.reshape((3,) + s), psi=psi.reshape(s), phi=phi.reshape(s))

    def mu(self):
        a, b = np.empty(self.N), np.empty(self.N)
        _check(_lib.lb_read_mu(self.h, _dptr(a), _dptr(b)), "lb_read_mu")
        return a.reshape(self.shape), b.reshape(self.shape)

    def populations(self) -> np.ndarray:
        f = np.empty(19 * self.N)
        _check(_lib.lb_read_populations(self.h, _dptr(f)), "lb_read_populations")
        return f.reshape((19,) + self.shape)

    def save_state(self) -> bytes:
        """The whole state after the last step (:func:`lb_save_state`)."""
        n = C.c_size_t(0)
        _check(_lib.lb_state_bytes(self.h, C.byref(n)), "lb_state_bytes")
        buf = (C.c_ubyte * n.value)()
        _check(_lib.lb_save_state(self.h, buf, n.value), "lb_save_state")
        return bytes(buf)

    def load_state(self, blob: bytes):
        """Restore a state saved from a box of the same size and model
        (:func:`lb_load_state`); its particles replace this box's."""
        buf = (C.c_ubyte * len(blob)).from_buffer_copy(blob)
        _check(_lib.lb_load_state(self.h, buf, len(blob)), "lb_load_state")
        self.np = len(self.particles_raw())

    def particles_raw(self):
        return lb_read_particles(self.h, 64)

    def mask(self) -> np.ndarray:
        m = np.empty(self.N, dtype=np.uint8)
        _check(_lib.lb_read_mask(self.h, m.ctypes.data_as(C.POINTER(C.c_ubyte))), "lb_read_mask")
        return m.reshape(self.shape)

    def particles(self) -> List[Dict[str, np.ndarray]]:
        st = lb_read_particles(self.h, max(self.np, 1))
        return [{f: np.array(getattr(s, f)[:]) for f in ("pos", "vel", "omega", "m_hat", "force", "torque")}
                for s in st]

    def conservation(self) -> np.ndarray:
        return lb_conservation(self.h)
