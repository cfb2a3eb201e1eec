"""Python wrapper of the FP64 CPU oracle (``lbref.c``).

TEST INFRASTRUCTURE ONLY: the plain, slow definition of the lattice step that
the CUDA library is checked against.  Only ``tests/``, the smoke check and the
CPU-baseline leg of the benchmark import this module; the library never does.

The C source is compiled on first use with ``gcc -O2 -ffp-contract=off`` (no
fused multiply-adds, so the oracle gives the same bits on x86_64 and aarch64),
with ``-fopenmp`` where the compiler supports it: ``set_threads`` then runs
the independent node loops on several cores, with bit-identical results.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbref.c")
_HDR = os.path.join(_HERE, "lbref.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liblbref.so")
_lock = threading.Lock()
_lib = None


class RefParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("periodic", C.c_int * 3),
        ("tau", C.c_double), ("rho0", C.c_double),
        ("body_force", C.c_double * 3),
        ("A", C.c_double), ("kappa", C.c_double), ("M_psi", C.c_double),
        ("C", C.c_double), ("M_phi", C.c_double), ("E", C.c_double),
        ("phi_b", C.c_double), ("k_d", C.c_double),
        ("thermo_force", C.c_int),
        ("scalar_scheme", C.c_int),
    ]


class RefParticleDesc(C.Structure):
    _fields_ = [
        ("pos", C.c_double * 3), ("m_hat", C.c_double * 3),
        ("R", C.c_double), ("rho_p", C.c_double), ("alpha", C.c_double),
        ("mu_plus", C.c_double), ("mu_minus", C.c_double),
        ("H", C.c_double),
        ("vel", C.c_double * 3), ("omega", C.c_double * 3),
        ("ext_force", C.c_double * 3), ("ext_torque", C.c_double * 3),
        ("fixed", C.c_int),
    ]


class RefParticleState(C.Structure):
    _fields_ = [(k, C.c_double * 3) for k in ("pos", "vel", "omega", "m_hat", "force", "torque")]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liblbref.so`` (idempotent)."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= newest):
            return _LIB_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
               "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        r = subprocess.run(cmd[:-1] + ["-fopenmp", "-lm"], capture_output=True, text=True)
        if r.returncode != 0:   # no OpenMP runtime: one thread
            subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    P = C.POINTER
    dp = P(C.c_double)
    lib.ref_create.restype = C.c_void_p
    lib.ref_create.argtypes = [P(RefParams)]
    lib.ref_destroy.argtypes = [C.c_void_p]
    lib.ref_set_fields.argtypes = [C.c_void_p, dp, dp, dp, dp]
    lib.ref_add_particle.argtypes = [C.c_void_p, P(RefParticleDesc)]
    lib.ref_step.argtypes = [C.c_void_p, C.c_int]
    lib.ref_read_fields.argtypes = [C.c_void_p, dp, dp, dp, dp]
    lib.ref_read_mu.argtypes = [C.c_void_p, dp, dp]
    lib.ref_read_populations.argtypes = [C.c_void_p, dp]
    lib.ref_read_mask.argtypes = [C.c_void_p, P(C.c_ubyte)]
    lib.ref_read_particles.argtypes = [C.c_void_p, P(RefParticleState), C.c_int]
    lib.ref_conservation.argtypes = [C.c_void_p, dp]
    lib.ref_error.argtypes = [C.c_void_p]
    lib.ref_fluid_count.argtypes = [C.c_void_p]
    lib.ref_fluid_count.restype = C.c_long
    lib.ref_set_threads.argtypes = [C.c_int]
    lib.ref_set_threads.restype = C.c_int
    lib.ref_wetting_h.argtypes = [C.c_double]
    lib.ref_wetting_h.restype = C.c_double
    _lib = lib
    return lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's node loops (0: all cores); returns the count in
    use (1 when the oracle was built without OpenMP)."""
    return int(_load().ref_set_threads(int(n)))


def wetting_h(theta_deg: float) -> float:
    """h = H / sqrt(kappa A) for a contact angle in degrees (wetting relation)."""
    return _load().ref_wetting_h(float(theta_deg))


def solubility_E(ratio: float, phi_b: float = 1.0) -> float:
    """E for a solubility ratio r = phi0(+1) / phi0(-1) with phi0 = phi_b + E tanh(psi)."""
    t = math.tanh(1.0)
    return phi_b * (ratio - 1.0) / ((ratio + 1.0) * t)


class Oracle:
    """One simulation box stepped by the FP64 CPU oracle.

    ``params`` is a dict with the keys of :class:`RefParams` (missing keys take
    the defaults below); particles are dicts with the keys of
    :class:`RefParticleDesc` plus an optional ``theta_c_deg`` that is mapped to
    ``H`` by the wetting relation.
    """

    DEFAULTS = dict(periodic=(1, 1, 1), tau=1.0, rho0=1.0, body_force=(0.0, 0.0, 0.0),
                    A=0.0625, kappa=0.04, M_psi=0.1, C=0.0625, M_phi=1.6, E=0.0,
                    phi_b=0.0, k_d=0.0, thermo_force=1, scalar_scheme=0)

    def __init__(self, params: dict):
        self.lib = _load()
        q = dict(self.DEFAULTS)
        q.update(params)
        if "solubility_ratio" in q:
            r = q.pop("solubility_ratio")
            if "E" not in params:
                q["E"] = solubility_E(r, q["phi_b"])
        q.pop("precision", None)
        self.params = q
        p = RefParams()
        p.nx, p.ny, p.nz = int(q["nx"]), int(q["ny"]), int(q["nz"])
        p.periodic = (C.c_int * 3)(*[int(v) for v in q["periodic"]])
        p.body_force = (C.c_double * 3)(*[float(v) for v in q["body_force"]])
        for k in ("tau", "rho0", "A", "kappa", "M_psi", "C", "M_phi", "E", "phi_b", "k_d"):
            setattr(p, k, float(q[k]))
        p.thermo_force = int(q["thermo_force"])
        p.scalar_scheme = int(q["scalar_scheme"])
        self.shape = (p.nz, p.ny, p.nx)
        self.N = p.nx * p.ny * p.nz
        h = self.lib.ref_create(C.byref(p))
        if not h:
            raise ValueError("ref_create rejected the parameters")
        self.h = h
        self.np = 0

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.ref_destroy(h)
            self.h = None

    def set_fields(self, rho=None, u=None, psi=None, phi=None):
        def prep(a, n):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
            assert a.size == n
            return a
        rho, u = prep(rho, self.N), prep(u, 3 * self.N)
        psi, phi = prep(psi, self.N), prep(phi, self.N)
        self.lib.ref_set_fields(self.h, _ptr(rho), _ptr(u), _ptr(psi), _ptr(phi))

    def add_particle(self, **kw) -> int:
        d = RefParticleDesc()
        for k in ("pos", "m_hat", "vel", "omega", "ext_force", "ext_torque"):
            v = kw.get(k, (1.0, 0.0, 0.0) if k == "m_hat" else (0.0, 0.0, 0.0))
            setattr(d, k, (C.c_double * 3)(*[float(x) for x in v]))
        d.R = float(kw["R"])
        d.rho_p = float(kw.get("rho_p", 1.0))
        d.alpha = float(kw.get("alpha", 0.0))
        d.mu_plus = float(kw.get("mu_plus", 0.0))
        d.mu_minus = float(kw.get("mu_minus", 0.0))
        if "H" in kw:
            d.H = float(kw["H"])
        else:
            th = float(kw.get("theta_c_deg", 90.0))
            d.H = wetting_h(th) * math.sqrt(self.params["kappa"] * self.params["A"])
        d.fixed = int(kw.get("fixed", 0))
        k = self.lib.ref_add_particle(self.h, C.byref(d))
        if k < 0:
            raise ValueError("ref_add_particle rejected the particle")
        self.np += 1
        return k

    def step(self, n: int = 1) -> int:
        return self.lib.ref_step(self.h, int(n))

    def fields(self):
        """Return dict rho [nz,ny,nx], u [3,nz,ny,nx], psi, phi."""
        N = self.N
        rho, u = np.empty(N), np.empty(3 * N)
        psi, phi = np.empty(N), np.empty(N)
        self.lib.ref_read_fields(self.h, _ptr(rho), _ptr(u), _ptr(psi), _ptr(phi))
        s = self.shape
        return dict(rho=rho.reshape(s), u=u.reshape((3,) + s), psi=psi.reshape(s), phi=phi.reshape(s))

    def mu(self):
        mps, mph = np.empty(self.N), np.empty(self.N)
        self.lib.ref_read_mu(self.h, _ptr(mps), _ptr(mph))
        return mps.reshape(self.shape), mph.reshape(self.shape)

    def populations(self):
        f = np.empty(19 * self.N)
        self.lib.ref_read_populations(self.h, _ptr(f))
        return f.reshape((19,) + self.shape)

    def mask(self):
        m = np.empty(self.N, dtype=np.uint8)
        self.lib.ref_read_mask(self.h, m.ctypes.data_as(C.POINTER(C.c_ubyte)))
        return m.reshape(self.shape)

    def particles(self):
        out = (RefParticleState * max(self.np, 1))()
        n = self.lib.ref_read_particles(self.h, out, max(self.np, 1))
        res = []
        for k in range(n):
            res.append({f: np.array(getattr(out[k], f)[:]) for f in
                        ("pos", "vel", "omega", "m_hat", "force", "torque")})
        return res

    def conservation(self):
        s = np.empty(3)
        self.lib.ref_conservation(self.h, _ptr(s))
        return s

    def error(self) -> int:
        return self.lib.ref_error(self.h)

    def fluid_count(self) -> int:
        return self.lib.ref_fluid_count(self.h)
