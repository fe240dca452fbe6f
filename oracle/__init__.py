"""FP64 CPU oracle for the grand-potential phase-field time step (arXiv:1506.01684).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of
the benchmark load this module; the product library never does.  The oracle is
plain C (``pf_oracle.c``) compiled with gcc and wrapped here with ctypes.  It
shares no code with the CUDA library.

Field layout everywhere in this module: numpy float64 arrays, ``phi`` with shape
``(4, nz, ny, nx)`` (phase 3 = liquid) and ``mu`` with shape ``(2, nz, ny, nx)``.

Functions without an independent pin are marked "parity unpinned" in their
docstring; every other function is checked in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pf_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libpf_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, OpenMP over z-planes)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c99", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("dx", ctypes.c_double), ("eps", ctypes.c_double), ("tau", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("gamma2", ctypes.c_double * 6), ("gamma3", ctypes.c_double * 4),
        ("A", ctypes.c_double * 4), ("Am", (ctypes.c_double * 3) * 4), ("tau_ab", ctypes.c_double * 6),
        ("cE", (ctypes.c_double * 2) * 4),
        ("kT", (ctypes.c_double * 2) * 4), ("s", ctypes.c_double * 4),
        ("D", ctypes.c_double * 4),
        ("TE", ctypes.c_double), ("T0", ctypes.c_double), ("G", ctypes.c_double),
        ("v", ctypes.c_double),
        ("seed_layers", ctypes.c_int), ("n_grains", ctypes.c_int),
        ("window_trigger_z", ctypes.c_double),
    ]


_D = ctypes.c_double
_I = ctypes.c_int
_P = ctypes.POINTER
_DP = _P(ctypes.c_double)
_IP = _P(ctypes.c_int)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            pp = _P(OrcParams)
            sig = {
                "orc_default_dt": (_D, [pp, _I]),
                "orc_kmat": (None, [pp, _I, _DP]),
                "orc_tau": (_D, [pp, _DP]),
                "orc_temperature": (_D, [pp, _D, _D]),
                "orc_psi_alpha": (_D, [pp, _I, _DP, _D]),
                "orc_c_alpha": (None, [pp, _I, _DP, _D, _DP]),
                "orc_h": (None, [_DP, _DP]),
                "orc_psi": (_D, [pp, _DP, _DP, _D]),
                "orc_dpsi": (None, [pp, _DP, _DP, _D, _DP]),
                "orc_a": (_D, [pp, _DP, _DP]),
                "orc_dadphi": (None, [pp, _DP, _DP, _DP]),
                "orc_dadgrad": (None, [pp, _DP, _DP, _DP]),
                "orc_omega": (_D, [pp, _DP]),
                "orc_domega": (None, [pp, _DP, _DP]),
                "orc_project": (None, [_DP, _DP]),
                "orc_phi_sweep": (None, [pp, _I, _I, _I, _D, _D, _DP, _DP, _DP, _DP, _DP]),
                "orc_mu_sweep": (None, [pp, _I, _I, _I, _D, _D, _DP, _DP, _DP, _DP]),
                "orc_face_flux_field": (None, [pp, _I, _I, _I, _D, _D, _DP, _DP, _DP, _DP]),
                "orc_reduce": (None, [pp, _I, _I, _I, _D, _D, _DP, _DP, _DP, _DP, _DP, _IP]),
                "orc_window_shift": (_I, [pp, _I, _I, _I, _D, _DP, _DP, _DP]),
                "orc_step": (_I, [pp, _I, _I, _I, _DP, _DP, _DP, _DP, _I]),
                "orc_splitmix64_n": (ctypes.c_uint64, [ctypes.c_uint64, _I, _P(ctypes.c_uint64)]),
                "orc_voronoi_seeds": (None, [_I, _I, _I, _I, ctypes.c_uint64, _DP]),
                "orc_init": (None, [pp, _I, _I, _I, ctypes.c_uint64, _DP, _DP, _IP]),
                "orc_num_threads": (_I, []),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


def _arr(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.size == n
    return a


def make_params(d: dict) -> OrcParams:
    """Build the oracle's parameter struct from a plain dict (see ``workloads``)."""
    p = OrcParams()
    p.dx, p.eps, p.tau, p.dt = d["dx"], d["eps"], d["tau"], d["dt"]
    for i in range(6):
        p.gamma2[i] = d["gamma2"][i]
    for i in range(4):
        p.gamma3[i] = d["gamma3"][i]
    Am = d.get("Am")
    for q in range(6):
        p.tau_ab[q] = d["tau_ab"][q] if d.get("tau_ab") is not None else 0.0
    for a in range(4):
        p.A[a] = d["A"][a]
        for c in range(3):
            p.Am[a][c] = Am[a][c] if Am is not None else 0.0
        p.s[a] = d["s"][a]
        p.D[a] = d["D"][a]
        for c in range(2):
            p.cE[a][c] = d["cE"][a][c]
            p.kT[a][c] = d["kT"][a][c]
    p.TE, p.T0, p.G, p.v = d["TE"], d["T0"], d["G"], d["v"]
    p.seed_layers, p.n_grains = int(d["seed_layers"]), int(d["n_grains"])
    p.window_trigger_z = d["window_trigger_z"]
    return p


def resolve_params(d: dict, nz: int) -> dict:
    """Return a copy of ``d`` with dt <= 0 replaced by the R12 default (0.5 x explicit limit)."""
    out = dict(d)
    if not out["dt"] > 0.0:
        out["dt"] = default_dt(d, nz)
    return out


def default_dt(d: dict, nz: int) -> float:
    """0.5 x min(tau dx^2/(12 gamma_max T_max), dx^2/(6 D_max)) with T_max over the initial window."""
    return lib().orc_default_dt(ctypes.byref(make_params(d)), nz)


# ---------------------------------------------------------------------------
# pointwise functions
# ---------------------------------------------------------------------------

def kmat(d, a):
    """K_a = dc^a/dmu = (1/2) A_a^{-1} (2x2)."""
    K = np.zeros((2, 2))
    lib().orc_kmat(ctypes.byref(make_params(d)), a, _dp(K))
    return K


def tau(d, phi):
    """Relaxation time at a cell with phase fractions phi (reading R17)."""
    return lib().orc_tau(ctypes.byref(make_params(d)), _dp(_arr(phi, 4)))


def temperature(d, z, t):
    return lib().orc_temperature(ctypes.byref(make_params(d)), z, t)


def psi_alpha(d, a, mu, T):
    m = _arr(mu, 2)
    return lib().orc_psi_alpha(ctypes.byref(make_params(d)), a, _dp(m), T)


def c_alpha(d, a, mu, T):
    m = _arr(mu, 2)
    out = np.zeros(2)
    lib().orc_c_alpha(ctypes.byref(make_params(d)), a, _dp(m), T, _dp(out))
    return out


def h(phi):
    p = _arr(phi, 4)
    out = np.zeros(4)
    lib().orc_h(_dp(p), _dp(out))
    return out


def psi(d, phi, mu, T):
    return lib().orc_psi(ctypes.byref(make_params(d)), _dp(_arr(phi, 4)), _dp(_arr(mu, 2)), T)


def dpsi(d, phi, mu, T):
    out = np.zeros(4)
    lib().orc_dpsi(ctypes.byref(make_params(d)), _dp(_arr(phi, 4)), _dp(_arr(mu, 2)), T, _dp(out))
    return out


def a_energy(d, phi, grad):
    return lib().orc_a(ctypes.byref(make_params(d)), _dp(_arr(phi, 4)), _dp(_arr(grad, 12)))


def dadphi(d, phi, grad):
    out = np.zeros(4)
    lib().orc_dadphi(ctypes.byref(make_params(d)), _dp(_arr(phi, 4)), _dp(_arr(grad, 12)), _dp(out))
    return out


def dadgrad(d, phi, grad):
    out = np.zeros((4, 3))
    lib().orc_dadgrad(ctypes.byref(make_params(d)), _dp(_arr(phi, 4)), _dp(_arr(grad, 12)), _dp(out))
    return out


def omega(d, phi):
    return lib().orc_omega(ctypes.byref(make_params(d)), _dp(_arr(phi, 4)))


def domega(d, phi):
    out = np.zeros(4)
    lib().orc_domega(ctypes.byref(make_params(d)), _dp(_arr(phi, 4)), _dp(out))
    return out


def project(u):
    out = np.zeros(4)
    lib().orc_project(_dp(_arr(u, 4)), _dp(out))
    return out


# ---------------------------------------------------------------------------
# field operations
# ---------------------------------------------------------------------------

def phi_sweep(d, phi, mu, t=0.0, off=0.0, want_star=False, want_rhs=False):
    """One phi-sweep (Eq. 1, Eq. 2, projection).  Returns phi_new (and phi_star, rhs on request)."""
    _, nz, ny, nx = phi.shape
    phi = _arr(phi)
    mu = _arr(mu)
    out = np.zeros_like(phi)
    star = np.zeros_like(phi) if want_star else None
    rhs = np.zeros_like(phi) if want_rhs else None
    lib().orc_phi_sweep(ctypes.byref(make_params(d)), nx, ny, nz, t, off, _dp(phi), _dp(mu), _dp(out),
                        _dp(star) if star is not None else None, _dp(rhs) if rhs is not None else None)
    res = [out]
    if want_star:
        res.append(star)
    if want_rhs:
        res.append(rhs)
    return res[0] if len(res) == 1 else tuple(res)


def mu_sweep(d, phi_old, phi_new, mu, t=0.0, off=0.0):
    """One mu-sweep (Eq. 3 with Eq. 4)."""
    _, nz, ny, nx = phi_old.shape
    out = np.zeros_like(_arr(mu))
    lib().orc_mu_sweep(ctypes.byref(make_params(d)), nx, ny, nz, t, off, _dp(_arr(phi_old)),
                       _dp(_arr(phi_new)), _dp(_arr(mu)), _dp(out))
    return out


def face_flux_field(d, phi_old, phi_new, mu, t=0.0, off=0.0):
    """Face values v = M grad mu - J_at; shape (2, 3, nz, ny, nx): component, face direction, cell."""
    _, nz, ny, nx = phi_old.shape
    out = np.zeros((2, 3, nz, ny, nx))
    lib().orc_face_flux_field(ctypes.byref(make_params(d)), nx, ny, nz, t, off, _dp(_arr(phi_old)),
                              _dp(_arr(phi_new)), _dp(_arr(mu)), _dp(out))
    return out


def reduce(d, phi, mu, t=0.0, off=0.0):
    """(fractions[4], solute[2], h_int, nonfinite)"""
    _, nz, ny, nx = phi.shape
    fr = np.zeros(4)
    so = np.zeros(2)
    hh = ctypes.c_double()
    bad = ctypes.c_int()
    lib().orc_reduce(ctypes.byref(make_params(d)), nx, ny, nz, t, off, _dp(_arr(phi)), _dp(_arr(mu)),
                     _dp(fr), _dp(so), ctypes.byref(hh), ctypes.byref(bad))
    return fr, so, hh.value, bool(bad.value)


def window_shift(d, phi, mu, h_int, off):
    """The moving window (Section 3.3) on (phi, mu) in place: returns (planes shifted, new offset)."""
    _, nz, ny, nx = phi.shape
    assert phi.dtype == np.float64 and phi.flags["C_CONTIGUOUS"] and mu.dtype == np.float64 and mu.flags["C_CONTIGUOUS"]
    o = ctypes.c_double(off)
    s = lib().orc_window_shift(ctypes.byref(make_params(d)), nx, ny, nz, h_int, ctypes.byref(o), _dp(phi), _dp(mu))
    return s, o.value


class State:
    """A simulation state held by the oracle: fields, time and window offset."""

    def __init__(self, params: dict, nx: int, ny: int, nz: int):
        self.params = resolve_params(params, nz)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.phi = np.zeros((4, nz, ny, nx))
        self.phi[3] = 1.0
        self.mu = np.zeros((2, nz, ny, nx))
        self.t = 0.0
        self.off = 0.0
        self.shifts = 0

    def init(self, seed: int):
        grain = np.zeros((self.nz, self.ny, self.nx), dtype=np.int32)
        lib().orc_init(ctypes.byref(make_params(self.params)), self.nx, self.ny, self.nz,
                       ctypes.c_uint64(seed), _dp(self.phi), _dp(self.mu),
                       grain.ctypes.data_as(_IP))
        self.t = 0.0
        self.off = 0.0
        self.grain = grain
        return self

    def step(self, n: int = 1):
        t = ctypes.c_double(self.t)
        off = ctypes.c_double(self.off)
        s = lib().orc_step(ctypes.byref(make_params(self.params)), self.nx, self.ny, self.nz,
                           ctypes.byref(t), ctypes.byref(off), _dp(self.phi), _dp(self.mu), n)
        self.t, self.off = t.value, off.value
        self.shifts += s
        return self

    def reduce(self):
        return reduce(self.params, self.phi, self.mu, self.t, self.off)


def num_threads() -> int:
    """OpenMP threads the oracle's sweeps run on."""
    return int(lib().orc_num_threads())


def splitmix64(seed: int, n: int):
    out = (ctypes.c_uint64 * n)()
    lib().orc_splitmix64_n(ctypes.c_uint64(seed), n, out)
    return [int(x) for x in out]


def voronoi_seeds(nx, ny, H, n_grains, seed):
    out = np.zeros((max(n_grains, 1), 4))
    lib().orc_voronoi_seeds(nx, ny, H, n_grains, ctypes.c_uint64(seed), _dp(out))
    return out[:n_grains]
