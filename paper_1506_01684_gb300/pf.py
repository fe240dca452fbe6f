"""Thin ctypes binding of the C ABI in ``include/pf.h`` (argument marshalling only).

Every computation runs in the CUDA library ``_lib/libpf_gb300.so``; this module never
computes any part of the time step.  If the library cannot be loaded the import of the
functions fails loudly: there is no CPU fallback.

Python names follow the C names (``pf_create``, ``pf_init``, ``pf_step``, ...).  Handles
are opaque ``ctypes.c_void_p`` values.  Non-OK statuses raise :class:`PfError` (except
``pf_poll``'s ``PF_E_PENDING``, which is returned).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

PF_OK = 0
PF_E_INVAL = -1
PF_E_NOMEM = -2
PF_E_CUDA = -3
PF_E_UNSTABLE = -4
PF_E_TIMEOUT = -5
PF_E_CANCELLED = -6
PF_E_PENDING = 1

PF_FP64 = 0
PF_FP32 = 1
PF_FP32_COMP = 2
PF_PARAMS_VERSION = 2

PRECISIONS = {"fp64": PF_FP64, "fp32": PF_FP32, "fp32c": PF_FP32_COMP}


class PfError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {pf_strerror(status)} ({status})" if what else pf_strerror(status))


class pf_params(ctypes.Structure):
    _fields_ = [
        ("version", ctypes.c_int), ("precision", ctypes.c_int),
        ("dx", ctypes.c_double), ("eps", ctypes.c_double), ("tau", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("gamma2", ctypes.c_double * 6), ("gamma3", ctypes.c_double * 4),
        ("A", ctypes.c_double * 4), ("cE", (ctypes.c_double * 2) * 4),
        ("kT", (ctypes.c_double * 2) * 4), ("s", ctypes.c_double * 4), ("D", ctypes.c_double * 4),
        ("TE", ctypes.c_double), ("T0", ctypes.c_double), ("G", ctypes.c_double), ("v", ctypes.c_double),
        ("seed_layers", ctypes.c_int), ("n_grains", ctypes.c_int),
        ("window_trigger_z", ctypes.c_double),
        ("Am", (ctypes.c_double * 3) * 4), ("tau_ab", ctypes.c_double * 6),
    ]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes); every symbol declared in include/pf.h appears here
_D = ctypes.c_double
_DP = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p
_I = ctypes.c_int
SIGNATURES = {
    "pf_strerror": (ctypes.c_char_p, [_I]),
    "pf_default_params": (_I, [ctypes.POINTER(pf_params)]),
    "pf_set_allocator": (_I, [_ALLOC_FN, _FREE_FN, _VP]),
    "pf_create": (_I, [_I, _I, _I, ctypes.POINTER(pf_params), _VP, ctypes.POINTER(_VP)]),
    "pf_destroy": (_I, [_VP]),
    "pf_get_params": (_I, [_VP, ctypes.POINTER(pf_params)]),
    "pf_init": (_I, [_VP, ctypes.c_uint64]),
    "pf_step": (_I, [_VP, _I]),
    "pf_sync": (_I, [_VP]),
    "pf_read_fields": (_I, [_VP, _DP, _DP, ctypes.c_size_t]),
    "pf_write_fields": (_I, [_VP, _DP, _DP]),
    "pf_read_fields_f32": (_I, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), ctypes.c_size_t]),
    "pf_write_fields_f32": (_I, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
    "pf_phase_fractions": (_I, [_VP, _DP]),
    "pf_stats": (_I, [_VP, _DP, _DP, _DP, _DP]),
    "pf_window_shifts": (_I, [_VP, ctypes.POINTER(_I)]),
    "pf_step_bytes": (_I, [_VP, _DP]),
    "pf_test_withhold_copies": (_I, [_VP, _I]),
    "pf_checkpoint_write": (_I, [_VP, ctypes.c_char_p]),
    "pf_checkpoint_read": (_I, [_VP, ctypes.c_char_p]),
    "pf_checkpoint_write_f32": (_I, [_VP, ctypes.c_char_p]),
    "pf_interface_mesh": (_I, [_VP, _I, _D, ctypes.POINTER(ctypes.c_float), ctypes.c_size_t,
                               ctypes.POINTER(ctypes.c_size_t)]),
    "pf_profile": (_I, [_VP, _I]),
    "pf_set_variant": (_I, [_VP, _I]),
    "pf_profile_read": (_I, [_VP, _DP, ctypes.POINTER(_I)]),
    "pf_step_noalloc": (_I, [_I, _I, _I, ctypes.POINTER(pf_params), _D, _D, _VP, _VP, _VP, _VP, _DP, _VP]),
    "pf_batch_create": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(pf_params),
                             _VP, ctypes.POINTER(_VP)]),
    "pf_batch_destroy": (_I, [_VP]),
    "pf_batch_domain": (_I, [_VP, _I, ctypes.POINTER(_VP)]),
    "pf_batch_init": (_I, [_VP, ctypes.POINTER(ctypes.c_uint64)]),
    "pf_batch_step": (_I, [_VP, _I]),
    "pf_batch_sync": (_I, [_VP]),
    "pf_batch_set_zchunk": (_I, [_VP, _I]),
    "pf_batch_autotune": (_I, [_VP, _I, ctypes.POINTER(_I), _DP]),
    "pf_batch_step_bytes": (_I, [_VP, _DP]),
    "pf_batch_config": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "pf_batch_set_config": (_I, [_VP, _I, _I, _I, _I]),
    "pf_server_create": (_I, [ctypes.c_size_t, _I, _I, ctypes.POINTER(_VP)]),
    "pf_server_destroy": (_I, [_VP]),
    "pf_submit": (_I, [_VP, _I, _I, _I, ctypes.POINTER(pf_params), ctypes.c_uint64, _I,
                       ctypes.POINTER(ctypes.c_uint64)]),
    "pf_poll": (_I, [_VP, ctypes.c_uint64, _DP, ctypes.POINTER(ctypes.c_float), _DP]),
    "pf_cancel": (_I, [_VP, ctypes.c_uint64]),
    "pf_server_stats": (_I, [_VP, _DP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_size_t)]),
    "pf_split_create": (_I, [_I, _I, _I, ctypes.POINTER(pf_params), _I, ctypes.POINTER(_VP)]),
    "pf_split_destroy": (_I, [_VP]),
    "pf_split_init": (_I, [_VP, ctypes.c_uint64]),
    "pf_split_step": (_I, [_VP, _I]),
    "pf_split_sync": (_I, [_VP]),
    "pf_split_read_fields": (_I, [_VP, _DP, _DP, ctypes.c_size_t]),
    "pf_split_stats": (_I, [_VP, _DP, _DP, _DP, ctypes.POINTER(_I)]),
}

PF_K_PHI, PF_K_MU, PF_K_FINALIZE, PF_K_POST, PF_K_FUSED, PF_K_LEAN, PF_K_PLAN, PF_K_GENERAL = 0, 1, 2, 3, 4, 5, 6, 7
PF_K_MESH_COUNT, PF_K_MESH_SCAN, PF_K_MESH_EMIT, PF_K_COUNT = 8, 9, 10, 11
KERNEL_NAMES = {PF_K_PHI: "phi_sweep", PF_K_MU: "mu_sweep", PF_K_FINALIZE: "finalize", PF_K_POST: "post",
                PF_K_FUSED: "fused_step", PF_K_LEAN: "lean_step", PF_K_PLAN: "plan", PF_K_GENERAL: "general_sweeps",
                PF_K_MESH_COUNT: "mesh_count", PF_K_MESH_SCAN: "mesh_scan", PF_K_MESH_EMIT: "mesh_emit"}
PF_VARIANT_AUTO, PF_VARIANT_UNFUSED, PF_VARIANT_FUSED = 0, 1, 2
VARIANTS = {"auto": PF_VARIANT_AUTO, "unfused": PF_VARIANT_UNFUSED, "fused": PF_VARIANT_FUSED}


def library_path() -> str:
    return _build.LIB


def lib(auto_build: bool = True):
    """Load the CUDA library (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if auto_build and _build.is_stale():
                _build.build()
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built: {path} (run paper_1506_01684_gb300.build.build())")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(st: int, what: str):
    if st != PF_OK:
        raise PfError(st, what)
    return st


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


# ---------------------------------------------------------------------------------------
# C ABI, one Python function per C entry point
# ---------------------------------------------------------------------------------------

def pf_strerror(st: int) -> str:
    try:
        return lib(auto_build=False).pf_strerror(st).decode()
    except Exception:  # library not loadable: still give a readable message
        return f"status {st}"


def pf_default_params(precision: int = PF_FP64) -> pf_params:
    p = pf_params()
    _check(lib().pf_default_params(ctypes.byref(p)), "pf_default_params")
    p.precision = precision
    return p


def params_from_dict(d: dict, precision: int = PF_FP64) -> pf_params:
    """Fill a pf_params from the plain parameter dict used by ``workloads``."""
    p = pf_params()
    p.version = PF_PARAMS_VERSION
    p.precision = precision
    p.dx, p.eps, p.tau, p.dt = d["dx"], d["eps"], d["tau"], d["dt"]
    for i in range(6):
        p.gamma2[i] = d["gamma2"][i]
    for i in range(4):
        p.gamma3[i] = d["gamma3"][i]
    for a in range(4):
        p.A[a], p.s[a], p.D[a] = d["A"][a], d["s"][a], d["D"][a]
        for c in range(2):
            p.cE[a][c] = d["cE"][a][c]
            p.kT[a][c] = d["kT"][a][c]
    p.TE, p.T0, p.G, p.v = d["TE"], d["T0"], d["G"], d["v"]
    p.seed_layers, p.n_grains = int(d["seed_layers"]), int(d["n_grains"])
    p.window_trigger_z = d["window_trigger_z"]
    Am, tau_ab = d.get("Am"), d.get("tau_ab")
    for a in range(4):
        for c in range(3):
            p.Am[a][c] = Am[a][c] if Am is not None else 0.0
    for q in range(6):
        p.tau_ab[q] = tau_ab[q] if tau_ab is not None else 0.0
    return p


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def pf_set_allocator(alloc, free_fn, ctx=None):
    """Install device allocator hooks (ctypes callbacks of the pf_alloc_fn / pf_free_fn types);
    None, None restores cudaMalloc/cudaFree.  The caller keeps the callbacks alive."""
    return _check(lib().pf_set_allocator(alloc or _ALLOC_FN(), free_fn or _FREE_FN(), ctx), "pf_set_allocator")


def pf_create(nx: int, ny: int, nz: int, params: pf_params, stream=None):
    h = _VP()
    _check(lib().pf_create(nx, ny, nz, ctypes.byref(params), _stream_handle(stream), ctypes.byref(h)),
           "pf_create")
    return h


def pf_destroy(sim):
    return _check(lib().pf_destroy(sim), "pf_destroy")


def pf_get_params(sim) -> pf_params:
    p = pf_params()
    _check(lib().pf_get_params(sim, ctypes.byref(p)), "pf_get_params")
    return p


def pf_init(sim, seed: int):
    return _check(lib().pf_init(sim, ctypes.c_uint64(seed)), "pf_init")


def pf_step(sim, nsteps: int):
    return _check(lib().pf_step(sim, nsteps), "pf_step")


def pf_sync(sim):
    return _check(lib().pf_sync(sim), "pf_sync")


def pf_read_fields(sim, phi: np.ndarray | None, mu: np.ndarray | None):
    n = None
    for a in (phi, mu):
        if a is not None:
            n = a.shape[-1] * a.shape[-2] * a.shape[-3]
    return _check(lib().pf_read_fields(sim, _dp(phi) if phi is not None else None,
                                       _dp(mu) if mu is not None else None, n or 0), "pf_read_fields")


def pf_write_fields(sim, phi: np.ndarray, mu: np.ndarray):
    return _check(lib().pf_write_fields(sim, _dp(phi), _dp(mu)), "pf_write_fields")


def _fp(a: np.ndarray):
    assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def pf_read_fields_f32(sim, phi: np.ndarray | None, mu: np.ndarray | None):
    n = None
    for a in (phi, mu):
        if a is not None:
            n = a.shape[-1] * a.shape[-2] * a.shape[-3]
    return _check(lib().pf_read_fields_f32(sim, _fp(phi) if phi is not None else None,
                                           _fp(mu) if mu is not None else None, n or 0), "pf_read_fields_f32")


def pf_write_fields_f32(sim, phi: np.ndarray, mu: np.ndarray):
    return _check(lib().pf_write_fields_f32(sim, _fp(phi), _fp(mu)), "pf_write_fields_f32")


def pf_phase_fractions(sim) -> np.ndarray:
    out = np.zeros(4)
    _check(lib().pf_phase_fractions(sim, _dp(out)), "pf_phase_fractions")
    return out


def pf_stats(sim):
    t, off, h = _D(), _D(), _D()
    sol = np.zeros(2)
    _check(lib().pf_stats(sim, ctypes.byref(t), ctypes.byref(off), _dp(sol), ctypes.byref(h)), "pf_stats")
    return {"t": t.value, "window_offset": off.value, "solute": sol, "h_int": h.value}


def pf_window_shifts(sim) -> int:
    n = _I()
    _check(lib().pf_window_shifts(sim, ctypes.byref(n)), "pf_window_shifts")
    return n.value


def pf_test_withhold_copies(sim, on: bool):
    _check(lib().pf_test_withhold_copies(sim, 1 if on else 0), "pf_test_withhold_copies")


def pf_checkpoint_write(sim, path: str):
    _check(lib().pf_checkpoint_write(sim, os.fsencode(path)), "pf_checkpoint_write")


def pf_checkpoint_write_f32(sim, path: str):
    _check(lib().pf_checkpoint_write_f32(sim, os.fsencode(path)), "pf_checkpoint_write_f32")


def pf_checkpoint_read(sim, path: str):
    _check(lib().pf_checkpoint_read(sim, os.fsencode(path)), "pf_checkpoint_read")


def pf_interface_mesh(sim, phase: int, iso: float = 0.5) -> np.ndarray:
    """Triangles (T, 3, 3) float32 of the surface phi_phase = iso (count, then fetch)."""
    n = ctypes.c_size_t()
    _check(lib().pf_interface_mesh(sim, int(phase), float(iso), None, 0, ctypes.byref(n)), "pf_interface_mesh")
    out = np.empty((n.value, 3, 3), dtype=np.float32)
    if n.value:
        m = ctypes.c_size_t()
        _check(lib().pf_interface_mesh(sim, int(phase), float(iso),
                                       out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n.value,
                                       ctypes.byref(m)), "pf_interface_mesh")
        assert m.value == n.value
    return out


def pf_step_bytes(sim) -> dict:
    """Algorithmic bytes of the last step per kernel name (kernels that ran only)."""
    b = np.zeros(PF_K_COUNT)
    _check(lib().pf_step_bytes(sim, _dp(b)), "pf_step_bytes")
    return {KERNEL_NAMES[c]: float(b[c]) for c in KERNEL_NAMES if b[c] > 0}


def pf_set_variant(sim, variant):
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    return _check(lib().pf_set_variant(sim, v), "pf_set_variant")


def pf_profile(sim, enable: bool = True):
    return _check(lib().pf_profile(sim, 1 if enable else 0), "pf_profile")


def pf_profile_read(sim):
    """{kernel name: (device ms, launches)} accumulated since the last read."""
    ms = np.zeros(PF_K_COUNT)
    n = (_I * PF_K_COUNT)()
    _check(lib().pf_profile_read(sim, _dp(ms), n), "pf_profile_read")
    return {KERNEL_NAMES.get(c, f"k{c}"): (float(ms[c]), int(n[c])) for c in range(PF_K_COUNT) if n[c] > 0}


def pf_step_noalloc(nx: int, ny: int, nz: int, params: pf_params, t: float, window_offset: float,
                    phi_src: int, mu_src: int, phi_dst: int, mu_dst: int, want_h_int: bool = True,
                    stream=None):
    """One step on caller-owned device fields (device pointers as ints), allocating nothing.
    Returns the interface height of the new state when want_h_int (this waits for the stream)."""
    h = _D()
    _check(lib().pf_step_noalloc(nx, ny, nz, ctypes.byref(params), t, window_offset, phi_src, mu_src,
                                 phi_dst, mu_dst, ctypes.byref(h) if want_h_int else None,
                                 _stream_handle(stream)), "pf_step_noalloc")
    return h.value if want_h_int else None


def pf_batch_create(shapes, params_list, stream=None):
    n = len(shapes)
    nx = (_I * n)(*[s[0] for s in shapes])
    ny = (_I * n)(*[s[1] for s in shapes])
    nz = (_I * n)(*[s[2] for s in shapes])
    ps = (pf_params * n)(*params_list)
    h = _VP()
    _check(lib().pf_batch_create(n, nx, ny, nz, ps, _stream_handle(stream), ctypes.byref(h)), "pf_batch_create")
    return h


def pf_batch_destroy(b):
    return _check(lib().pf_batch_destroy(b), "pf_batch_destroy")


def pf_batch_domain(b, d):
    h = _VP()
    _check(lib().pf_batch_domain(b, d, ctypes.byref(h)), "pf_batch_domain")
    return h


def pf_batch_init(b, seeds):
    arr = (ctypes.c_uint64 * len(seeds))(*[int(x) for x in seeds])
    return _check(lib().pf_batch_init(b, arr), "pf_batch_init")


def pf_batch_step(b, nsteps):
    return _check(lib().pf_batch_step(b, nsteps), "pf_batch_step")


def pf_batch_sync(b):
    return _check(lib().pf_batch_sync(b), "pf_batch_sync")


def pf_batch_set_zchunk(b, zchunk):
    return _check(lib().pf_batch_set_zchunk(b, zchunk), "pf_batch_set_zchunk")


def pf_batch_autotune(b, trial_steps=10):
    best = _I()
    ms = _D()
    _check(lib().pf_batch_autotune(b, trial_steps, ctypes.byref(best), ctypes.byref(ms)), "pf_batch_autotune")
    return best.value, ms.value


def pf_batch_config(b):
    z, g, l, r = _I(), _I(), _I(), _I()
    _check(lib().pf_batch_config(b, ctypes.byref(z), ctypes.byref(g), ctypes.byref(l), ctypes.byref(r)),
           "pf_batch_config")
    return {"zchunk": z.value, "general_ctas_per_sm": g.value, "lean_split": l.value, "lean_tile_rows": r.value}


def pf_batch_set_config(b, zchunk=0, general_ctas_per_sm=2, lean_split=1, lean_tile_rows=8):
    _check(lib().pf_batch_set_config(b, zchunk, general_ctas_per_sm, lean_split, lean_tile_rows),
           "pf_batch_set_config")


def pf_batch_step_bytes(b):
    out = np.zeros(2)
    _check(lib().pf_batch_step_bytes(b, _dp(out)), "pf_batch_step_bytes")
    return {"general_and_fused": float(out[0]), "lean_step": float(out[1])}


def pf_server_create(hbm_budget_bytes: int = 0, max_active: int = 0, chunk: int = 0):
    h = _VP()
    _check(lib().pf_server_create(hbm_budget_bytes, max_active, chunk, ctypes.byref(h)), "pf_server_create")
    return h


def pf_server_destroy(srv):
    return _check(lib().pf_server_destroy(srv), "pf_server_destroy")


def pf_submit(srv, nx, ny, nz, params: pf_params, seed: int, nsteps: int) -> int:
    t = ctypes.c_uint64()
    _check(lib().pf_submit(srv, nx, ny, nz, ctypes.byref(params), ctypes.c_uint64(seed), nsteps, ctypes.byref(t)),
           "pf_submit")
    return t.value


def pf_poll(srv, ticket: int, nx: int = 0, ny: int = 0):
    """None while pending; else (fractions, slab (4, ny, nx) float32 or None, latency_s).  Raises on failure."""
    fr = np.zeros(4)
    slab = np.zeros((4, ny, nx), dtype=np.float32) if nx and ny else None
    lat = _D()
    st = lib().pf_poll(srv, ctypes.c_uint64(ticket), _dp(fr),
                       slab.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if slab is not None else None,
                       ctypes.byref(lat))
    if st == PF_E_PENDING:
        return None
    _check(st, "pf_poll")
    return fr, slab, lat.value


def pf_cancel(srv, ticket: int):
    return _check(lib().pf_cancel(srv, ctypes.c_uint64(ticket)), "pf_cancel")


def pf_server_stats(srv):
    m = _D()
    r, q = _I(), _I()
    u = ctypes.c_size_t()
    _check(lib().pf_server_stats(srv, ctypes.byref(m), ctypes.byref(r), ctypes.byref(q), ctypes.byref(u)),
           "pf_server_stats")
    return {"mlups": m.value, "running": r.value, "queued": q.value, "used_bytes": u.value}


def pf_split_create(nx, ny, nz, params: pf_params, nslabs: int):
    h = _VP()
    _check(lib().pf_split_create(nx, ny, nz, ctypes.byref(params), nslabs, ctypes.byref(h)), "pf_split_create")
    return h.value


def pf_split_destroy(d):
    return _check(lib().pf_split_destroy(d), "pf_split_destroy")


def pf_split_init(d, seed: int):
    return _check(lib().pf_split_init(d, seed), "pf_split_init")


def pf_split_step(d, nsteps: int):
    return _check(lib().pf_split_step(d, nsteps), "pf_split_step")


def pf_split_sync(d):
    return _check(lib().pf_split_sync(d), "pf_split_sync")


def pf_split_read_fields(d, phi: np.ndarray | None, mu: np.ndarray | None):
    n = None
    for a in (phi, mu):
        if a is not None:
            n = a.shape[-1] * a.shape[-2] * a.shape[-3]
    return _check(lib().pf_split_read_fields(d, _dp(phi) if phi is not None else None,
                                             _dp(mu) if mu is not None else None, n or 0), "pf_split_read_fields")


def pf_split_stats(d):
    t, off, h, n = _D(), _D(), _D(), _I()
    _check(lib().pf_split_stats(d, ctypes.byref(t), ctypes.byref(off), ctypes.byref(h), ctypes.byref(n)),
           "pf_split_stats")
    return {"t": t.value, "window_offset": off.value, "h_int": h.value, "shifts": n.value}


class Split:
    """Owns one pf_split: one domain cut into y-slabs with ghost rows, stepped as separate blocks."""

    def __init__(self, nx, ny, nz, params: dict | pf_params, nslabs, precision="fp64"):
        prec = PRECISIONS[precision] if isinstance(precision, str) else precision
        p = params if isinstance(params, pf_params) else params_from_dict(params, prec)
        p.precision = prec
        self.nx, self.ny, self.nz = nx, ny, nz
        self.h = pf_split_create(nx, ny, nz, p, nslabs)

    def close(self):
        if self.h:
            pf_split_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, seed: int):
        pf_split_init(self.h, seed)
        return self

    def step(self, n: int = 1):
        pf_split_step(self.h, n)
        return self

    def sync(self):
        pf_split_sync(self.h)
        return self

    def fields(self):
        phi = np.empty((4, self.nz, self.ny, self.nx))
        mu = np.empty((2, self.nz, self.ny, self.nx))
        pf_split_read_fields(self.h, phi, mu)
        return phi, mu

    def stats(self):
        return pf_split_stats(self.h)


class Batch:
    """Owns one pf_batch: domains of uneven size stepped by one persistent launch per step."""

    def __init__(self, shapes, params_list, precision="fp32", stream=None):
        prec = PRECISIONS[precision] if isinstance(precision, str) else precision
        ps = []
        for p in params_list:
            q = p if isinstance(p, pf_params) else params_from_dict(p, prec)
            q.precision = prec
            ps.append(q)
        self.shapes = [tuple(s) for s in shapes]
        self.h = pf_batch_create(self.shapes, ps, stream)

    def close(self):
        if self.h:
            pf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def domain(self, d):
        return pf_batch_domain(self.h, d)

    def init(self, seeds):
        pf_batch_init(self.h, seeds)
        return self

    def step(self, n=1):
        pf_batch_step(self.h, n)
        return self

    def sync(self):
        pf_batch_sync(self.h)
        return self

    def fields(self, d):
        nx, ny, nz = self.shapes[d]
        phi = np.empty((4, nz, ny, nx))
        mu = np.empty((2, nz, ny, nx))
        pf_read_fields(self.domain(d), phi, mu)
        return phi, mu

    def stats(self, d):
        return pf_stats(self.domain(d))

    def shifts(self, d):
        return pf_window_shifts(self.domain(d))


# ---------------------------------------------------------------------------------------
# device memory through PyTorch's caching allocator (optional plumbing)
# ---------------------------------------------------------------------------------------
_hooks = None


def use_torch_allocator(enable: bool = True):
    """Route the library's device allocations through torch.cuda's caching allocator."""
    global _hooks
    if not enable:
        _check(lib().pf_set_allocator(_ALLOC_FN(), _FREE_FN(), None), "pf_set_allocator")
        _hooks = None
        return
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=stream or 0)
        except Exception:
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    _hooks = (_ALLOC_FN(_alloc), _FREE_FN(_free))
    _check(lib().pf_set_allocator(_hooks[0], _hooks[1], None), "pf_set_allocator")


# ---------------------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------------------
class Simulation:
    """Owns one pf_sim handle; numpy in/out in the host layout (component, z, y, x)."""

    def __init__(self, nx, ny, nz, params: dict | pf_params, precision="fp64", stream=None, variant="auto"):
        prec = PRECISIONS[precision] if isinstance(precision, str) else precision
        p = params if isinstance(params, pf_params) else params_from_dict(params, prec)
        p.precision = prec
        self.nx, self.ny, self.nz = nx, ny, nz
        self.h = pf_create(nx, ny, nz, p, stream)
        pf_set_variant(self.h, variant)

    def close(self):
        if self.h:
            pf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def params(self) -> pf_params:
        return pf_get_params(self.h)

    def init(self, seed: int):
        pf_init(self.h, seed)
        return self

    def step(self, n: int = 1):
        pf_step(self.h, n)
        return self

    def sync(self):
        pf_sync(self.h)
        return self

    def fields(self):
        phi = np.empty((4, self.nz, self.ny, self.nx))
        mu = np.empty((2, self.nz, self.ny, self.nx))
        pf_read_fields(self.h, phi, mu)
        return phi, mu

    def set_fields(self, phi, mu):
        pf_write_fields(self.h, np.ascontiguousarray(phi, dtype=np.float64),
                        np.ascontiguousarray(mu, dtype=np.float64))
        return self

    def fields_f32(self):
        phi = np.empty((4, self.nz, self.ny, self.nx), dtype=np.float32)
        mu = np.empty((2, self.nz, self.ny, self.nx), dtype=np.float32)
        pf_read_fields_f32(self.h, phi, mu)
        return phi, mu

    def set_fields_f32(self, phi, mu):
        pf_write_fields_f32(self.h, np.ascontiguousarray(phi, dtype=np.float32),
                            np.ascontiguousarray(mu, dtype=np.float32))
        return self

    def fractions(self):
        return pf_phase_fractions(self.h)

    def stats(self):
        return pf_stats(self.h)

    def shifts(self):
        return pf_window_shifts(self.h)

    def step_bytes(self):
        return pf_step_bytes(self.h)

    def interface_mesh(self, phase, iso=0.5):
        return pf_interface_mesh(self.h, phase, iso)

    def checkpoint(self, path, single=False):
        """single: the single-precision checkpoint (values rounded once to FP32)."""
        (pf_checkpoint_write_f32 if single else pf_checkpoint_write)(self.h, path)
        return self

    def restore(self, path):
        pf_checkpoint_read(self.h, path)
        return self
