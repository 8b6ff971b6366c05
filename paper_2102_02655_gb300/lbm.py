"""Python binding of the C ABI in include/lbm.h (ctypes).

Argument marshalling only: every step of the lattice Boltzmann update runs in
the library's CUDA kernels. PyTorch provides the device memory (through the
allocator callback) and the CUDA stream. The functions keep the C names
(lbm_create, lbm_set_geometry, lbm_set_ink_rheology, lbm_set_fields,
lbm_step, lbm_fields, lbm_sync, lbm_destroy, lbm_last_error); ``Lattice``
wraps one handle.

Importing this module never falls back to any other implementation: if the
shared library is missing or fails to load, ``lib()`` raises.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcglbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ESTATE = range(7)
STATUS_NAMES = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA", 4: "LBM_EUNSTABLE",
                5: "LBM_ETIMEOUT", 6: "LBM_ESTATE"}
LBM_D2Q9, LBM_D3Q19 = 0, 1
LBM_F64, LBM_F32, LBM_F16DEV, LBM_BF16DEV = 0, 1, 2, 3
LBM_PATH_AUTO, LBM_PATH_PLAIN, LBM_PATH_FUSED = 0, 1, 2
LBM_Z_PERIODIC, LBM_Z_WALLS = 0, 1
LBM_TOP_OPEN, LBM_TOP_WALL = 0, 1
LBM_NEWTONIAN, LBM_CROSS, LBM_POWER_LAW = 0, 1, 2
LBM_FIELD_RHO_INK, LBM_FIELD_RHO_AMB, LBM_FIELD_U = 1, 2, 4
LBM_FIELD_NU, LBM_FIELD_P, LBM_FIELD_PHI, LBM_FIELD_SOLID = 8, 16, 32, 64
FIELD_ORDER = ("rho_ink", "rho_amb", "ux", "uy", "uz", "nu", "p", "rhoN", "solid")
ALL_FIELDS = 0x7F

EXPORTS = ("lbm_create", "lbm_set_geometry", "lbm_set_ink_rheology", "lbm_set_fields", "lbm_step",
           "lbm_fields", "lbm_sync", "lbm_destroy", "lbm_last_error", "lbm_kernel_launches",
           "lbm_profile", "lbm_timings", "lbm_step_noalloc",
           "lbm_batch_create", "lbm_batch_reset", "lbm_batch_step", "lbm_batch_sync", "lbm_batch_set_plan", "lbm_batch_autotune",
           "lbm_batch_info", "lbm_batch_destroy", "lbm_batch_last_error", "lbm_batch_plan",
           "lbm_lattice_bytes", "lbm_server_create", "lbm_server_submit", "lbm_server_poll", "lbm_server_finished",
           "lbm_server_result", "lbm_server_stats", "lbm_server_destroy", "lbm_server_last_error")
LBM_TUNE_MAX = 40

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class lbm_config(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("velset", C.c_int),
                ("storage", C.c_int), ("path", C.c_int),
                ("tau_ambient", C.c_double), ("rho0_ink", C.c_double), ("rho0_amb", C.c_double),
                ("alpha_ink", C.c_double), ("alpha_amb", C.c_double), ("A", C.c_double),
                ("beta", C.c_double), ("zeta_ink", C.c_double), ("zeta_amb", C.c_double),
                ("drag_gamma", C.c_double), ("drag_height", C.c_double),
                ("body_force", C.c_double * 3), ("device", C.c_int), ("cuda_stream", C.c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p)]


class lbm_geometry(C.Structure):
    _fields_ = [("z_mode", C.c_int), ("top_mode", C.c_int), ("nozzle", C.c_int),
                ("head_pos", C.c_double * 2), ("head_vel", C.c_double * 2),
                ("r_inner", C.c_double), ("wall_thickness", C.c_double), ("gap", C.c_int),
                ("u_ink", C.c_double), ("top_vel", C.c_double * 3), ("rho_top_amb", C.c_double)]


class lbm_rheology(C.Structure):
    _fields_ = [("law", C.c_int), ("nu0", C.c_double), ("nu_inf", C.c_double),
                ("lambda_", C.c_double), ("n", C.c_double), ("K", C.c_double),
                ("tau_min", C.c_double), ("tau_max", C.c_double), ("tol", C.c_double),
                ("max_iter", C.c_int)]


class lbm_diag(C.Structure):
    _fields_ = [("mass", C.c_double * 2), ("momentum", C.c_double * 3), ("bc_flux", C.c_double * 2),
                ("created", C.c_double * 2), ("destroyed", C.c_double * 2), ("step", C.c_longlong),
                ("unstable", C.c_int)]


class lbm_timing(C.Structure):
    _fields_ = [("bulk_ms", C.c_double), ("plain_ms", C.c_double), ("bulk_launches", C.c_longlong),
                ("plain_groups", C.c_longlong), ("bulk_sites", C.c_longlong), ("plain_sites", C.c_longlong)]


class lbm_batch_tuning(C.Structure):
    _fields_ = [("variant", C.c_int), ("zchunk", C.c_int), ("ctas_per_sm", C.c_int), ("ms_per_step", C.c_double),
                ("n_tried", C.c_int), ("tried_variant", C.c_int * LBM_TUNE_MAX),
                ("tried_zchunk", C.c_int * LBM_TUNE_MAX), ("tried_ctas", C.c_int * LBM_TUNE_MAX),
                ("tried_ms", C.c_double * LBM_TUNE_MAX)]


class lbm_batch_plan_info(C.Structure):
    _fields_ = [("n_lattices", C.c_int), ("variant", C.c_int), ("tile_h", C.c_int), ("n_items", C.c_int),
                ("grid", C.c_int), ("steps_per_graph", C.c_int), ("steps", C.c_longlong),
                ("launches", C.c_longlong)]


class lbm_server_config(C.Structure):
    _fields_ = [("hbm_budget", C.c_ulonglong), ("device", C.c_int), ("storage", C.c_int), ("quantum", C.c_int),
                ("max_active", C.c_int)]


class lbm_server_timing(C.Structure):
    _fields_ = [("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double), ("steps", C.c_longlong)]


class lbm_server_counters(C.Structure):
    _fields_ = [("waiting", C.c_int), ("active", C.c_int), ("finished", C.c_int), ("peak_active", C.c_int),
                ("bytes_in_use", C.c_longlong), ("rounds", C.c_longlong), ("batch_steps", C.c_longlong),
                ("site_steps", C.c_longlong), ("batch_rebuilds", C.c_longlong), ("reused", C.c_longlong),
                ("pooled", C.c_int), ("clock", C.c_double)]


_lib = None


def lib():
    """Load the CUDA library. Raises if it has not been built or cannot load."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("CUDA library not built: %s (run __graft_entry__.build())" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        H = C.c_void_p
        L.lbm_create.argtypes = [C.POINTER(lbm_config), C.POINTER(H)]
        L.lbm_set_geometry.argtypes = [H, C.POINTER(lbm_geometry)]
        L.lbm_set_ink_rheology.argtypes = [H, C.POINTER(lbm_rheology)]
        L.lbm_set_fields.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
        L.lbm_step.argtypes = [H, C.c_int]
        L.lbm_fields.argtypes = [H, C.c_uint, C.POINTER(C.c_void_p), C.c_int, C.POINTER(lbm_diag)]
        L.lbm_sync.argtypes = [H, C.c_int]
        L.lbm_destroy.argtypes = [H]
        L.lbm_destroy.restype = None
        L.lbm_last_error.argtypes = [H]
        L.lbm_last_error.restype = C.c_char_p
        L.lbm_kernel_launches.argtypes = [H]
        L.lbm_kernel_launches.restype = C.c_longlong
        L.lbm_profile.argtypes = [H, C.c_int]
        L.lbm_timings.argtypes = [H, C.POINTER(lbm_timing)]
        L.lbm_step_noalloc.argtypes = [C.POINTER(lbm_config), C.POINTER(lbm_geometry), C.POINTER(lbm_rheology),
                                       C.c_longlong, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(lbm_diag)]
        L.lbm_batch_create.argtypes = [C.POINTER(H), C.c_int, C.POINTER(H)]
        L.lbm_batch_step.argtypes = [H, C.c_int]
        L.lbm_batch_reset.argtypes = [H, C.POINTER(H), C.c_int]
        L.lbm_batch_sync.argtypes = [H]
        L.lbm_batch_set_plan.argtypes = [H, C.c_int, C.POINTER(C.c_int)]
        L.lbm_batch_autotune.argtypes = [H, C.c_int, C.POINTER(lbm_batch_tuning)]
        L.lbm_batch_info.argtypes = [H, C.POINTER(lbm_batch_plan_info)]
        L.lbm_batch_destroy.argtypes = [H]
        L.lbm_batch_destroy.restype = None
        L.lbm_batch_last_error.argtypes = [H]
        L.lbm_batch_last_error.restype = C.c_char_p
        L.lbm_batch_plan.argtypes = [C.POINTER(C.c_int), C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                     C.c_longlong]
        L.lbm_batch_plan.restype = C.c_longlong
        L.lbm_lattice_bytes.argtypes = [C.POINTER(lbm_config)]
        L.lbm_lattice_bytes.restype = C.c_longlong
        L.lbm_server_create.argtypes = [C.POINTER(lbm_server_config), C.POINTER(H)]
        L.lbm_server_submit.argtypes = [H, C.POINTER(lbm_config), C.POINTER(lbm_geometry), C.POINTER(lbm_rheology),
                                        C.c_longlong, C.POINTER(C.c_longlong)]
        L.lbm_server_poll.argtypes = [H, C.POINTER(C.c_int)]
        L.lbm_server_finished.argtypes = [H, C.POINTER(C.c_longlong), C.c_int]
        L.lbm_server_finished.restype = C.c_int
        L.lbm_server_result.argtypes = [H, C.c_longlong, C.POINTER(C.c_void_p), C.POINTER(lbm_diag),
                                        C.POINTER(lbm_server_timing)]
        L.lbm_server_stats.argtypes = [H, C.POINTER(lbm_server_counters)]
        L.lbm_server_destroy.argtypes = [H]
        L.lbm_server_destroy.restype = None
        L.lbm_server_last_error.argtypes = [H]
        L.lbm_server_last_error.restype = C.c_char_p
        for name in ("lbm_server_create", "lbm_server_submit", "lbm_server_poll", "lbm_server_result",
                     "lbm_server_stats"):
            getattr(L, name).restype = C.c_int
        for name in ("lbm_create", "lbm_set_geometry", "lbm_set_ink_rheology", "lbm_set_fields", "lbm_step",
                     "lbm_fields", "lbm_sync", "lbm_profile", "lbm_timings", "lbm_step_noalloc",
                     "lbm_batch_create", "lbm_batch_reset", "lbm_batch_step", "lbm_batch_sync", "lbm_batch_set_plan",
                     "lbm_batch_autotune", "lbm_batch_info"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


class LBMError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


# --------------------------------------------------------------------------
# thin wrappers with the C names
# --------------------------------------------------------------------------

def _check(h, st):
    if st != LBM_OK:
        raise LBMError(st, lib().lbm_last_error(h).decode())
    return st


def lbm_create(cfg):
    h = C.c_void_p()
    st = lib().lbm_create(C.byref(cfg), C.byref(h))
    if st != LBM_OK:
        raise LBMError(st, lib().lbm_last_error(None).decode())
    return h


def lbm_set_geometry(h, g):
    return _check(h, lib().lbm_set_geometry(h, C.byref(g)))


def lbm_set_ink_rheology(h, r):
    return _check(h, lib().lbm_set_ink_rheology(h, C.byref(r)))


def lbm_set_fields(h, rho_ink_ptr, rho_amb_ptr, u_ptr, on_device):
    return _check(h, lib().lbm_set_fields(h, rho_ink_ptr, rho_amb_ptr, u_ptr, int(on_device)))


def lbm_step(h, nsteps):
    return _check(h, lib().lbm_step(h, int(nsteps)))


def lbm_fields(h, mask, ptrs, on_device, diag=None):
    arr = (C.c_void_p * max(1, len(ptrs)))(*ptrs)
    st = lib().lbm_fields(h, mask, arr, int(on_device), C.byref(diag) if diag is not None else None)
    return st


def lbm_sync(h, timeout_ms=0):
    return _check(h, lib().lbm_sync(h, int(timeout_ms)))


def lbm_destroy(h):
    lib().lbm_destroy(h)


def lbm_last_error(h):
    return lib().lbm_last_error(h).decode()


def lbm_kernel_launches(h):
    return lib().lbm_kernel_launches(h)


def lbm_step_noalloc(cfg, geom, rheo, step, f_in_ptr, f_out_ptr, fields_ptr=None, diag=None):
    """One step on caller-owned device buffers without any device allocation
    (see include/lbm.h). Returns the status; raises nothing."""
    return lib().lbm_step_noalloc(C.byref(cfg), C.byref(geom), C.byref(rheo), int(step), f_in_ptr, f_out_ptr,
                                  fields_ptr, C.byref(diag) if diag is not None else None)


def lbm_profile(h, enable):
    return _check(h, lib().lbm_profile(h, int(enable)))


def lbm_timings(h):
    t = lbm_timing()
    _check(h, lib().lbm_timings(h, C.byref(t)))
    return dict(bulk_ms=t.bulk_ms, plain_ms=t.plain_ms, bulk_launches=t.bulk_launches,
                plain_groups=t.plain_groups, bulk_sites=t.bulk_sites, plain_sites=t.plain_sites)


def _bcheck(b, st):
    if st != LBM_OK:
        raise LBMError(st, lib().lbm_batch_last_error(b).decode())
    return st


def lbm_batch_create(handles):
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    b = C.c_void_p()
    st = lib().lbm_batch_create(arr, len(handles), C.byref(b))
    if st != LBM_OK:
        raise LBMError(st, lib().lbm_batch_last_error(None).decode())
    return b


def lbm_batch_reset(b, handles):
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    return _bcheck(b, lib().lbm_batch_reset(b, arr, len(handles)))


def lbm_batch_step(b, nsteps):
    return _bcheck(b, lib().lbm_batch_step(b, int(nsteps)))


def lbm_batch_sync(b):
    return _bcheck(b, lib().lbm_batch_sync(b))


def lbm_batch_set_plan(b, variant, zchunks):
    arr = (C.c_int * len(zchunks))(*zchunks)
    return _bcheck(b, lib().lbm_batch_set_plan(b, int(variant), arr))


def lbm_batch_autotune(b, trial_steps):
    t = lbm_batch_tuning()
    _bcheck(b, lib().lbm_batch_autotune(b, int(trial_steps), C.byref(t)))
    n = min(t.n_tried, LBM_TUNE_MAX)
    return dict(variant=t.variant, zchunk=t.zchunk, ctas_per_sm=t.ctas_per_sm, ms_per_step=t.ms_per_step,
                tried=[(t.tried_variant[k], t.tried_zchunk[k], t.tried_ms[k]) for k in range(n)],
                tried_ctas=[t.tried_ctas[k] for k in range(n)])


def lbm_batch_info(b):
    i = lbm_batch_plan_info()
    _bcheck(b, lib().lbm_batch_info(b, C.byref(i)))
    return {k: getattr(i, k) for k, _ in lbm_batch_plan_info._fields_}


def lbm_batch_destroy(b):
    lib().lbm_batch_destroy(b)


def lbm_batch_plan(dims, tile_h, zchunks):
    """Work list of the persistent bulk kernel (host-only): list of
    (lattice, x0, y0, za, zb) for lattices of sizes dims [(nx, ny, nz), ...]."""
    n = len(dims)
    d = (C.c_int * (3 * n))(*[v for t in dims for v in t])
    z = (C.c_int * n)(*zchunks)
    cnt = lib().lbm_batch_plan(d, n, int(tile_h), z, None, 0)
    if cnt < 0:
        raise LBMError(LBM_EINVAL, "lbm_batch_plan: invalid arguments")
    out = (C.c_int * (4 * cnt))()
    lib().lbm_batch_plan(d, n, int(tile_h), z, out, cnt)
    return [(out[4 * k], out[4 * k + 1] & 0xFFFF, out[4 * k + 1] >> 16, out[4 * k + 2], out[4 * k + 3])
            for k in range(cnt)]


# --------------------------------------------------------------------------
# structs from dictionaries (same keys as the seeded workloads)
# --------------------------------------------------------------------------

_STORAGE = {"f64": LBM_F64, "f32": LBM_F32, "f16dev": LBM_F16DEV, "bf16dev": LBM_BF16DEV}
_PATH = {"auto": LBM_PATH_AUTO, "plain": LBM_PATH_PLAIN, "fused": LBM_PATH_FUSED}


def make_config(shape, params, path="auto", device=0, stream=0):
    p = dict(params)
    cfg = lbm_config()
    cfg.nx, cfg.ny, cfg.nz = shape
    cfg.velset = p.get("velset", LBM_D3Q19)
    st = p.get("storage", "f64")
    cfg.storage = _STORAGE[st] if isinstance(st, str) else int(st)
    cfg.path = _PATH[path] if isinstance(path, str) else int(path)
    cfg.tau_ambient = p.get("tau_amb", 1.0)
    cfg.rho0_ink = p.get("rho0_ink", 1.0)
    cfg.rho0_amb = p.get("rho0_amb", 1.0)
    cfg.alpha_ink = p.get("alpha_ink") or 0.0
    cfg.alpha_amb = p.get("alpha_amb") or 0.0
    cfg.A = p.get("A", 0.01)
    cfg.beta = p.get("beta", 0.7)
    cfg.zeta_ink = p.get("zeta_ink", 1.0)
    cfg.zeta_amb = p.get("zeta_amb", 1.0)
    cfg.drag_gamma = p.get("drag_gamma", 0.0)
    cfg.drag_height = p.get("drag_height", 4.0)
    cfg.body_force = (C.c_double * 3)(*p.get("body_force", (0.0, 0.0, 0.0)))
    cfg.device = device
    cfg.cuda_stream = stream
    return cfg


def make_geometry(g):
    d = dict(z_mode=LBM_Z_WALLS, top_mode=LBM_TOP_OPEN, nozzle=1, head_pos=(0.0, 0.0), head_vel=(0.0, 0.0),
             r_inner=4.0, wall_thickness=2.0, gap=12, u_ink=0.0, top_vel=(0.0, 0.0, 0.0), rho_top_amb=1.0)
    d.update(g or {})
    return lbm_geometry(d["z_mode"], d["top_mode"], d["nozzle"], (C.c_double * 2)(*d["head_pos"]),
                        (C.c_double * 2)(*d["head_vel"]), d["r_inner"], d["wall_thickness"], d["gap"],
                        d["u_ink"], (C.c_double * 3)(*d["top_vel"]), d["rho_top_amb"])


def make_rheology(r):
    d = dict(law=LBM_POWER_LAW, nu0=0.1, nu_inf=0.0, lam=1.0, n=0.6, K=0.05, tau_min=0.51, tau_max=2.0,
             tol=0.0, max_iter=0)
    d.update(r or {})
    return lbm_rheology(d["law"], d["nu0"], d["nu_inf"], d["lam"], d["n"], d["K"], d["tau_min"], d["tau_max"],
                        d["tol"], d["max_iter"])


# --------------------------------------------------------------------------
# Lattice: one handle with torch-owned device memory
# --------------------------------------------------------------------------

class _TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self.live = {}
        self.c_alloc = ALLOC_FN(self._alloc)
        self.c_free = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except RuntimeError:
            return None
        ptr = t.data_ptr()
        self.live[ptr] = t
        return ptr

    def _free(self, ptr, ctx):
        self.live.pop(ptr, None)


class Lattice:
    """One lattice resident on the GPU, driven through the C ABI.

    shape = (nx, ny, nz); params/geom/rheo are dictionaries with the keys of
    ``paper_2102_02655_gb300.inputs`` workloads."""

    def __init__(self, shape, params=None, geom=None, rheo=None, path="auto", device=0, stream=None):
        import torch
        self.torch = torch
        self.shape = tuple(shape)
        self.params = dict(params or {})
        st = self.params.get("storage", "f64")
        self.dtype = torch.float64 if st in ("f64", LBM_F64) else torch.float32
        self.device = torch.device("cuda", device)
        if stream is None:
            # a stream of its own: handle 0 would mean "library-created stream"
            # to the C ABI, and events recorded on torch's default stream would
            # not order with it
            stream = torch.cuda.Stream(self.device)
        self.stream = stream
        self._allocator = _TorchAllocator(self.device)
        cfg = make_config(self.shape, self.params, path=path, device=device, stream=stream.cuda_stream)
        cfg.alloc = self._allocator.c_alloc
        cfg.free = self._allocator.c_free
        self._cfg = cfg
        self.h = lbm_create(cfg)
        if rheo is not None:
            self.set_rheology(rheo)
        if geom is not None:
            self.set_geometry(geom)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_sites(self):
        nx, ny, nz = self.shape
        return nx * ny * nz

    def set_geometry(self, geom):
        lbm_set_geometry(self.h, make_geometry(geom))

    def set_rheology(self, rheo):
        lbm_set_ink_rheology(self.h, make_rheology(rheo))

    def set_fields(self, rho_ink, rho_amb, u=None):
        """Densities [nz, ny, nx] and optional velocity [3, nz, ny, nx]; numpy
        arrays (host path) or torch tensors on this device."""
        t = self.torch
        on_dev = isinstance(rho_ink, t.Tensor) and rho_ink.is_cuda
        if on_dev:
            a = rho_ink.to(self.dtype).contiguous()
            b = rho_amb.to(self.dtype).contiguous()
            c = u.to(self.dtype).contiguous() if u is not None else None
            lbm_set_fields(self.h, a.data_ptr(), b.data_ptr(), c.data_ptr() if c is not None else None, 1)
            lbm_sync(self.h)
        else:
            npd = np.float64 if self.dtype == t.float64 else np.float32
            a = np.ascontiguousarray(rho_ink, dtype=npd)
            b = np.ascontiguousarray(rho_amb, dtype=npd)
            c = np.ascontiguousarray(u, dtype=npd) if u is not None else None
            lbm_set_fields(self.h, a.ctypes.data, b.ctypes.data, c.ctypes.data if c is not None else None, 0)
            lbm_sync(self.h)

    def step(self, n=1):
        lbm_step(self.h, n)

    def sync(self, timeout_ms=0):
        lbm_sync(self.h, timeout_ms)

    def fields(self, mask=ALL_FIELDS, device=False, out=None):
        """Fields of the last step as a dict of numpy arrays [nz, ny, nx] (or
        torch tensors on the device), plus 'diag'. ``out`` may give the
        destination arrays (e.g. pinned host memory) in field order. Raises on
        LBM_EUNSTABLE."""
        nx, ny, nz = self.shape
        names = []
        bits = [(LBM_FIELD_RHO_INK, ["rho_ink"]), (LBM_FIELD_RHO_AMB, ["rho_amb"]),
                (LBM_FIELD_U, ["ux", "uy", "uz"]), (LBM_FIELD_NU, ["nu"]), (LBM_FIELD_P, ["p"]),
                (LBM_FIELD_PHI, ["rhoN"]), (LBM_FIELD_SOLID, ["solid"])]
        for b, ns in bits:
            if mask & b:
                names += ns
        t = self.torch
        if out is not None:
            bufs = list(out)
            assert len(bufs) == len(names)
            ptrs = [b.data_ptr() if isinstance(b, t.Tensor) else b.ctypes.data for b in bufs]
        elif device:
            bufs = [t.empty((nz, ny, nx), dtype=self.dtype, device=self.device) for _ in names]
            ptrs = [b.data_ptr() for b in bufs]
        else:
            npd = np.float64 if self.dtype == t.float64 else np.float32
            bufs = [np.empty((nz, ny, nx), dtype=npd) for _ in names]
            ptrs = [b.ctypes.data for b in bufs]
        d = lbm_diag()
        st = lbm_fields(self.h, mask, ptrs, 1 if device else 0, d)
        out = dict(zip(names, bufs))
        out["diag"] = dict(mass=list(d.mass), momentum=list(d.momentum), bc_flux=list(d.bc_flux),
                           created=list(d.created), destroyed=list(d.destroyed), step=d.step,
                           unstable=d.unstable)
        if st != LBM_OK:
            raise LBMError(st, lbm_last_error(self.h))
        return out

    def diag(self):
        return self.fields(mask=0)["diag"]

    def kernel_launches(self):
        return lbm_kernel_launches(self.h)

    def profile(self, enable=True):
        lbm_profile(self.h, enable)

    def timings(self):
        return lbm_timings(self.h)


class Batch:
    """Many lattices advanced together (see lbm_batch_* in include/lbm.h).
    The Lattice objects stay owned by the caller and must outlive the batch."""

    def __init__(self, lattices):
        self.lattices = list(lattices)
        self.b = lbm_batch_create([lat.h for lat in self.lattices])

    def reset(self, lattices):
        lbm_batch_reset(self.b, [lat.h for lat in lattices])
        self.lattices = list(lattices)

    def step(self, n):
        lbm_batch_step(self.b, n)

    def sync(self):
        lbm_batch_sync(self.b)

    def set_plan(self, variant, zchunks):
        if isinstance(zchunks, int):
            zchunks = [zchunks] * len(self.lattices)
        lbm_batch_set_plan(self.b, variant, zchunks)

    def autotune(self, trial_steps=4):
        return lbm_batch_autotune(self.b, trial_steps)

    def info(self):
        return lbm_batch_info(self.b)

    def close(self):
        if self.b is not None:
            lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop over the C ABI (see lbm_server_* in include/lbm.h):
    submit print-run requests, poll to run scheduling rounds, collect results."""

    def __init__(self, hbm_budget, storage="f32", quantum=100, max_active=32, device=0):
        cfg = lbm_server_config(int(hbm_budget), int(device),
                                _STORAGE[storage] if isinstance(storage, str) else int(storage),
                                int(quantum), int(max_active))
        self.storage = storage
        self.s = C.c_void_p()
        st = lib().lbm_server_create(C.byref(cfg), C.byref(self.s))
        if st != LBM_OK:
            raise LBMError(st, lib().lbm_server_last_error(None).decode())
        self.shapes = {}

    def _check(self, st):
        if st != LBM_OK:
            raise LBMError(st, lib().lbm_server_last_error(self.s).decode())

    def submit(self, shape, params, geom, rheo, nsteps):
        cfg = make_config(tuple(shape), dict(params, storage=self.storage), path="fused")
        g = make_geometry(geom)
        r = make_rheology(rheo)
        rid = C.c_longlong()
        self._check(lib().lbm_server_submit(self.s, C.byref(cfg), C.byref(g), C.byref(r), int(nsteps),
                                            C.byref(rid)))
        self.shapes[rid.value] = tuple(shape)
        return rid.value

    def poll(self):
        n = C.c_int()
        self._check(lib().lbm_server_poll(self.s, C.byref(n)))
        return n.value

    def finished(self):
        n = lib().lbm_server_finished(self.s, None, 0)
        ids = (C.c_longlong * max(1, n))()
        lib().lbm_server_finished(self.s, ids, n)
        return list(ids[:n])

    def result(self, rid, fields=True):
        """(status, fields dict or None, diag dict, timing dict); forgets the request."""
        nx, ny, nz = self.shapes.pop(rid)
        npd = np.float64 if self.storage in ("f64", LBM_F64) else np.float32
        bufs = [np.empty((nz, ny, nx), dtype=npd) for _ in range(5)] if fields else None
        ptrs = (C.c_void_p * 5)(*[b.ctypes.data for b in bufs]) if fields else None
        d = lbm_diag()
        t = lbm_server_timing()
        st = lib().lbm_server_result(self.s, int(rid), ptrs, C.byref(d), C.byref(t))
        out = dict(zip(("rho_ink", "rho_amb", "ux", "uy", "uz"), bufs)) if fields else None
        diag = dict(mass=list(d.mass), momentum=list(d.momentum), bc_flux=list(d.bc_flux), created=list(d.created),
                    destroyed=list(d.destroyed), step=d.step, unstable=d.unstable)
        timing = dict(t_submit=t.t_submit, t_admit=t.t_admit, t_done=t.t_done, steps=t.steps)
        return st, out, diag, timing

    def stats(self):
        c = lbm_server_counters()
        lib().lbm_server_stats(self.s, C.byref(c))
        return {k: getattr(c, k) for k, _ in lbm_server_counters._fields_}

    def close(self):
        if self.s is not None:
            lib().lbm_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lattice_bytes(shape, params):
    cfg = make_config(tuple(shape), params)
    return lib().lbm_lattice_bytes(C.byref(cfg))
