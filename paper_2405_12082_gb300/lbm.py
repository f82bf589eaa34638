"""ctypes binding of liblbm.so (include/lbm.h): the same names, argument marshalling only.

Every computation runs in the CUDA library; this module converts Python values,
numpy arrays and torch tensors into the C structs and pointers of the ABI and turns
non-zero status codes into LbmError.  Importing it raises if the library has not
been built (there is no CPU fallback): call __graft_entry__.build() or
``python -m paper_2405_12082_gb300.build``.
"""
import ctypes
import math
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblbm.so")

# ---- constants (include/lbm.h) -------------------------------------------------------
LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA = 0, -1, -2, -3
LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_EUNSUPPORTED = -4, -5, -6
LBM_F64, LBM_F32, LBM_F16S, LBM_BF16 = 0, 1, 2, 3
LBM_PIPE, LBM_BOX = 0, 1
LBM_HALFWAY, LBM_FULLWAY, LBM_BOUZIDI = 0, 1, 2
LBM_REST, LBM_LAMINAR, LBM_LOGLAW = 0, 1, 2
LBM_J_UBULK, LBM_J_WSS = 0, 1
LBM_MRT, LBM_BGK = 0, 1
LBM_EQ_HERMITE6, LBM_EQ_ORDER2 = 0, 1
LBM_MAX_TRIGGER_MODES = 8
LBM_MAX_MEMBERS = 64
LBM_STATIC_REDUCE_MAX_BLOCKS = 1216
LBM_STATIC_REDUCE_MAX_CELLS = 159072862

PRECISIONS = {"f64": LBM_F64, "f32": LBM_F32, "f16s": LBM_F16S, "bf16": LBM_BF16}
WALLS = {"halfway": LBM_HALFWAY, "fullway": LBM_FULLWAY, "bouzidi": LBM_BOUZIDI}
PROFILES = {"rest": LBM_REST, "laminar": LBM_LAMINAR, "loglaw": LBM_LOGLAW}
MODELS = {"mrt": LBM_MRT, "bgk": LBM_BGK}
EQUILIBRIA = {"hermite6": LBM_EQ_HERMITE6, "order2": LBM_EQ_ORDER2}


class LbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("lbm status %d: %s" % (status, message))
        self.status = status


class lbm_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("geometry", ctypes.c_int32), ("R", ctypes.c_double), ("precision", ctypes.c_int32),
                ("wall", ctypes.c_int32), ("f16_log2_scale", ctypes.c_int32)]


class lbm_relax(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_double), ("rates", ctypes.POINTER(ctypes.c_double))]


def make_relax(omega, rates=None):
    """lbm_relax with an optional 27-entry rate vector (kept alive with the struct)."""
    r = lbm_relax(float(omega))
    if rates is not None:
        if len(rates) != 27:
            raise ValueError("rates needs 27 entries")
        arr = (ctypes.c_double * 27)(*[float(x) for x in rates])
        r.rates = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
        r._rates_keep = arr
    return r


class lbm_force(ctypes.Structure):
    _fields_ = [("g", ctypes.c_double * 3), ("trigger", ctypes.c_int32), ("n_modes", ctypes.c_int32),
                ("k_theta", ctypes.c_int32 * LBM_MAX_TRIGGER_MODES),
                ("weight", ctypes.c_double * LBM_MAX_TRIGGER_MODES),
                ("phase", ctypes.c_double * LBM_MAX_TRIGGER_MODES),
                ("A0", ctypes.c_double), ("kappa", ctypes.c_double), ("l0", ctypes.c_double),
                ("l", ctypes.c_double), ("period", ctypes.c_double), ("h", ctypes.c_double),
                ("kz", ctypes.c_int32), ("t_end", ctypes.c_int64), ("gz_field", ctypes.c_void_p)]


class lbm_modes_cfg(ctypes.Structure):
    _fields_ = [("n_sections", ctypes.c_int32), ("n_rings", ctypes.c_int32),
                ("r_over_R", ctypes.c_double * 16), ("n_theta", ctypes.c_int32), ("n_modes", ctypes.c_int32)]


class lbm_info(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int64), ("n_fluid", ctypes.c_int64), ("t", ctypes.c_int64),
                ("population_bytes", ctypes.c_int64), ("n_members", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("launches", ctypes.c_int64), ("variant", ctypes.c_int32),
                ("step_threads", ctypes.c_int32), ("n_variants", ctypes.c_int32), ("graph_chunk", ctypes.c_int32),
                ("variant_odd", ctypes.c_int32)]


# device-memory hooks (lbm_set_allocator)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


def _load():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("liblbm.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, D, U64, SZ = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                               ctypes.c_uint64, ctypes.c_size_t)
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "lbm_create": [PP, ctypes.POINTER(lbm_grid), ctypes.POINTER(lbm_relax), ctypes.POINTER(lbm_force), P],
        "lbm_ensemble_create": [PP, I32, ctypes.POINTER(lbm_grid), ctypes.POINTER(lbm_relax),
                                ctypes.POINTER(lbm_force), P],
        "lbm_set_stream": [P, P],
        "lbm_select_member": [P, I32],
        "lbm_get_info": [P, ctypes.POINTER(lbm_info)],
        "lbm_set_relax": [P, ctypes.POINTER(lbm_relax)],
        "lbm_set_force": [P, ctypes.POINTER(lbm_force)],
        "lbm_set_collision": [P, I32, I32],
        "lbm_init": [P, I32, D, U64],
        "lbm_init_fields": [P, P, P],
        "lbm_step": [P, I64],
        "lbm_set_check": [P, I64, D],
        "lbm_moments": [P, P, P],
        "lbm_get_populations": [P, P],
        "lbm_set_populations": [P, P],
        "lbm_get_raw": [P, P, SZ],
        "lbm_set_raw": [P, P, SZ],
        "lbm_reduce": [P, P],
        "lbm_stats_enable": [P, I32],
        "lbm_stats_get": [P, P, ctypes.POINTER(ctypes.c_int64)],
        "lbm_modes": [P, ctypes.POINTER(lbm_modes_cfg), P],
        "lbm_adjoint": [P, I64, I32, I64, ctypes.POINTER(ctypes.c_double), P, ctypes.POINTER(ctypes.c_double)],
        "lbm_profile_enable": [P, I32],
        "lbm_profile_read": [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)],
        "lbm_fluid_mask": [P, P],
        "lbm_reduce_static": [P, I32, I32, I64, P, P],
        "lbm_probe_fp32": [P, P],
        "lbm_set_graph": [P, I32],
        "lbm_save": [P, ctypes.c_char_p],
        "lbm_stats_profile": [P, I32, D, P],
        "lbm_dominant_modes": [P, I32, I32, I32, I32, I32, I32, P],
        "lbm_transition_matrix": [P, I64, I32, I32, I32, P, P],
        "lbm_mode_correlation": [P, I64, I32, I32, I32, P],
        "lbm_load": [P, ctypes.c_char_p],
        "lbm_set_variant": [P, I32],
        "lbm_set_variants": [P, I32, I32],
        "lbm_test_expire_wait": [P, I32],
        "lbm_autotune": [P, I32, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)],
    }
    sig["lbm_set_allocator"] = [ALLOC_FN, FREE_FN, P]
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.lbm_free.argtypes = [P]
    lib.lbm_free.restype = None
    lib.lbm_last_error.argtypes = [P]
    lib.lbm_last_error.restype = ctypes.c_char_p
    return lib


LIB = _load()
EXPORTED = ("lbm_create", "lbm_ensemble_create", "lbm_free", "lbm_last_error", "lbm_set_stream",
            "lbm_select_member", "lbm_get_info", "lbm_set_relax", "lbm_set_force", "lbm_init",
            "lbm_init_fields", "lbm_step", "lbm_set_check", "lbm_moments", "lbm_get_populations",
            "lbm_set_populations", "lbm_get_raw", "lbm_set_raw", "lbm_reduce", "lbm_stats_enable",
            "lbm_stats_get", "lbm_modes", "lbm_adjoint", "lbm_profile_enable", "lbm_profile_read",
            "lbm_fluid_mask", "lbm_reduce_static", "lbm_set_graph", "lbm_set_variant", "lbm_autotune",
            "lbm_save", "lbm_load", "lbm_stats_profile", "lbm_dominant_modes", "lbm_transition_matrix",
            "lbm_mode_correlation", "lbm_set_collision", "lbm_set_allocator", "lbm_test_expire_wait", "lbm_set_variants",
            "lbm_probe_fp32")


# ---- marshalling helpers -----------------------------------------------------------------
def ptr(x):
    """Address of a torch tensor, numpy array, ctypes object or int (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    return ctypes.addressof(x)


def _check(ctx, rc):
    if rc != LBM_OK:
        raise LbmError(rc, LIB.lbm_last_error(ctx).decode())
    return rc


def make_grid(nx, ny, nz, R=0.0, geometry="pipe", precision="f32", wall="halfway", f16_log2_scale=0):
    return lbm_grid(nx, ny, nz, LBM_PIPE if geometry == "pipe" else LBM_BOX, float(R),
                    PRECISIONS[precision] if isinstance(precision, str) else precision,
                    WALLS[wall] if isinstance(wall, str) else wall, f16_log2_scale)


def make_force(g=(0.0, 0.0, 0.0), trigger=None, gz_field=None):
    """trigger: dict with keys A0, kappa, kz, l0, l, period, h, t_end and modes =
    [(k_theta, weight, phase), ...] (Eq. (TurbForce) per mode)."""
    f = lbm_force()
    for k in range(3):
        f.g[k] = float(g[k])
    if trigger is not None:
        f.trigger = 1
        modes = trigger["modes"]
        f.n_modes = len(modes)
        for q, (kt, wgt, ph) in enumerate(modes):
            f.k_theta[q] = int(kt)
            f.weight[q] = float(wgt)
            f.phase[q] = float(ph)
        f.A0 = float(trigger["A0"])
        f.kappa = float(trigger["kappa"])
        f.kz = int(trigger["kz"])
        f.l0 = float(trigger["l0"])
        f.l = float(trigger["l"])
        f.period = float(trigger["period"])
        f.h = float(trigger["h"])
        f.t_end = int(trigger.get("t_end", 2 ** 62))
    f.gz_field = ptr(gz_field)
    return f


def make_modes_cfg(n_sections, r_over_R, n_theta, n_modes):
    c = lbm_modes_cfg()
    c.n_sections = n_sections
    c.n_rings = len(r_over_R)
    for j, r in enumerate(r_over_R):
        c.r_over_R[j] = float(r)
    c.n_theta = n_theta
    c.n_modes = n_modes
    return c


# ---- the ABI, name for name --------------------------------------------------------------
def lbm_create(grid, relax, force=None, stream=None):
    out = ctypes.c_void_p()
    rc = LIB.lbm_create(ctypes.byref(out), ctypes.byref(grid), ctypes.byref(relax),
                        ctypes.byref(force) if force is not None else None, ptr(stream))
    _check(None, rc)
    return out.value


def lbm_ensemble_create(grids, relaxes, forces=None, stream=None):
    n = len(grids)
    G = (lbm_grid * n)(*grids)
    Rl = (lbm_relax * n)(*relaxes)
    F = (lbm_force * n)(*forces) if forces is not None else None
    out = ctypes.c_void_p()
    rc = LIB.lbm_ensemble_create(ctypes.byref(out), n, G, Rl, F, ptr(stream))
    _check(None, rc)
    return out.value


def lbm_free(ctx):
    LIB.lbm_free(ctx)


def lbm_last_error(ctx):
    return LIB.lbm_last_error(ctx).decode()


def lbm_set_stream(ctx, stream):
    return _check(ctx, LIB.lbm_set_stream(ctx, ptr(stream)))


def lbm_select_member(ctx, member):
    return _check(ctx, LIB.lbm_select_member(ctx, member))


def lbm_get_info(ctx):
    info = lbm_info()
    _check(ctx, LIB.lbm_get_info(ctx, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in lbm_info._fields_}


def lbm_set_relax(ctx, relax):
    return _check(ctx, LIB.lbm_set_relax(ctx, ctypes.byref(relax)))


def lbm_set_force(ctx, force):
    return _check(ctx, LIB.lbm_set_force(ctx, ctypes.byref(force)))


def lbm_set_collision(ctx, model="mrt", equilibrium="hermite6"):
    model = MODELS[model] if isinstance(model, str) else model
    equilibrium = EQUILIBRIA[equilibrium] if isinstance(equilibrium, str) else equilibrium
    return _check(ctx, LIB.lbm_set_collision(ctx, int(model), int(equilibrium)))


def lbm_init(ctx, profile=LBM_REST, noise_amp=0.0, seed=0):
    profile = PROFILES[profile] if isinstance(profile, str) else profile
    return _check(ctx, LIB.lbm_init(ctx, profile, float(noise_amp), int(seed)))


def lbm_init_fields(ctx, rho, u):
    return _check(ctx, LIB.lbm_init_fields(ctx, ptr(rho), ptr(u)))


def lbm_step(ctx, n=1):
    return _check(ctx, LIB.lbm_step(ctx, int(n)))


def lbm_set_check(ctx, every, max_mass_drift):
    return _check(ctx, LIB.lbm_set_check(ctx, int(every), float(max_mass_drift)))


def lbm_moments(ctx, rho, u):
    return _check(ctx, LIB.lbm_moments(ctx, ptr(rho), ptr(u)))


def lbm_get_populations(ctx, f):
    return _check(ctx, LIB.lbm_get_populations(ctx, ptr(f)))


def lbm_set_populations(ctx, f):
    return _check(ctx, LIB.lbm_set_populations(ctx, ptr(f)))


def lbm_get_raw(ctx, buf, nbytes):
    return _check(ctx, LIB.lbm_get_raw(ctx, ptr(buf), int(nbytes)))


def lbm_set_raw(ctx, buf, nbytes):
    return _check(ctx, LIB.lbm_set_raw(ctx, ptr(buf), int(nbytes)))


def lbm_reduce(ctx):
    out = (ctypes.c_double * 5)()
    _check(ctx, LIB.lbm_reduce(ctx, ctypes.addressof(out)))
    return list(out)


def lbm_stats_enable(ctx, every):
    return _check(ctx, LIB.lbm_stats_enable(ctx, int(every)))


def lbm_stats_get(ctx, acc):
    count = ctypes.c_int64()
    _check(ctx, LIB.lbm_stats_get(ctx, ptr(acc), ctypes.byref(count)))
    return count.value


def lbm_modes(ctx, cfg, E):
    return _check(ctx, LIB.lbm_modes(ctx, ctypes.byref(cfg), ptr(E)))


def lbm_adjoint(ctx, T, objective, checkpoint_every, dJ_dgz):
    J = ctypes.c_double()
    dw = ctypes.c_double()
    _check(ctx, LIB.lbm_adjoint(ctx, int(T), int(objective), int(checkpoint_every), ctypes.byref(J),
                                ptr(dJ_dgz), ctypes.byref(dw)))
    return J.value, dw.value


def lbm_profile_enable(ctx, on):
    return _check(ctx, LIB.lbm_profile_enable(ctx, 1 if on else 0))


def lbm_profile_read(ctx):
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(ctx, LIB.lbm_profile_read(ctx, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def lbm_stats_profile(ctx, nbins, dr):
    import numpy as np
    out = np.empty((nbins, 6))
    _check(ctx, LIB.lbm_stats_profile(ctx, int(nbins), float(dr), ptr(out)))
    return out


def _host_call(rc, what):
    if rc != LBM_OK:
        raise LbmError(rc, what + " rejected its arguments")


def lbm_dominant_modes(E, ring=0, m_lo=1, m_hi=10):
    """E: float64 [n_sections][n_rings][n_modes + 1] (host) -> int32 [n_sections]."""
    import numpy as np
    E = np.ascontiguousarray(E, dtype=np.float64)
    ns, nr, nm1 = E.shape
    k = np.empty(ns, dtype=np.int32)
    _host_call(LIB.lbm_dominant_modes(ptr(E), ns, nr, nm1 - 1, ring, m_lo, m_hi, ptr(k)), "lbm_dominant_modes")
    return k


def lbm_transition_matrix(series, m_lo=1, m_hi=10, lag=1):
    import numpy as np
    s = np.ascontiguousarray(series, dtype=np.int32)
    K = m_hi - m_lo + 1
    T = np.empty((K, K))
    c = np.empty((K, K), dtype=np.int64)
    _host_call(LIB.lbm_transition_matrix(ptr(s), s.size, m_lo, m_hi, lag, ptr(T), ptr(c)), "lbm_transition_matrix")
    return T, c


def lbm_mode_correlation(series, m_lo=1, m_hi=10, max_lag=100):
    import numpy as np
    s = np.ascontiguousarray(series, dtype=np.int32)
    F = np.empty((m_hi - m_lo + 1, max_lag + 1))
    _host_call(LIB.lbm_mode_correlation(ptr(s), s.size, m_lo, m_hi, max_lag, ptr(F)), "lbm_mode_correlation")
    return F


def lbm_save(ctx, path):
    return _check(ctx, LIB.lbm_save(ctx, os.fsencode(path)))


def lbm_load(ctx, path):
    return _check(ctx, LIB.lbm_load(ctx, os.fsencode(path)))


def lbm_set_graph(ctx, chunk):
    return _check(ctx, LIB.lbm_set_graph(ctx, int(chunk)))


def lbm_set_variant(ctx, variant):
    return _check(ctx, LIB.lbm_set_variant(ctx, int(variant)))


def lbm_set_variants(ctx, even, odd):
    return _check(ctx, LIB.lbm_set_variants(ctx, int(even), int(odd)))


def lbm_test_expire_wait(ctx, tile):
    return _check(ctx, LIB.lbm_test_expire_wait(ctx, int(tile)))


def lbm_autotune(ctx, steps):
    v = ctypes.c_int32()
    us = ctypes.c_double()
    _check(ctx, LIB.lbm_autotune(ctx, int(steps), ctypes.byref(v), ctypes.byref(us)))
    return v.value, us.value


def lbm_fluid_mask(ctx, mask):
    return _check(ctx, LIB.lbm_fluid_mask(ctx, ptr(mask)))


def lbm_reduce_static(pops, precision, f16_log2_scale, n_cells, out, stream=None):
    """Allocation-free reduction (see include/lbm.h); out is a device buffer of 5 doubles."""
    precision = PRECISIONS[precision] if isinstance(precision, str) else precision
    rc = LIB.lbm_reduce_static(ptr(pops), int(precision), int(f16_log2_scale), int(n_cells), ptr(out), ptr(stream))
    if rc != LBM_OK:
        raise LbmError(rc, "lbm_reduce_static: " + LIB.lbm_last_error(None).decode())
    return rc


def lbm_probe_fp32(stream=None):
    """Measured FP32 rate of the current device (see include/lbm.h): a dict with the scalar
    and paired FMA rates in TFLOP/s and the FFMA warp-instruction rate per SM sub-partition."""
    out = (ctypes.c_double * 4)()
    rc = LIB.lbm_probe_fp32(ptr(out), ptr(stream))
    if rc != LBM_OK:
        raise LbmError(rc, "lbm_probe_fp32: " + LIB.lbm_last_error(None).decode())
    return {"ffma_tflops": out[0], "ffma2_tflops": out[1], "warp_ffma_per_s_per_smsp": out[2], "ms": out[3]}


class Lattice:
    """Owning handle of one context (single pipe or ensemble) with tensor conveniences."""

    def __init__(self, grid, relax, force=None, stream=None, ensemble=None):
        import torch
        if stream is None and torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
        self._keep = [force]
        self.force = force
        if ensemble is not None:
            grids, relaxes, forces = ensemble
            self._keep.append(forces)
            self.ctx = lbm_ensemble_create(grids, relaxes, forces, stream)
            self.grids = list(grids)
        else:
            self.ctx = lbm_create(grid, relax, force, stream)
            self.grids = [grid]
        self.member = 0

    def close(self):
        if getattr(self, "ctx", None):
            lbm_free(self.ctx)
            self.ctx = None

    def __del__(self):
        self.close()

    @property
    def grid(self):
        return self.grids[self.member]

    def select(self, m):
        lbm_select_member(self.ctx, m)
        self.member = m

    def info(self):
        return lbm_get_info(self.ctx)

    def init(self, profile="rest", noise_amp=0.0, seed=0):
        lbm_init(self.ctx, profile, noise_amp, seed)

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def moments(self, device="cuda"):
        import torch
        g = self.grid
        dt = torch.float64 if g.precision == LBM_F64 else torch.float32
        rho = torch.empty((g.nz, g.ny, g.nx), dtype=dt, device=device)
        u = torch.empty((3, g.nz, g.ny, g.nx), dtype=dt, device=device)
        lbm_moments(self.ctx, rho, u)
        return rho, u

    def populations(self):
        import numpy as np
        g = self.grid
        f = np.empty((27, g.nz, g.ny, g.nx), dtype=np.float64)
        lbm_get_populations(self.ctx, f)
        return f

    def set_populations(self, f):
        import numpy as np
        lbm_set_populations(self.ctx, np.ascontiguousarray(f, dtype=np.float64))

    def modes(self, n_sections=16, r_over_R=(0.78,), n_theta=None, n_modes=32):
        import numpy as np
        g = self.grid
        if n_theta is None:
            n_theta = 1 << max(3, math.ceil(math.log2(2 * math.pi * r_over_R[0] * g.R)))
        cfg = make_modes_cfg(n_sections, r_over_R, n_theta, n_modes)
        E = np.empty((n_sections, len(r_over_R), n_modes + 1))
        lbm_modes(self.ctx, cfg, E)
        return E


# ---- autograd wrapper of the adjoint --------------------------------------------------------
def _autograd_function():
    import torch

    class PipeObjective(torch.autograd.Function):
        """J(g_z, omega) of a single half-way pipe over T steps from the lattice's current state
        (lbm_adjoint): forward sets the per-cell axial acceleration g_z and omega, runs the
        adjoint call and returns J; backward scales the gradients the call returned.  The
        lattice advances by T steps."""

        @staticmethod
        def forward(ctx, gz, omega, lattice, T, objective, checkpoint_every):
            force = lbm_force.from_buffer_copy(lattice.force if lattice.force is not None else lbm_force())
            gz_c = gz.detach().contiguous()
            force.gz_field = gz_c.data_ptr()
            lbm_set_force(lattice.ctx, force)
            lattice._keep.append(gz_c)
            lattice.force = force
            lbm_set_relax(lattice.ctx, make_relax(float(omega)))
            dgz = torch.zeros(gz.shape, dtype=torch.float64, device=gz.device)
            obj = LBM_J_WSS if objective in ("wss", LBM_J_WSS) else LBM_J_UBULK
            J, dw = lbm_adjoint(lattice.ctx, T, obj, checkpoint_every, dgz)
            ctx.save_for_backward(dgz)
            ctx.dw = dw
            ctx.gz_dtype = gz.dtype
            ctx.omega_like = omega
            return torch.tensor(J, dtype=torch.float64, device=gz.device)

        @staticmethod
        def backward(ctx, gJ):
            (dgz,) = ctx.saved_tensors
            g_gz = (gJ * dgz).to(ctx.gz_dtype)
            om = ctx.omega_like
            g_om = (gJ * ctx.dw).to(om.dtype).to(om.device) if torch.is_tensor(om) else None
            return g_gz, g_om, None, None, None, None

    return PipeObjective


def pipe_objective(lattice, gz, omega, T, objective="ubulk", checkpoint_every=0):
    """Differentiable J of the adjoint objectives: J = pipe_objective(L, gz, omega, T) with gz a
    device tensor of the storage's compute type, shape (nz, ny, nx), and omega a 0-d tensor;
    J.backward() fills gz.grad and omega.grad from one lbm_adjoint call."""
    global _PIPE_OBJECTIVE
    if _PIPE_OBJECTIVE is None:
        _PIPE_OBJECTIVE = _autograd_function()
    return _PIPE_OBJECTIVE.apply(gz, omega, lattice, int(T), objective, int(checkpoint_every))


_PIPE_OBJECTIVE = None


# ---- device-memory hooks ---------------------------------------------------------------------
_ALLOCATOR = None      # the installed callbacks, kept alive while the library may call them


def lbm_set_allocator(alloc=None, free=None):
    """Install Python callables alloc(bytes, stream) -> int address and free(address, stream)
    as the device allocator of contexts created from now on; no arguments restore
    cudaMalloc.  Contexts keep the hooks they were created with: keep them installed (or
    referenced) until those contexts are freed."""
    global _ALLOCATOR
    if alloc is None and free is None:
        _check(None, LIB.lbm_set_allocator(ctypes.cast(None, ALLOC_FN), ctypes.cast(None, FREE_FN), None))
        return

    def _a(nbytes, stream, user):
        return int(alloc(int(nbytes), stream or 0))

    def _f(ptr_, stream, user):
        free(int(ptr_), stream or 0)

    cbs = (ALLOC_FN(_a), FREE_FN(_f))
    _check(None, LIB.lbm_set_allocator(cbs[0], cbs[1], None))
    _ALLOCATOR = (cbs, alloc, free, _ALLOCATOR)      # older hooks stay referenced too


def use_torch_allocator():
    """Back every later context's device memory with PyTorch's caching allocator."""
    import torch

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, torch.cuda.current_device(), stream)

    def free(ptr_, stream):
        torch.cuda.caching_allocator_delete(ptr_)

    lbm_set_allocator(alloc, free)
