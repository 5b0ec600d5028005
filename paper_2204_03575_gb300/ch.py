"""Python binding of libch.so (include/ch.h): argument marshalling only.

Every computation runs in the CUDA library; this module passes torch device
pointers and the current CUDA stream through ctypes and turns status codes into
exceptions.  The library must have been built (``python -m
paper_2204_03575_gb300.build``); there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libch.so")

_lib = None


class ChError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: status {status} ({STATUS.get(status, '?')}): {message}")
        self.status = status


STATUS = {0: "CH_OK", 1: "CH_ERR_ARG", 2: "CH_ERR_CUDA", 3: "CH_ERR_OOM", 4: "CH_ERR_NOT_CONVERGED",
          5: "CH_ERR_BREAKDOWN", 6: "CH_ERR_NONFINITE", 7: "CH_ERR_STATE", 8: "CH_ERR_INTERNAL"}
OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_NONFINITE, ERR_STATE, ERR_INTERNAL = range(9)


class Params(ctypes.Structure):
    """Mirror of ch_params."""
    _fields_ = [
        ("dim", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
        ("tau", ctypes.c_double), ("eps", ctypes.c_double), ("mobility", ctypes.c_double),
        ("bc_mode", ctypes.c_int32), ("evap_sign", ctypes.c_int32), ("potential", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("k_evap", ctypes.c_double), ("g_p", ctypes.c_double), ("g_nfa", ctypes.c_double),
        ("h_p", ctypes.c_double), ("h_nfa", ctypes.c_double), ("rtol", ctypes.c_double),
        ("restart", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("cheb_degree", ctypes.c_int32),
        ("coarse_max", ctypes.c_int32), ("amg_theta", ctypes.c_double),
        ("vcycles_M", ctypes.c_int32), ("vcycles_H", ctypes.c_int32), ("autotune", ctypes.c_int32),
        ("cheb_lower", ctypes.c_double), ("graphs", ctypes.c_int32), ("cheb_degree_coarse", ctypes.c_int32),
        ("cheb_degree_M", ctypes.c_int32), ("krylov", ctypes.c_int32), ("pattern", ctypes.c_int32),
        ("precond_M", ctypes.c_int32), ("cheb_M_steps", ctypes.c_int32),
        ("chi_pn", ctypes.c_double), ("chi_ps", ctypes.c_double), ("chi_ns", ctypes.c_double),
        ("N_p", ctypes.c_double), ("N_nfa", ctypes.c_double), ("N_s", ctypes.c_double),
        ("fh_delta", ctypes.c_double), ("pdl", ctypes.c_int32), ("gs_reorth", ctypes.c_int32),
    ]

    def __init__(self, **kw):
        super().__init__()
        lib().ch_params_default(ctypes.byref(self))
        for k, v in kw.items():
            if k not in dict(self._fields_):
                raise TypeError(f"unknown parameter {k}")
            setattr(self, k, v)

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class StepStats(ctypes.Structure):
    """Mirror of ch_step_stats."""
    _fields_ = [("iters", ctypes.c_int32 * 2), ("restarts", ctypes.c_int32), ("status", ctypes.c_int32),
                ("relres", ctypes.c_double * 2), ("mass", ctypes.c_double * 2), ("ms", ctypes.c_double),
                ("warm", ctypes.c_int32 * 2), ("reorth", ctypes.c_int32 * 2)]

    def as_dict(self):
        return {"iters": list(self.iters), "restarts": self.restarts, "status": self.status,
                "relres": list(self.relres), "mass": list(self.mass), "ms": self.ms, "warm": list(self.warm),
                "reorth": list(self.reorth)}


class ProfEntry(ctypes.Structure):
    """Mirror of ch_prof_entry."""
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("fmas", ctypes.c_double)]


_VP = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)
_I32P = ctypes.POINTER(ctypes.c_int32)

_SIGNATURES = {
    "ch_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "ch_last_error": (ctypes.c_char_p, []),
    "ch_params_default": (None, [ctypes.POINTER(Params)]),
    "ch_mesh": (ctypes.c_int, [ctypes.POINTER(Params), _VP, ctypes.POINTER(_VP)]),
    "ch_mesh_info": (ctypes.c_int, [_VP, _I64P, _I64P, _I64P, _I64P]),
    "ch_mesh_batch": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(Params), _VP, ctypes.POINTER(_VP)]),
    "ch_mesh_runs": (ctypes.c_int, [_VP, _I32P, _I32P]),
    "ch_mesh_copy": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "ch_mesh_destroy": (None, [_VP]),
    "ch_assemble": (ctypes.c_int, [_VP, ctypes.POINTER(Params), _VP, ctypes.POINTER(_VP)]),
    "ch_system_info": (ctypes.c_int, [_VP, _I64P, _I64P]),
    "ch_system_copy": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "ch_system_destroy": (None, [_VP]),
    "ch_loads": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "ch_rhs": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "ch_apply_A": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "ch_precond_setup": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(_VP)]),
    "ch_precond_info": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, _I32P, _I64P, _I64P]),
    "ch_precond_apply": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "ch_precond_tiles": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, _I32P, _I32P, _I32P]),
    "ch_precond_level": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, _I64P, _I64P, _I64P,
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                        _I32P, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "ch_vcycle": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP]),
    "ch_smooth": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP]),
    "ch_precond_destroy": (None, [_VP]),
    "ch_vcycle_noalloc": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int32, _VP, _VP, _VP]),
    "ch_mass_solve": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "ch_ws_fit_norm": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double), _VP]),
    "ch_morphology_project": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                             ctypes.c_int32, _VP, _VP, _VP, _VP]),
    "ch_state_create": (ctypes.c_int, [_VP, _VP, _VP, ctypes.POINTER(_VP)]),
    "ch_state_set": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "ch_state_init_seeded": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_uint64, _VP]),
    "ch_state_get": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "ch_state_init_seeded_batch": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                                  ctypes.c_double, ctypes.c_uint64, _VP]),
    "ch_state_run_stats": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(StepStats)]),
    "ch_step": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(StepStats)]),
    "ch_run": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, ctypes.POINTER(StepStats)]),
    "ch_state_destroy": (None, [_VP]),
    "ch_step_learned": (ctypes.c_int, [_VP, _VP, _VP, ctypes.POINTER(StepStats)]),
    "ch_state_save": (ctypes.c_int, [_VP, ctypes.c_char_p, _VP]),
    "ch_state_load": (ctypes.c_int, [_VP, ctypes.c_char_p, _VP]),
    "ch_step_guess": (ctypes.c_int, [_VP, _VP, _VP, ctypes.POINTER(StepStats)]),
    "ch_ws_nparams": (ctypes.c_int32, []),
    "ch_ws_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_VP)]),
    "ch_ws_destroy": (None, [_VP]),
    "ch_ws_set_engine": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "ch_ws_inject_mma_timeout": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "ch_ws_set_params": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float), _VP]),
    "ch_ws_get_params": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), _VP]),
    "ch_ws_set_norm": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float), _VP]),
    "ch_ws_predict": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "ch_ws_train_residual": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_int32, ctypes.c_float,
                                            ctypes.POINTER(ctypes.c_float), _VP]),
    "ch_ws_train_step": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                        ctypes.POINTER(ctypes.c_float), _VP]),
    "ch_profile_enable": (ctypes.c_int, [ctypes.c_int32]),
    "ch_profile_read": (ctypes.c_int, [ctypes.POINTER(ProfEntry), ctypes.c_int32, _I32P, ctypes.c_int32]),
}


def lib() -> ctypes.CDLL:
    """Load libch.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2204_03575_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGNATURES)


def _check(status: int, where: str):
    if status != OK:
        msg = lib().ch_last_error().decode(errors="replace")
        raise ChError(status, where, msg)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _f64(t, n=None, cols=None):
    if t.dtype != torch.float64 or not t.is_cuda:
        raise ValueError("expected a float64 CUDA tensor")
    t = t.contiguous()
    if n is not None and t.shape[0] != n:
        raise ValueError(f"expected {n} rows, got {t.shape[0]}")
    return t


class Mesh:
    def __init__(self, params: Params, stream=None, runs=None):
        """One box mesh from params, or (runs = list of Params) the disjoint union of run meshes."""
        self.params = params
        self._h = _VP()
        if runs is None:
            _check(lib().ch_mesh(ctypes.byref(params), _stream(stream), ctypes.byref(self._h)), "ch_mesh")
        else:
            arr = (Params * len(runs))(*runs)
            _check(lib().ch_mesh_batch(len(runs), arr, _stream(stream), ctypes.byref(self._h)), "ch_mesh_batch")
        nr = ctypes.c_int32()
        _check(lib().ch_mesh_runs(self._h, ctypes.byref(nr), None), "ch_mesh_runs")
        offs = (ctypes.c_int32 * (nr.value + 1))()
        _check(lib().ch_mesh_runs(self._h, None, offs), "ch_mesh_runs")
        self.nruns, self.run_offsets = nr.value, list(offs)
        n, e, fb, ft = (ctypes.c_int64() for _ in range(4))
        _check(lib().ch_mesh_info(self._h, ctypes.byref(n), ctypes.byref(e), ctypes.byref(fb),
                                  ctypes.byref(ft)), "ch_mesh_info")
        self.n_nodes, self.n_elems, self.n_bottom, self.n_top = n.value, e.value, fb.value, ft.value
        self.dim = params.dim

    def copy(self, stream=None):
        d = self.dim
        dev = torch.device("cuda")
        coords = torch.empty(self.n_nodes, d, dtype=torch.float64, device=dev)
        elems = torch.empty(self.n_elems, d + 1, dtype=torch.int32, device=dev)
        bot = torch.empty(self.n_bottom, d, dtype=torch.int32, device=dev)
        top = torch.empty(self.n_top, d, dtype=torch.int32, device=dev)
        _check(lib().ch_mesh_copy(self._h, _ptr(coords), _ptr(elems), _ptr(bot), _ptr(top), _stream(stream)),
               "ch_mesh_copy")
        return coords, elems, bot, top

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ch_mesh_destroy(self._h)
            self._h = None


class System:
    def __init__(self, mesh: Mesh, params: Params | None = None, stream=None):
        self.mesh = mesh  # keeps the borrowed mesh alive
        self.params = params if params is not None else mesh.params
        self._h = _VP()
        _check(lib().ch_assemble(mesh._h, ctypes.byref(self.params), _stream(stream), ctypes.byref(self._h)),
               "ch_assemble")
        n, nnz = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().ch_system_info(self._h, ctypes.byref(n), ctypes.byref(nnz)), "ch_system_info")
        self.n, self.nnz = n.value, nnz.value

    def csr(self, stream=None):
        dev = torch.device("cuda")
        rowptr = torch.empty(self.n + 1, dtype=torch.int32, device=dev)
        col = torch.empty(self.nnz, dtype=torch.int32, device=dev)
        vm, vk, vh = (torch.empty(self.nnz, dtype=torch.float64, device=dev) for _ in range(3))
        _check(lib().ch_system_copy(self._h, _ptr(rowptr), _ptr(col), _ptr(vm), _ptr(vk), _ptr(vh),
                                    _stream(stream)), "ch_system_copy")
        return rowptr, col, vm, vk, vh

    def loads(self, phi_p, phi_nfa, stream=None):
        pp, pn = _f64(phi_p, self.n), _f64(phi_nfa, self.n)
        out = [torch.empty(self.n, dtype=torch.float64, device=pp.device) for _ in range(4)]
        _check(lib().ch_loads(self._h, _ptr(pp), _ptr(pn), *[_ptr(o) for o in out], _stream(stream)), "ch_loads")
        return out

    def rhs(self, phi_p, phi_nfa, stream=None):
        pp, pn = _f64(phi_p, self.n), _f64(phi_nfa, self.n)
        b = torch.empty(self.n, 4, dtype=torch.float64, device=pp.device)
        _check(lib().ch_rhs(self._h, _ptr(pp), _ptr(pn), _ptr(b), _stream(stream)), "ch_rhs")
        return b

    def apply_A(self, x, stream=None):
        x = _f64(x, self.n)
        y = torch.empty_like(x)
        _check(lib().ch_apply_A(self._h, _ptr(x), _ptr(y), _stream(stream)), "ch_apply_A")
        return y

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ch_system_destroy(self._h)
            self._h = None


class Precond:
    def __init__(self, system: System, stream=None):
        self.system = system
        self._h = _VP()
        _check(lib().ch_precond_setup(system._h, _stream(stream), ctypes.byref(self._h)), "ch_precond_setup")

    def levels(self, which: int):
        nl = ctypes.c_int32()
        _check(lib().ch_precond_info(self._h, which, 0, ctypes.byref(nl), None, None), "ch_precond_info")
        out = []
        for l in range(nl.value):
            r, z = ctypes.c_int64(), ctypes.c_int64()
            _check(lib().ch_precond_info(self._h, which, l, None, ctypes.byref(r), ctypes.byref(z)),
                   "ch_precond_info")
            out.append((r.value, z.value))
        return out

    def tiles(self, which: int):
        """[(lanes per row for A, R, P) per level] chosen by the SpMV autotuner."""
        out = []
        for l in range(len(self.levels(which))):
            a, r, q = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
            _check(lib().ch_precond_tiles(self._h, which, l, ctypes.byref(a), ctypes.byref(r), ctypes.byref(q)),
                   "ch_precond_tiles")
            out.append((a.value, r.value, q.value))
        return out

    def level(self, which: int, l: int, stream=None):
        """Level l of hierarchy `which` (0: M, 1: H) as the V-cycle uses it: dict with the FP64
        CSR arrays of A (and P below the coarsest level) as device tensors, the Chebyshev interval
        (lo, hi) of D^-1 A and the smoothing degree."""
        rows, nnz, nnz_p = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        lo, hi, deg = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
        args = [ctypes.byref(rows), ctypes.byref(nnz), ctypes.byref(nnz_p), ctypes.byref(lo),
                ctypes.byref(hi), ctypes.byref(deg)]
        _check(lib().ch_precond_level(self._h, which, l, *args, None, None, None, None, None, None,
                                      _stream(stream)), "ch_precond_level")
        dev = torch.device("cuda")
        n, z, zp = rows.value, nnz.value, nnz_p.value
        A = (torch.empty(n + 1, dtype=torch.int32, device=dev), torch.empty(z, dtype=torch.int32, device=dev),
             torch.empty(z, dtype=torch.float64, device=dev))
        P = ((torch.empty(n + 1, dtype=torch.int32, device=dev), torch.empty(zp, dtype=torch.int32, device=dev),
              torch.empty(zp, dtype=torch.float64, device=dev)) if zp else (None, None, None))
        _check(lib().ch_precond_level(self._h, which, l, None, None, None, None, None, None,
                                      *[_ptr(t) if t is not None else None for t in A + P],
                                      _stream(stream)), "ch_precond_level")
        return {"rows": n, "A": A, "P": P if zp else None, "bounds": (lo.value, hi.value), "degree": deg.value}

    def apply(self, v, stream=None):
        v = _f64(v, self.system.n)
        w = torch.empty_like(v)
        _check(lib().ch_precond_apply(self._h, _ptr(v), _ptr(w), _stream(stream)), "ch_precond_apply")
        return w

    def vcycle(self, which: int, b, vcycles: int = 1, stream=None):
        b = _f64(b, self.system.n)
        x = torch.empty_like(b)
        _check(lib().ch_vcycle(self._h, which, vcycles, _ptr(b), _ptr(x), _stream(stream)), "ch_vcycle")
        return x

    def smooth(self, which: int, b, x, degree: int, passes: int = 1, stream=None):
        """ch_smooth: `passes` passes of the finest level's degree-`degree` Chebyshev smoother on
        M (which = 0) or H (which = 1), updating x (N x 2, fp64, on the device) in place."""
        b = _f64(b, self.system.n)
        if not (isinstance(x, torch.Tensor) and x.dtype == torch.float64 and x.is_cuda and x.is_contiguous()
                and tuple(x.shape) == (self.system.n, 2)):
            raise TypeError("x must be a contiguous N x 2 float64 CUDA tensor")
        _check(lib().ch_smooth(self._h, which, degree, passes, _ptr(b), _ptr(x), _stream(stream)), "ch_smooth")
        return x

    def mass_solve(self, b, stream=None):
        """ch_mass_solve: Algorithm 1's step 1 (M~^-1 b) on N x 2 right-hand sides."""
        b = _f64(b, self.system.n)
        x = torch.empty_like(b)
        _check(lib().ch_mass_solve(self._h, _ptr(b), _ptr(x), _stream(stream)), "ch_mass_solve")
        return x

    def vcycle_noalloc(self, which: int, b, vcycles: int = 1, stream=None):
        """ch_vcycle_noalloc: the same V-cycles with work space in the library's static array."""
        b = _f64(b, self.system.n)
        x = torch.empty_like(b)
        _check(lib().ch_vcycle_noalloc(self._h, which, vcycles, _ptr(b), _ptr(x), _stream(stream)),
               "ch_vcycle_noalloc")
        return x

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ch_precond_destroy(self._h)
            self._h = None


class State:
    def __init__(self, system: System, precond: Precond, stream=None):
        self.system, self.precond = system, precond
        self._h = _VP()
        _check(lib().ch_state_create(system._h, precond._h, _stream(stream), ctypes.byref(self._h)),
               "ch_state_create")

    def set(self, phi_p, phi_nfa, mu_p=None, mu_nfa=None, stream=None):
        n = self.system.n
        ts = [_f64(t, n) if t is not None else None for t in (phi_p, phi_nfa, mu_p, mu_nfa)]
        _check(lib().ch_state_set(self._h, *[_ptr(t) for t in ts], _stream(stream)), "ch_state_set")

    def init_seeded(self, phi_p0, phi_nfa0, noise=0.01, seed=0, stream=None):
        _check(lib().ch_state_init_seeded(self._h, phi_p0, phi_nfa0, noise, seed, _stream(stream)),
               "ch_state_init_seeded")

    def init_seeded_batch(self, phi_p0, phi_nfa0, noise=0.01, seed=0, stream=None):
        R = len(phi_p0)
        bp = (ctypes.c_double * R)(*phi_p0)
        bn = (ctypes.c_double * R)(*phi_nfa0)
        _check(lib().ch_state_init_seeded_batch(self._h, bp, bn, noise, seed, _stream(stream)),
               "ch_state_init_seeded_batch")

    def run_stats(self, run: int):
        st = StepStats()
        _check(lib().ch_state_run_stats(self._h, run, ctypes.byref(st)), "ch_state_run_stats")
        return st.as_dict()

    def get(self, stream=None):
        n = self.system.n
        out = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(5)]
        _check(lib().ch_state_get(self._h, *[_ptr(o) for o in out], _stream(stream)), "ch_state_get")
        return dict(zip(("phi_p", "phi_nfa", "phi_s", "mu_p", "mu_nfa"), out))

    def step(self, stream=None, check=True):
        st = StepStats()
        status = lib().ch_step(self._h, _stream(stream), ctypes.byref(st))
        if check:
            _check(status, "ch_step")
        return st.as_dict()

    def step_guess(self, guess, stream=None, check=True):
        """One step starting from `guess` (N x 4 fp64: phi_p, phi_nfa, mu_p, mu_nfa) where it beats
        the previous state's residual."""
        g = _f64(guess, self.system.n)
        st = StepStats()
        status = lib().ch_step_guess(self._h, _ptr(g), _stream(stream), ctypes.byref(st))
        if check:
            _check(status, "ch_step_guess")
        return st.as_dict()

    def step_learned(self, net, stream=None, check=True):
        """One step from the warm-start network's prediction (ch_step_learned)."""
        st = StepStats()
        status = lib().ch_step_learned(self._h, net._h, _stream(stream), ctypes.byref(st))
        if check:
            _check(status, "ch_step_learned")
        return st.as_dict()

    def save(self, path, stream=None):
        """Write the state to `path` (ch_state_save)."""
        _check(lib().ch_state_save(self._h, str(path).encode(), _stream(stream)), "ch_state_save")

    def load(self, path, stream=None):
        """Read a state written by save() (ch_state_load)."""
        _check(lib().ch_state_load(self._h, str(path).encode(), _stream(stream)), "ch_state_load")

    def state4(self, stream=None):
        """The state as one N x 4 fp64 tensor (phi_p, phi_nfa, mu_p, mu_nfa)."""
        g = self.get(stream)
        return torch.stack([g["phi_p"], g["phi_nfa"], g["mu_p"], g["mu_nfa"]], 1).contiguous()

    def run(self, nsteps: int, stream=None):
        arr = (StepStats * max(nsteps, 1))()
        _check(lib().ch_run(self._h, nsteps, _stream(stream), arr), "ch_run")
        return [arr[k].as_dict() for k in range(nsteps)]

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ch_state_destroy(self._h)
            self._h = None


def morphology_project(phi_p, phi_nfa, nx: int, ny: int, Lx: float, Ly: float, gx: int, gy: int,
                       threshold=None, stream=None):
    """ch_morphology_project (Section 5): the thresholded nodal image of an nx x ny 2D mesh
    classified onto the centres of a gx x gy grid by upward ray-crossing parity.  Returns device
    tensors (polymer uint8, mu_e, mu_h), each gy x gx."""
    n = (nx + 1) * (ny + 1)
    pp = _f64(phi_p, n)
    pn = _f64(phi_nfa, n) if phi_nfa is not None else None
    dev = pp.device
    polymer = torch.empty((gy, gx), dtype=torch.uint8, device=dev)
    mu_e = torch.empty((gy, gx), dtype=torch.float64, device=dev)
    mu_h = torch.empty((gy, gx), dtype=torch.float64, device=dev)
    use = 0 if threshold is None else 1
    _check(lib().ch_morphology_project(_ptr(pp), _ptr(pn) if pn is not None else None, nx, ny, Lx, Ly, use,
                                       float(threshold) if use else 0.0, gx, gy, _ptr(polymer), _ptr(mu_e),
                                       _ptr(mu_h), _stream(stream)), "ch_morphology_project")
    return polymer, mu_e, mu_h


def profile_enable(on: bool):
    """Turn per-launch CUDA-event timing on or off (launch counts are always kept)."""
    _check(lib().ch_profile_enable(1 if on else 0), "ch_profile_enable")


def profile_read(reset: bool = False):
    """{kernel name: {launches, ms, bytes, fmas}} accumulated since the last reset."""
    n = ctypes.c_int32()
    _check(lib().ch_profile_read(None, 0, ctypes.byref(n), 0), "ch_profile_read")
    arr = (ProfEntry * max(n.value, 1))()
    _check(lib().ch_profile_read(arr, n.value, ctypes.byref(n), 1 if reset else 0), "ch_profile_read")
    return {arr[i].name.decode(): {"launches": arr[i].launches, "ms": arr[i].ms, "bytes": arr[i].bytes,
                                   "fmas": arr[i].fmas} for i in range(n.value)}


class WarmStartNet:
    """The learned warm-start network (ch_ws_*): BF16 convolutional net on the nodal image."""

    def __init__(self, H: int, W: int, max_batch: int = 8):
        self.H, self.W, self.max_batch = H, W, max_batch
        self._h = _VP()
        _check(lib().ch_ws_create(H, W, max_batch, ctypes.byref(self._h)), "ch_ws_create")
        self.nparams = lib().ch_ws_nparams()

    def set_engine(self, engine: int):
        """ch_ws_set_engine: 0 mma.sync, 1 tcgen05 convolutions."""
        _check(lib().ch_ws_set_engine(self._h, engine), "ch_ws_set_engine")

    def inject_mma_timeout(self, on: bool):
        """ch_ws_inject_mma_timeout: the tcgen05 convolutions withhold their MMAs (a test of the
        bounded wait's failure path)."""
        _check(lib().ch_ws_inject_mma_timeout(self._h, 1 if on else 0), "ch_ws_inject_mma_timeout")

    def set_params(self, params, stream=None):
        import numpy as np
        a = np.ascontiguousarray(params, dtype=np.float32)
        assert a.size == self.nparams
        _check(lib().ch_ws_set_params(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _stream(stream)),
               "ch_ws_set_params")

    def get_params(self, stream=None):
        import numpy as np
        p = np.empty(self.nparams, np.float32)
        g = np.empty(self.nparams, np.float32)
        _check(lib().ch_ws_get_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                      g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _stream(stream)),
               "ch_ws_get_params")
        return p, g

    def set_norm(self, mean, inv_std, out_scale, stream=None):
        """mean, inv_std: 8 values (the 4 fields, then their change); out_scale: 4."""
        import numpy as np
        a = np.ascontiguousarray(np.concatenate([mean, inv_std, out_scale]), dtype=np.float32)
        assert a.size == 20
        _check(lib().ch_ws_set_norm(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _stream(stream)),
               "ch_ws_set_norm")

    def fit_norm(self, X, stream=None):
        """ch_ws_fit_norm on the states of a training set (S x N x 4 CUDA tensor, float64 or
        float32): sets the network's normalisation and returns (mean[8], inv_std[8], out_scale[4])."""
        import numpy as np
        if X.dtype not in (torch.float64, torch.float32) or not X.is_cuda:
            raise ValueError("X must be a float64 or float32 CUDA tensor")
        X = X.contiguous()
        out = (ctypes.c_double * 20)()
        _check(lib().ch_ws_fit_norm(self._h, _ptr(X), X.shape[0], 1 if X.dtype == torch.float32 else 0, out,
                                    _stream(stream)), "ch_ws_fit_norm")
        a = np.array(out[:])
        return a[:8], a[8:16], a[16:20]

    def predict(self, state4, prev4, prev2_4, stream=None):
        """The next state predicted from s_k, s_{k-1}, s_{k-2} (N x 4 fp64 CUDA each)."""
        s, q, q2 = _f64(state4), _f64(prev4), _f64(prev2_4)
        pred = torch.empty_like(s)
        _check(lib().ch_ws_predict(self._h, _ptr(s), _ptr(q), _ptr(q2), _ptr(pred), _stream(stream)),
               "ch_ws_predict")
        return pred

    def train_residual(self, system, x, q, q2, lr: float, precond=None, stream=None):
        """One step against the residual of the time step (x = s_k, q = s_{k-1}, q2 = s_{k-2}:
        B x N x 4 fp64 CUDA), in the norm of `precond` if given; returns the loss
        (mean ln(|r|^2 / |r_linear extrapolation|^2))."""
        for a in (x, q, q2):
            if a.dtype != torch.float64 or not a.is_contiguous() or not a.is_cuda:
                raise ValueError("expected contiguous float64 CUDA tensors")
        loss = ctypes.c_float()
        pc = precond._h if precond is not None else None
        _check(lib().ch_ws_train_residual(self._h, system._h, pc, _ptr(x), _ptr(q), _ptr(q2), x.shape[0], lr,
                                          ctypes.byref(loss), _stream(stream)), "ch_ws_train_residual")
        return loss.value

    def train_step(self, x, q, q2, n, lr: float, lap: float = 0.0, stream=None):
        """One step on states x, their predecessors q, q2 and successors n (B x N x 4 fp32 CUDA);
        `lap` weighs the grid-Laplacian term of the state-space loss."""
        for a in (x, q, q2, n):
            if a.dtype != torch.float32 or not a.is_contiguous() or not a.is_cuda:
                raise ValueError("expected contiguous float32 CUDA tensors")
        loss = ctypes.c_float()
        _check(lib().ch_ws_train_step(self._h, _ptr(x), _ptr(q), _ptr(q2), _ptr(n), x.shape[0], lap, lr,
                                      ctypes.byref(loss), _stream(stream)), "ch_ws_train_step")
        return loss.value

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ch_ws_destroy(self._h)
            self._h = None
