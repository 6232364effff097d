"""Python binding of the C ABI in ``include/lbm.h`` (argument marshalling only).

Every step of the method runs in the CUDA library ``_build/liblbm_gb300.so``;
this module only converts parameter dictionaries to ``lbm_params``, hands
PyTorch device memory and streams to the library, and wraps results as
tensors or numpy arrays.  There is no CPU fallback: if the library is missing
or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "_build" / "liblbm_gb300.so"

LBM_OK = 0
ERRORS = {
    -1: "LBM_ERR_ARG", -2: "LBM_ERR_STABILITY", -3: "LBM_ERR_OOM", -4: "LBM_ERR_CUDA",
    -5: "LBM_ERR_UNSTABLE", -6: "LBM_ERR_TIMEOUT", -7: "LBM_ERR_STATE", -8: "LBM_ERR_TOO_LARGE",
}
F64, F32, F16, BF16 = 0, 1, 2, 3
FIELDS = ("T_f", "T_s", "f_l", "u_x", "u_y", "rho", "H_f")


class LbmError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({strerror(code)})")


class LbmParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("thermal_q", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("flow", ctypes.c_int32),
        ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
        ("wall_kind", ctypes.c_int32 * 4), ("wall_T", ctypes.c_double * 4),
        ("porosity", ctypes.c_double), ("Ra", ctypes.c_double), ("Pr", ctypes.c_double),
        ("Da", ctypes.c_double), ("Ste", ctypes.c_double), ("cond_ratio", ctypes.c_double),
        ("Nu_i", ctypes.c_double), ("J", ctypes.c_double), ("F_phi", ctypes.c_double),
        ("sigma_hat", ctypes.c_double), ("dp_over_L", ctypes.c_double), ("k_f", ctypes.c_double),
        ("cfref_over_cpl", ctypes.c_double), ("cmref_over_cpm", ctypes.c_double),
        ("T_hot", ctypes.c_double), ("T_cold", ctypes.c_double), ("T_init", ctypes.c_double),
        ("T_ref0", ctypes.c_double), ("T_solidus", ctypes.c_double), ("T_liquidus", ctypes.c_double),
        ("L_char", ctypes.c_double), ("varpi", ctypes.c_double),
        ("thermal_collision", ctypes.c_int32), ("solid_scheme", ctypes.c_int32), ("zeta_e", ctypes.c_double),
        ("ks_over_kl", ctypes.c_double), ("cps_over_cpl", ctypes.c_double),
    ]


class LbmDerived(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "nu_f", "nu_e", "gbeta", "K", "k_m", "rho_m", "L_a", "d_p", "h_v",
        "alpha_f", "alpha_fref", "alpha_mref", "c_fref", "c_mref", "csT2",
        "H_fs", "H_fl", "l0", "l1", "exchange_rate")] + [
        ("s", ctypes.c_double * 9), ("zeta", ctypes.c_double * 9), ("eta", ctypes.c_double * 9),
        ("H_wall", ctypes.c_double * 4), ("k_s", ctypes.c_double), ("c_ps", ctypes.c_double),
        ("zeta_a_solid", ctypes.c_double), ("F_phi", ctypes.c_double)]


class RequestResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("steps", ctypes.c_int64), ("nodes", ctypes.c_int64),
                ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double), ("finish_s", ctypes.c_double),
                ("melt_frac", ctypes.c_double), ("nu_hot", ctypes.c_double), ("enthalpy", ctypes.c_double),
                ("mass", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


def lib() -> ctypes.CDLL:
    """Loads the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run paper_1701_00702_gb300.build.build())")
        L = ctypes.CDLL(str(LIB_PATH))
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        pp = ctypes.POINTER(LbmParams)
        dp = ctypes.POINTER(LbmDerived)
        L.lbm_params_default.argtypes = [pp]
        L.lbm_params_default.restype = None
        L.lbm_derive.argtypes = [pp, dp]
        L.lbm_derive.restype = ctypes.c_int
        L.lbm_state_bytes.argtypes = [pp]
        L.lbm_state_bytes.restype = i64
        L.lbm_history_bytes.argtypes = [pp]
        L.lbm_history_bytes.restype = i64
        L.lbm_create.argtypes = [pp, vp, ctypes.POINTER(vp)]
        L.lbm_create.restype = ctypes.c_int
        L.lbm_create_ex.argtypes = [pp, vp, ALLOC_FN, FREE_FN, vp, ctypes.POINTER(vp)]
        L.lbm_create_ex.restype = ctypes.c_int
        L.lbm_step.argtypes = [vp, i64]
        L.lbm_step.restype = ctypes.c_int
        L.lbm_set_step_form.argtypes = [vp, i32]
        L.lbm_set_step_form.restype = ctypes.c_int
        L.lbm_step_form_for.argtypes = [pp, i32, ctypes.POINTER(i32)]
        L.lbm_step_form_for.restype = ctypes.c_int
        L.lbm_fields.argtypes = [vp, i32, ctypes.POINTER(vp), i32]
        L.lbm_fields.restype = ctypes.c_int
        L.lbm_diag.argtypes = [vp] + [ctypes.POINTER(ctypes.c_double)] * 4
        L.lbm_diag.restype = ctypes.c_int
        L.lbm_get_state.argtypes = [vp, vp, vp, vp, vp, vp, i32]
        L.lbm_get_state.restype = ctypes.c_int
        L.lbm_set_state.argtypes = [vp, vp, vp, vp, vp, vp, i32]
        L.lbm_set_state.restype = ctypes.c_int
        L.lbm_checkpoint_bytes.argtypes = [vp]
        L.lbm_checkpoint_bytes.restype = i64
        L.lbm_save.argtypes = [vp, vp, i32]
        L.lbm_save.restype = ctypes.c_int
        L.lbm_load.argtypes = [vp, vp, i32]
        L.lbm_load.restype = ctypes.c_int
        L.lbm_status.argtypes = [vp]
        L.lbm_status.restype = ctypes.c_int
        L.lbm_steps_done.argtypes = [vp]
        L.lbm_steps_done.restype = i64
        L.lbm_describe.argtypes = [vp, pp, dp]
        L.lbm_describe.restype = ctypes.c_int
        L.lbm_destroy.argtypes = [vp]
        L.lbm_destroy.restype = ctypes.c_int
        L.lbm_strerror.argtypes = [ctypes.c_int]
        L.lbm_strerror.restype = ctypes.c_char_p
        L.lbm_batch_create.argtypes = [ctypes.POINTER(vp), i32, i32, vp, ctypes.POINTER(vp)]
        L.lbm_batch_create.restype = ctypes.c_int
        L.lbm_batch_step.argtypes = [vp, i64]
        L.lbm_batch_step.restype = ctypes.c_int
        L.lbm_batch_configure.argtypes = [vp, i32, i32]
        L.lbm_batch_configure.restype = ctypes.c_int
        L.lbm_batch_set_block.argtypes = [vp, i32, i32, i32]
        L.lbm_batch_set_block.restype = ctypes.c_int
        L.lbm_batch_get_block.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.lbm_batch_get_block.restype = ctypes.c_int
        L.lbm_batch_info.argtypes = [vp] + [ctypes.POINTER(i32)] * 4 + [ctypes.POINTER(ctypes.c_double)]
        L.lbm_batch_info.restype = ctypes.c_int
        L.lbm_batch_destroy.argtypes = [vp]
        L.lbm_batch_destroy.restype = ctypes.c_int
        L.lbm_server_create.argtypes = [i64, i32, i32, i32, i32, i32, i32, vp, ALLOC_FN, FREE_FN, vp,
                                        ctypes.POINTER(vp)]
        L.lbm_server_create.restype = ctypes.c_int
        L.lbm_server_configure.argtypes = [vp, i32, i32]
        L.lbm_server_configure.restype = ctypes.c_int
        L.lbm_server_submit.argtypes = [vp, pp, i64, ctypes.POINTER(i64)]
        L.lbm_server_submit.restype = ctypes.c_int
        L.lbm_server_tick.argtypes = [vp] + [ctypes.POINTER(i32)] * 3
        L.lbm_server_tick.restype = ctypes.c_int
        L.lbm_server_results.argtypes = [vp, ctypes.POINTER(RequestResult), i32, ctypes.POINTER(i32)]
        L.lbm_server_results.restype = ctypes.c_int
        L.lbm_server_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.lbm_server_stats.restype = ctypes.c_int
        L.lbm_server_destroy.argtypes = [vp]
        L.lbm_server_destroy.restype = ctypes.c_int
        L.lbm_diag_fields_noalloc.argtypes = [pp, vp, vp, vp, vp, vp, vp, vp]
        L.lbm_diag_fields_noalloc.restype = ctypes.c_int
        _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().lbm_strerror(int(code)).decode()
    except Exception:
        return "?"


def _check(rc: int, what: str):
    if rc != LBM_OK:
        raise LbmError(rc, what)


def to_struct(p: dict) -> LbmParams:
    s = LbmParams()
    lib().lbm_params_default(ctypes.byref(s))
    for name, _ in LbmParams._fields_:
        if name not in p:
            continue
        v = p[name]
        if name in ("wall_kind", "wall_T"):
            arr = getattr(s, name)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(s, name, v)
    return s


def default_params() -> dict:
    s = LbmParams()
    lib().lbm_params_default(ctypes.byref(s))
    return {n: (list(getattr(s, n)) if n in ("wall_kind", "wall_T") else getattr(s, n)) for n, _ in LbmParams._fields_}


def _derived_dict(d: LbmDerived) -> dict:
    out = {}
    for name, _ in LbmDerived._fields_:
        v = getattr(d, name)
        out[name] = list(v) if name in ("s", "zeta", "eta", "H_wall") else float(v)
    return out


def derive(p: dict) -> dict:
    """Lattice constants computed by the library's own parameter map (no GPU needed)."""
    d = LbmDerived()
    _check(lib().lbm_derive(ctypes.byref(to_struct(p)), ctypes.byref(d)), "lbm_derive")
    return _derived_dict(d)


def step_form_for(p: dict, form: int = 0) -> int:
    """The step form (1: one node per thread, 2: node pairs) a run with
    parameters p takes when set to `form` (lbm_step_form_for; no GPU needed)."""
    used = ctypes.c_int32()
    _check(lib().lbm_step_form_for(ctypes.byref(to_struct(p)), int(form), ctypes.byref(used)), "lbm_step_form_for")
    return int(used.value)


def state_bytes(p: dict) -> int:
    return int(lib().lbm_state_bytes(ctypes.byref(to_struct(p))))


def history_bytes(p: dict) -> int:
    """Device bytes of one exchange-history array (lbm_history_bytes)."""
    return int(lib().lbm_history_bytes(ctypes.byref(to_struct(p))))


def diag_fields_noalloc(params: dict, fields: dict, out, stream=None) -> None:
    """Enqueues the allocation-free diagnostics of caller-owned device fields
    (torch tensors keyed T_f, T_s, f_l, rho, H_f) into ``out`` (a CUDA float64
    tensor of 4 elements): melt fraction, hot-wall Nusselt number, enthalpy,
    mass.  Only pointers are passed; the library allocates nothing."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    ptrs = [ctypes.c_void_p(fields[k].data_ptr()) for k in ("T_f", "T_s", "f_l", "rho", "H_f")]
    rc = lib().lbm_diag_fields_noalloc(ctypes.byref(to_struct(params)), *ptrs, ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(s.cuda_stream))
    _check(rc, "lbm_diag_fields_noalloc")


class TorchAllocator:
    """Device memory for the library from PyTorch's caching allocator."""

    def __init__(self, device):
        import torch
        self._torch = torch
        self.device = device
        self.live = {}
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, _ctx):
        try:
            t = self._torch.empty(int(nbytes) + 256, dtype=self._torch.uint8, device=self.device)
        except Exception:
            return None
        ptr = t.data_ptr()
        aligned = (ptr + 255) // 256 * 256
        self.live[aligned] = t
        return aligned

    def _free(self, ptr, _ctx):
        self.live.pop(int(ptr), None)


class Solver:
    """One run of the fused three-lattice solver on the current CUDA device."""

    def __init__(self, params: dict, stream=None, device=None, use_torch_alloc: bool = True):
        import torch
        self._torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA GPU is required (the solver has no CPU path)")
        self.params = dict(params)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._struct = to_struct(self.params)
        self.dtype = torch.float64 if self._struct.precision == F64 else torch.float32
        self.np_dtype = np.float64 if self._struct.precision == F64 else np.float32
        self.nx, self.ny, self.qt = self._struct.nx, self._struct.ny, self._struct.thermal_q
        self.flow = bool(self._struct.flow)
        self._h = ctypes.c_void_p()
        self._alloc = TorchAllocator(self.device) if use_torch_alloc else None
        with torch.cuda.device(self.device):
            if self._alloc is not None:
                rc = lib().lbm_create_ex(ctypes.byref(self._struct), ctypes.c_void_p(self.stream.cuda_stream),
                                         self._alloc.alloc_cb, self._alloc.free_cb, None, ctypes.byref(self._h))
            else:
                rc = lib().lbm_create(ctypes.byref(self._struct), ctypes.c_void_p(self.stream.cuda_stream),
                                      ctypes.byref(self._h))
        _check(rc, "lbm_create")

    # -- stepping -----------------------------------------------------------
    def step(self, n: int) -> "Solver":
        _check(lib().lbm_step(self._h, int(n)), "lbm_step")
        return self

    def set_step_form(self, form: int) -> "Solver":
        """0: automatic, 1: one node per thread, 2: node pairs, 3: two time steps
        per launch (lbm_set_step_form)."""
        _check(lib().lbm_set_step_form(self._h, int(form)), "lbm_set_step_form")
        return self

    @property
    def steps(self) -> int:
        return int(lib().lbm_steps_done(self._h))

    def status(self) -> int:
        return int(lib().lbm_status(self._h))

    # -- outputs ------------------------------------------------------------
    def fields(self, names=FIELDS, device: bool = True) -> dict:
        """Fields at the current time level, [ny, nx] each: torch tensors on the
        device (device=True) or numpy arrays copied to the host."""
        torch = self._torch
        mask = 0
        ptrs = (ctypes.c_void_p * 7)()
        out = {}
        for name in names:
            i = FIELDS.index(name)
            mask |= 1 << i
            if device:
                t = torch.empty((self.ny, self.nx), dtype=self.dtype, device=self.device)
                ptrs[i] = t.data_ptr()
            else:
                t = np.empty((self.ny, self.nx), dtype=self.np_dtype)
                ptrs[i] = t.ctypes.data
            out[name] = t
        _check(lib().lbm_fields(self._h, mask, ptrs, 1 if device else 0), "lbm_fields")
        return out

    def fields_into(self, out: dict):
        """Writes the named fields into caller-owned host arrays (C-contiguous,
        [ny, nx], the run's dtype), e.g. views of pinned buffers."""
        mask = 0
        ptrs = (ctypes.c_void_p * 7)()
        for name, arr in out.items():
            if arr.dtype != self.np_dtype or arr.shape != (self.ny, self.nx) or not arr.flags["C_CONTIGUOUS"]:
                raise ValueError(f"bad host buffer for {name}")
            i = FIELDS.index(name)
            mask |= 1 << i
            ptrs[i] = arr.ctypes.data
        _check(lib().lbm_fields(self._h, mask, ptrs, 0), "lbm_fields")

    def diag(self) -> dict:
        v = [ctypes.c_double() for _ in range(4)]
        _check(lib().lbm_diag(self._h, *[ctypes.byref(x) for x in v]), "lbm_diag")
        return dict(melt_frac=v[0].value, nu_hot=v[1].value, enthalpy=v[2].value, mass=v[3].value)

    def derived(self) -> dict:
        d = LbmDerived()
        _check(lib().lbm_describe(self._h, None, ctypes.byref(d)), "lbm_describe")
        return _derived_dict(d)

    # -- raw state ----------------------------------------------------------
    def get_state(self, with_lo: bool = False):
        """(f, g, h, dT) as numpy arrays [q][ny][nx] / [ny][nx] (f is None when the
        flow lattice is off).  f holds the deviations f_i - w_i from the rest
        equilibrium, the library's storage form; g and h are the populations.
        with_lo=True appends the low part of the FP32 PCM rest population
        (None for FP64 runs), so that the tuple restores the state bit for bit."""
        f = np.empty((9, self.ny, self.nx), self.np_dtype) if self.flow else None
        g = np.empty((self.qt, self.ny, self.nx), self.np_dtype)
        h = np.empty((self.qt, self.ny, self.nx), self.np_dtype)
        dT = np.empty((self.ny, self.nx), self.np_dtype)
        lo = np.empty((self.ny, self.nx), self.np_dtype) if self._struct.precision == F32 else None
        _check(lib().lbm_get_state(self._h, None if f is None else f.ctypes.data, g.ctypes.data, h.ctypes.data,
                                   dT.ctypes.data, None if lo is None else lo.ctypes.data, 0), "lbm_get_state")
        return (f, g, h, dT, lo) if with_lo else (f, g, h, dT)

    def set_state(self, f, g, h, dT, g0_lo=None):
        conv = [None if a is None else np.ascontiguousarray(a, dtype=self.np_dtype) for a in (f, g, h, dT, g0_lo)]
        if self.flow and conv[0] is None:
            raise ValueError("flow populations are required when the flow lattice is on")
        ptrs = [None if a is None else a.ctypes.data for a in conv]
        _check(lib().lbm_set_state(self._h, *ptrs, 0), "lbm_set_state")

    def save(self) -> np.ndarray:
        """Raw checkpoint (header + current state copy + history) as host bytes."""
        buf = np.empty(int(lib().lbm_checkpoint_bytes(self._h)), np.uint8)
        _check(lib().lbm_save(self._h, buf.ctypes.data, 0), "lbm_save")
        return buf

    def load(self, buf: np.ndarray):
        """Restores a checkpoint written by save() of a run with the same layout."""
        buf = np.ascontiguousarray(buf, np.uint8)
        _check(lib().lbm_load(self._h, buf.ctypes.data, 0), "lbm_load")

    def close(self):
        if self._h:
            lib().lbm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Runs advanced together from CUDA graphs (lbm_batch_*)."""

    MAPS = ("one block per tile", "persistent contiguous chunks", "persistent grid stride",
            "single-run kernel chains", "grouped launches", "grouped launches, two steps each")

    def __init__(self, runs, autotune: bool = True, stream=None):
        import torch
        self.runs = list(runs)
        self.stream = stream if stream is not None else self.runs[0].stream
        arr = (ctypes.c_void_p * len(self.runs))(*[r._h.value for r in self.runs])
        self._b = ctypes.c_void_p()
        with torch.cuda.device(self.runs[0].device):
            rc = lib().lbm_batch_create(arr, len(self.runs), 1 if autotune else 0,
                                        ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self._b))
        _check(rc, "lbm_batch_create")

    def step(self, n: int) -> "Batch":
        _check(lib().lbm_batch_step(self._b, int(n)), "lbm_batch_step")
        return self

    def configure(self, width_cap: int, mapping: int) -> "Batch":
        """Forces a tile-width cap (32, 64, 128, 256) and a map: 0-2 tile lists,
        3 single-run kernel chains, 4 grouped launches, 5 grouped launches of
        two steps each (runs with flow in FP32/FP16/BF16) (lbm_batch_configure)."""
        _check(lib().lbm_batch_configure(self._b, int(width_cap), int(mapping)), "lbm_batch_configure")
        return self

    def set_block(self, run: int, block_x: int, block_y: int) -> "Batch":
        """Block shape of one run under map 3 (128x2, 64x4, 32x8, 256x1, 128x1, 64x2, 32x4, 64x1, 32x2)."""
        _check(lib().lbm_batch_set_block(self._b, int(run), int(block_x), int(block_y)), "lbm_batch_set_block")
        return self

    def blocks(self) -> list:
        """Block shape (x, y) of every run under map 3."""
        out = []
        for r in range(len(self.runs)):
            bx, by = ctypes.c_int32(), ctypes.c_int32()
            _check(lib().lbm_batch_get_block(self._b, r, ctypes.byref(bx), ctypes.byref(by)), "lbm_batch_get_block")
            out.append((bx.value, by.value))
        return out

    def info(self) -> dict:
        v = [ctypes.c_int32() for _ in range(4)]
        us = ctypes.c_double()
        _check(lib().lbm_batch_info(self._b, *[ctypes.byref(x) for x in v], ctypes.byref(us)), "lbm_batch_info")
        return dict(n_tiles=v[0].value, width_cap=v[1].value, mapping=self.MAPS[v[2].value], grid=v[3].value,
                    tuned_us_per_step=us.value)

    def close(self):
        if self._b:
            lib().lbm_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching serving engine (lbm_server_*); `mapping` is the
    batch map of every tick (4: grouped launches, the default; 5: grouped
    launches of two steps each, whose runs also hold a second exchange
    history within the budget)."""

    def __init__(self, hbm_budget_bytes: int, max_active: int = 64, batched: bool = True, quantum: int = 256,
                 precision: int = F16, thermal_q: int = 5, flow: int = 1, stream=None, device=None,
                 width_cap: int = 128, mapping: int = 4):
        import torch
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._alloc = TorchAllocator(self.device)
        self._s = ctypes.c_void_p()
        _check(lib().lbm_server_create(int(hbm_budget_bytes), int(max_active), 1 if batched else 0, int(quantum),
                                       int(precision), int(thermal_q), int(flow),
                                       ctypes.c_void_p(self.stream.cuda_stream), self._alloc.alloc_cb,
                                       self._alloc.free_cb, None, ctypes.byref(self._s)), "lbm_server_create")
        _check(lib().lbm_server_configure(self._s, int(width_cap), int(mapping)), "lbm_server_configure")

    def submit(self, params: dict, nsteps: int) -> int:
        rid = ctypes.c_int64()
        _check(lib().lbm_server_submit(self._s, ctypes.byref(to_struct(params)), int(nsteps), ctypes.byref(rid)),
               "lbm_server_submit")
        return rid.value

    def tick(self):
        a, q, d = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().lbm_server_tick(self._s, ctypes.byref(a), ctypes.byref(q), ctypes.byref(d)), "lbm_server_tick")
        return a.value, q.value, d.value

    def results(self) -> list:
        buf = (RequestResult * 256)()
        n = ctypes.c_int32()
        out = []
        while True:
            _check(lib().lbm_server_results(self._s, buf, 256, ctypes.byref(n)), "lbm_server_results")
            out += [{k: getattr(buf[i], k) for k, _ in RequestResult._fields_ if k != "reserved"}
                    for i in range(n.value)]
            if n.value < 256:
                return out

    def stats(self) -> dict:
        ns, used, peak = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        busy, el = ctypes.c_double(), ctypes.c_double()
        _check(lib().lbm_server_stats(self._s, ctypes.byref(ns), ctypes.byref(busy), ctypes.byref(el),
                                      ctypes.byref(used), ctypes.byref(peak)), "lbm_server_stats")
        return dict(node_steps=ns.value, busy_s=busy.value, elapsed_s=el.value, used_bytes=used.value,
                    peak_used_bytes=peak.value)

    def replay(self, trace, time_scale: float = 1.0, idle_sleep: float = 0.001) -> list:
        """Submits each request of ``trace`` (dicts with arrival_s, params, steps)
        when its arrival time has passed on the host clock and ticks until all
        have finished.  Returns the result records."""
        import time
        pending = sorted(trace, key=lambda r: r["arrival_s"])
        t0 = time.perf_counter()
        i, results = 0, []
        while len(results) < len(pending):
            now = (time.perf_counter() - t0) / time_scale
            while i < len(pending) and pending[i]["arrival_s"] <= now:
                self.submit(pending[i]["params"], pending[i]["steps"])
                i += 1
            active, queued, _ = self.tick()
            results += self.results()
            if active == 0 and queued == 0 and i < len(pending):
                time.sleep(min(idle_sleep, max(0.0, pending[i]["arrival_s"] * time_scale - (time.perf_counter() - t0))))
        return results

    def close(self):
        if self._s:
            lib().lbm_server_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
