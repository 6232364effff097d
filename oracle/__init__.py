"""Plain FP64 CPU oracle of the enthalpy-based MRT-LB phase-change step.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its Python binding) never imports this package.

Contents
--------
* ``lattice_config``: the map from the paper's non-dimensional groups
  (Eq. 54, Sec. IV) to lattice-unit constants and relaxation rates
  (Sec. III C, Eq. 53, Eq. A19, Eq. 51, App. B).  Written here in Python,
  independently of the CUDA host runtime's own C++ map.
* ``Oracle``: a ctypes front end of ``lbm_oracle.c`` (the literal FP64
  stepper) holding the state arrays in numpy.
* ``diagnostics``: melt fraction, hot-wall Nusselt number, total enthalpy and
  mass computed from the oracle's fields with numpy.

Parity pins: the functions here are checked against closed forms, printed
values and invariants in ``tests/test_oracle_*.py``.  The square-cavity
melting run (natural convection with phase change) has no closed form; only
its invariants pin it, so its full-field values are "parity unpinned" beyond
those invariants, and GPU-vs-oracle agreement is the check there.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "liboracle.so"
_SRC = _HERE / "lbm_oracle.c"

WALL_DIRICHLET = 0
WALL_ADIABATIC = 1


def build(force: bool = False, src: Path | None = None, out: Path | None = None) -> Path:
    """Compile the C oracle with gcc (IEEE arithmetic, no FMA contraction).

    ``src``/``out`` compile another copy of the source (the pin tests plant
    mistakes in a copy this way, to show that a pin catches them)."""
    src = _SRC if src is None else Path(src)
    out = _LIB_PATH if out is None else Path(out)
    out.parent.mkdir(parents=True, exist_ok=True)
    if force or not out.exists() or out.stat().st_mtime < src.stat().st_mtime:
        tmp = out.with_suffix(f".{os.getpid()}.tmp")
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", str(src), "-o", str(tmp), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


class OrcCfg(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("qt", ctypes.c_int), ("flow", ctypes.c_int),
        ("periodic_x", ctypes.c_int), ("periodic_y", ctypes.c_int),
        ("wall_kind", ctypes.c_int * 4), ("wall_T", ctypes.c_double * 4),
        ("phi", ctypes.c_double), ("nu_f", ctypes.c_double), ("K", ctypes.c_double),
        ("F_phi", ctypes.c_double), ("gbeta", ctypes.c_double), ("T0", ctypes.c_double),
        ("rho_l", ctypes.c_double), ("rho_m", ctypes.c_double), ("c_pl", ctypes.c_double),
        ("c_ps", ctypes.c_double), ("c_pm", ctypes.c_double), ("c_fref", ctypes.c_double),
        ("c_mref", ctypes.c_double), ("L_a", ctypes.c_double), ("h_v", ctypes.c_double),
        ("T_fs", ctypes.c_double), ("T_fl", ctypes.c_double), ("varpi", ctypes.c_double),
        ("s", ctypes.c_double * 9), ("zeta", ctypes.c_double * 9), ("eta", ctypes.c_double * 9),
        ("solid_scheme", ctypes.c_int),
        ("phase_k", ctypes.c_int), ("zeta_role", ctypes.c_int * 9),
        ("k_l", ctypes.c_double), ("k_s", ctypes.c_double), ("csT2", ctypes.c_double),
    ]


_lib = None


def _bind(L):
    """Declare the argument types of a loaded oracle library."""
    dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
    cp = ctypes.POINTER(OrcCfg)
    L.orc_init.argtypes = [cp, ctypes.c_double, dp, dp, dp, dp]
    L.orc_step.argtypes = [cp, dp, dp, dp, dp, dp, dp, dp]
    L.orc_fields.argtypes = [cp, dp, dp, dp] + [dp] * 7
    L.orc_lattice.argtypes = [np.ctypeslib.ndpointer(dtype=np.int32), np.ctypeslib.ndpointer(dtype=np.int32), dp]
    L.orc_matrices.argtypes = [ctypes.c_int, dp, dp]
    for name in ("orc_f_eq", "orc_m_eq"):
        getattr(L, name).argtypes = [cp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
    L.orc_force_moments.argtypes = [cp] + [ctypes.c_double] * 5 + [dp]
    for name in ("orc_g_eq", "orc_ng_eq"):
        getattr(L, name).argtypes = [cp] + [ctypes.c_double] * 4 + [dp]
    for name in ("orc_h_eq", "orc_nh_eq"):
        getattr(L, name).argtypes = [cp, ctypes.c_double, dp]
    for name in ("orc_T_of_H", "orc_fl_of_H", "orc_H_of_T"):
        getattr(L, name).argtypes = [cp, ctypes.c_double]
        getattr(L, name).restype = ctypes.c_double
    L.orc_velocity.argtypes = [cp] + [ctypes.c_double] * 4 + [dp]
    ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
    L.orc_step_nodes.argtypes = [cp, dp, dp, dp, dp, ip, ip, ctypes.c_int, dp, dp, dp, dp]
    L.orc_set_threads.argtypes = [ctypes.c_int]
    L.orc_threads.restype = ctypes.c_int
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(str(build())))
    return _lib


def load(path) -> ctypes.CDLL:
    """Load another compiled copy of the oracle (see ``build``)."""
    return _bind(ctypes.CDLL(str(path)))


# ---------------------------------------------------------------------------
# Parameter map: Eq. 54 with delta_x = delta_t = c = 1, rho_l = 1 and
# c_pl = c_pm = 1 (Sec. IV); c_ps = c_pl and k_s = k_l unless the Eq. 9
# variant sets them apart.  Input keys follow the C ABI's lbm_params.
# ---------------------------------------------------------------------------

def lattice_config(p: dict) -> dict:
    """Lattice-unit constants and relaxation rates for one run."""
    qt = int(p["thermal_q"])
    L = float(p["L_char"])
    dT = float(p["T_hot"]) - float(p["T_cold"])
    c_pl = c_pm = 1.0
    c_ps = float(p.get("cps_over_cpl", 1.0)) * c_pl       # Eq. 9: solid specific heat
    rho_l = 1.0
    k_f = float(p["k_f"])                                # the liquid conductivity k_l of Eq. 9
    k_s = float(p.get("ks_over_kl", 1.0)) * k_f
    phi = float(p["porosity"])
    alpha_f = k_f / (rho_l * c_pl)                       # alpha_f = k_f/(rho c_p)_f
    nu_f = float(p["Pr"]) * alpha_f                      # Pr = nu_f/alpha_f
    nu_e = float(p["J"]) * nu_f                          # J = nu_e/nu_f
    gbeta = float(p["Ra"]) * nu_f * alpha_f / (dT * L ** 3)   # Ra
    K = float(p["Da"]) * L * L                           # Da = K/L^2
    k_m = float(p["cond_ratio"]) * k_f                   # lambda = k_m/k_f
    rho_m = float(p["sigma_hat"]) * rho_l * c_pl / c_pm  # sigma_hat = (rho c_p)_m/(rho c_p)_f
    L_a = c_pl * dT / float(p["Ste"])                    # St = c_pl dT/L_a
    d_p = float(p["dp_over_L"]) * L
    h_v = float(p["Nu_i"]) * k_f / (d_p * d_p)           # H_v = h_v d_p^2/k_f
    c_fref = float(p["cfref_over_cpl"]) * c_pl
    c_mref = float(p["cmref_over_cpm"]) * c_pm
    alpha_fref = k_f / (rho_l * c_fref)                  # Eq. A19
    alpha_mref = k_m / (rho_m * c_mref)                  # after Eq. 51
    varpi = float(p["varpi"])
    cs2 = 1.0 / 3.0
    csT2 = cs2 if qt == 9 else varpi / 2.0               # App. B: c_sT^2 = varpi c^2/2
    s_v = 1.0 / (0.5 + nu_e / cs2)                       # Sec. III C
    zeta_a = 1.0 / (0.5 + alpha_fref / csT2)
    eta_a = 1.0 / (0.5 + alpha_mref / csT2)
    zeta_e = 2.0 - zeta_a                                # Eq. 53
    if float(p.get("zeta_e", 0.0)) > 0.0:                # Sec. V D: an explicit zeta_e
        zeta_e = float(p["zeta_e"])
    s = [1.0, 1.1, 1.1, 1.0, 1.2, 1.0, 1.2, s_v, s_v]    # Eq. 16 with Sec. III C's rates
    e_role = 0 if float(p.get("zeta_e", 0.0)) > 0.0 else 2   # rate roles for the Eq. 9 variant
    if qt == 9:
        zeta = [1.0, zeta_e, zeta_e, zeta_a, zeta_a, zeta_a, zeta_a, 1.2, 1.2]
        eta = [1.0, 1.1, 1.1, eta_a, eta_a, eta_a, eta_a, 1.2, 1.2]
        role = [0, e_role, e_role, 1, 1, 1, 1, 0, 0]
    else:
        zeta = [1.0, zeta_a, zeta_a, zeta_e, 1.2] + [0.0] * 4
        eta = [1.0, eta_a, eta_a, 1.1, 1.2] + [0.0] * 4
        role = [0, 1, 1, e_role, 0] + [0] * 4
    if int(p.get("thermal_collision", 0)) == 1:          # Sec. V A: BGK, one rate per lattice
        zeta = [zeta_a] * qt + [0.0] * (9 - qt)
        eta = [eta_a] * qt + [0.0] * (9 - qt)
        role = [1] * qt + [0] * (9 - qt)
    F_phi = float(p["F_phi"])
    if F_phi < 0.0:                                      # Eq. 4 (Ergun): 1.75 / sqrt(150 phi^3)
        F_phi = 1.75 / math.sqrt(150.0 * phi ** 3)
    return dict(
        nx=int(p["nx"]), ny=int(p["ny"]), qt=qt, flow=int(p["flow"]),
        periodic_x=int(p["periodic_x"]), periodic_y=int(p["periodic_y"]),
        wall_kind=[int(v) for v in p["wall_kind"]], wall_T=[float(v) for v in p["wall_T"]],
        phi=phi, nu_f=nu_f, nu_e=nu_e, K=K, F_phi=F_phi, gbeta=gbeta, T0=float(p["T_ref0"]),
        rho_l=rho_l, rho_m=rho_m, c_pl=c_pl, c_ps=c_ps, c_pm=c_pm, c_fref=c_fref, c_mref=c_mref,
        L_a=L_a, h_v=h_v, T_fs=float(p["T_solidus"]), T_fl=float(p["T_liquidus"]), varpi=varpi,
        s=s, zeta=zeta, eta=eta, solid_scheme=int(p.get("solid_scheme", 0)),
        phase_k=int(k_s != k_f), zeta_role=role, k_l=k_f, k_s=k_s,
        # informational
        alpha_f=alpha_f, alpha_fref=alpha_fref, alpha_mref=alpha_mref, k_f=k_f, k_m=k_m,
        d_p=d_p, s_v=s_v, zeta_a=zeta_a, zeta_e=zeta_e, eta_a=eta_a, csT2=csT2,
        T_init=float(p["T_init"]), L=L, dT=dT,
    )


def make_cfg(lc: dict) -> OrcCfg:
    c = OrcCfg()
    for name, _ in OrcCfg._fields_:
        v = lc[name]
        if name in ("wall_kind", "wall_T", "s", "zeta", "eta", "zeta_role"):
            arr = getattr(c, name)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(c, name, v)
    return c


class Oracle:
    """One run of the FP64 oracle: state arrays [q][ny][nx] in numpy."""

    def __init__(self, params: dict, threads: int | None = None, library=None):
        self.params = dict(params)
        self.lc = lattice_config(params)
        self.cfg = make_cfg(self.lc)
        self._L = lib() if library is None else library
        if threads is not None:
            self._L.orc_set_threads(int(threads))
        nx, ny, qt = self.lc["nx"], self.lc["ny"], self.lc["qt"]
        shape9, shapeq = (9, ny, nx), (qt, ny, nx)
        self.F = [np.zeros(shape9), np.zeros(shape9)]
        self.G = [np.zeros(shapeq), np.zeros(shapeq)]
        self.H = [np.zeros(shapeq), np.zeros(shapeq)]
        self.dT = np.zeros((ny, nx))
        self.cur = 0
        self.steps = 0
        rc = self._L.orc_init(ctypes.byref(self.cfg), self.lc["T_init"], self.F[0], self.G[0], self.H[0], self.dT)
        if rc != 0:
            raise ValueError("oracle rejected the configuration")

    @property
    def threads(self) -> int:
        return int(self._L.orc_threads())

    def set_state(self, F, G, H, dT):
        c = self.cur
        if self.lc["flow"]:
            self.F[c][...] = F
        self.G[c][...] = G
        self.H[c][...] = H
        self.dT[...] = dT

    def state(self):
        c = self.cur
        return self.F[c].copy(), self.G[c].copy(), self.H[c].copy(), self.dT.copy()

    def run(self, nsteps: int):
        for _ in range(int(nsteps)):
            a, b = self.cur, 1 - self.cur
            rc = self._L.orc_step(ctypes.byref(self.cfg), self.F[a], self.G[a], self.H[a], self.dT,
                                  self.F[b], self.G[b], self.H[b])
            if rc != 0:
                raise RuntimeError("oracle step failed")
            self.cur = b
            self.steps += 1
        return self

    def step_nodes(self, xs, ys):
        """Post-collision values of one step at the listed nodes only (state unchanged).
        Returns (f [n,9] or None, g [n,qt], h [n,qt], dT [n])."""
        xs = np.ascontiguousarray(xs, dtype=np.int32)
        ys = np.ascontiguousarray(ys, dtype=np.int32)
        n, qt = xs.size, self.lc["qt"]
        fo, go, ho, dTo = np.zeros((n, 9)), np.zeros((n, qt)), np.zeros((n, qt)), np.zeros(n)
        c = self.cur
        rc = self._L.orc_step_nodes(ctypes.byref(self.cfg), self.F[c], self.G[c], self.H[c], self.dT,
                                    xs, ys, n, fo, go, ho, dTo)
        if rc != 0:
            raise RuntimeError("oracle step_nodes failed")
        return (fo if self.lc["flow"] else None), go, ho, dTo

    def fields(self) -> dict:
        nx, ny = self.lc["nx"], self.lc["ny"]
        out = {k: np.zeros((ny, nx)) for k in ("T_f", "T_m", "f_l", "u_x", "u_y", "rho", "H_f")}
        c = self.cur
        rc = self._L.orc_fields(ctypes.byref(self.cfg), self.F[c], self.G[c], self.H[c],
                                out["T_f"], out["T_m"], out["f_l"], out["u_x"], out["u_y"],
                                out["rho"], out["H_f"])
        if rc != 0:
            raise RuntimeError("oracle fields failed")
        return out

    def diag(self) -> dict:
        return diagnostics(self.fields(), self.lc)


def diagnostics(fields: dict, lc: dict) -> dict:
    """Melt fraction (mean f_l over all nodes, Fig. 9), hot-wall Nusselt number,
    total enthalpy and mass.

    The paper defines no Nusselt number; the reading used throughout is the
    left-wall heat flux of both phases, second-order one-sided difference,
    scaled by L/(k_e dT) with k_e = phi k_f + (1 - phi) k_m (Eq. 10), k_f the
    liquid conductivity.  Under the Eq. 9 variant the PCM flux takes the
    conductivity of each wall node's own liquid fraction."""
    Tf, Tm = fields["T_f"], fields["T_m"]
    phi = lc["phi"]
    k_e = phi * lc["k_f"] + (1.0 - phi) * lc["k_m"]
    nu = float("nan")
    if Tf.shape[1] >= 3:
        dTf = (3.0 * Tf[:, 0] - 4.0 * Tf[:, 1] + Tf[:, 2]) / 2.0   # -dT/dx at x = 0
        dTm = (3.0 * Tm[:, 0] - 4.0 * Tm[:, 1] + Tm[:, 2]) / 2.0
        k_wall = lc["k_f"]
        if lc["phase_k"]:
            fl0 = fields["f_l"][:, 0]
            k_wall = fl0 * lc["k_l"] + (1.0 - fl0) * lc["k_s"]     # Eq. 9
        q = phi * k_wall * dTf + (1.0 - phi) * lc["k_m"] * dTm
        nu = float(lc["L"] / (k_e * lc["dT"]) * q.mean())
    enthalpy = float(np.sum(phi * lc["rho_l"] * fields["H_f"] + (1.0 - phi) * lc["rho_m"] * lc["c_pm"] * Tm))
    return dict(melt_frac=float(fields["f_l"].mean()), nu_hot=nu, enthalpy=enthalpy,
                mass=float(fields["rho"].sum()))


def _cfg_only(params: dict) -> OrcCfg:
    return make_cfg(lattice_config(params))


# Single-formula helpers used by the pin tests --------------------------------

def lattice():
    ex = np.zeros(9, np.int32)
    ey = np.zeros(9, np.int32)
    w = np.zeros(9)
    lib().orc_lattice(ex, ey, w)
    return ex, ey, w


def matrices(q: int):
    M = np.zeros(q * q)
    Mi = np.zeros(q * q)
    if lib().orc_matrices(int(q), M, Mi) != 0:
        raise ValueError(q)
    return M.reshape(q, q), Mi.reshape(q, q)


def f_eq(params, rho, ux, uy):
    out = np.zeros(9)
    lib().orc_f_eq(ctypes.byref(_cfg_only(params)), rho, ux, uy, out)
    return out


def m_eq(params, rho, ux, uy):
    out = np.zeros(9)
    lib().orc_m_eq(ctypes.byref(_cfg_only(params)), rho, ux, uy, out)
    return out


def force_moments(params, rho, ux, uy, Fx, Fy):
    out = np.zeros(9)
    lib().orc_force_moments(ctypes.byref(_cfg_only(params)), rho, ux, uy, Fx, Fy, out)
    return out


def g_eq(params, H, T, ux, uy):
    c = _cfg_only(params)
    out = np.zeros(9)
    lib().orc_g_eq(ctypes.byref(c), H, T, ux, uy, out)
    return out[: c.qt]


def ng_eq(params, H, T, ux, uy):
    c = _cfg_only(params)
    out = np.zeros(9)
    lib().orc_ng_eq(ctypes.byref(c), H, T, ux, uy, out)
    return out[: c.qt]


def h_eq(params, Tm):
    c = _cfg_only(params)
    out = np.zeros(9)
    lib().orc_h_eq(ctypes.byref(c), Tm, out)
    return out[: c.qt]


def nh_eq(params, Tm):
    c = _cfg_only(params)
    out = np.zeros(9)
    lib().orc_nh_eq(ctypes.byref(c), Tm, out)
    return out[: c.qt]


def T_of_H(params, H):
    return lib().orc_T_of_H(ctypes.byref(_cfg_only(params)), H)


def fl_of_H(params, H):
    return lib().orc_fl_of_H(ctypes.byref(_cfg_only(params)), H)


def H_of_T(params, T):
    return lib().orc_H_of_T(ctypes.byref(_cfg_only(params)), T)


def velocity(params, rho, jx, jy, Gy):
    out = np.zeros(2)
    lib().orc_velocity(ctypes.byref(_cfg_only(params)), rho, jx, jy, Gy, out)
    return out

