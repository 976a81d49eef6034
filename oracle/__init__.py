"""FP64 CPU oracle for the HELIOS radiative-equilibrium hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It wraps the
plain C restatement of the paper's method in ``helios_ref.c`` (double
precision, no FMA contraction, OpenMP over wavelength bins) with ctypes.  It
shares no code with the CUDA library.

Parity status of each function (pins live in tests/test_oracle_*.py):
  E1, 2E3, exact diffusivity   pinned: scipy.special.exp1 / expn, quadrature, limits
  Gauss-Legendre               pinned: numpy leggauss, polynomial exactness
  Planck per bin               pinned: Stefan-Boltzmann law on a fine grid
  grid, table lookup           pinned: brute force on tiny tables, closed forms
  two-stream layer             pinned: matrix-exponential solution of the two-stream ODE
  exact layer                  pinned: direct angular quadrature of the formal solution
  column sweeps                pinned: isothermal cavity / semi-infinite closed forms,
                               conservative scattering, exact-vs-D=2 refinement
  temperature step             pinned: converged net flux = sigma T_int^4; grey two-band profile
  oscillation control          pinned: hand-made sign sequences with the multipliers written out
                               from the rule of Sect. 2.2.4 (monotonic, alternating, period-4,
                               cap, no change before six signs)
  RE trajectory                parity unpinned (the path of a heuristic iteration; its fixed point
                               is pinned)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_helios_ref.so")
_lib = None

SIGMA_SB = 5.670374419e-5
CONVERGED, UPDATED, NOT_CONVERGED, NONFINITE, OUT_OF_RANGE = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "helios_ref.c")
    hdr = os.path.join(_HERE, "helios_ref.h")
    newest = max(os.path.getmtime(src), os.path.getmtime(hdr))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared",
                               "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    from . import opcount
    opcount.build(force)
    return _SO


class RefAtm(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("L", ctypes.c_int), ("G", ctypes.c_int),
                ("P_top_bar", ctypes.c_double), ("P_bot_bar", ctypes.c_double),
                ("grav", ctypes.c_double), ("T_irr", ctypes.c_double), ("T_int", ctypes.c_double),
                ("T_star", ctypes.c_double),
                ("nu_edges", ctypes.c_void_p), ("omega0", ctypes.c_void_p), ("g0", ctypes.c_void_p),
                ("nP", ctypes.c_int), ("nT", ctypes.c_int), ("L_table", ctypes.c_int),
                ("log10P0", ctypes.c_double), ("dlog10P", ctypes.c_double),
                ("T0", ctypes.c_double), ("dT", ctypes.c_double),
                ("kappa", ctypes.c_void_p), ("grey", ctypes.c_int), ("rayleigh", ctypes.c_int)]


class RefParams(ctypes.Structure):
    _fields_ = [("D", ctypes.c_double), ("dtau_iso", ctypes.c_double), ("w0_pure", ctypes.c_double),
                ("tol", ctypes.c_double), ("fpre_num", ctypes.c_double), ("fpre_exp", ctypes.c_double),
                ("osc_down", ctypes.c_double), ("osc_up", ctypes.c_double), ("mult_max", ctypes.c_double),
                ("T_floor", ctypes.c_double), ("mbar_mp", ctypes.c_double), ("n_dof", ctypes.c_double),
                ("n_scat", ctypes.c_int), ("max_iter", ctypes.c_int), ("printed_gradient", ctypes.c_int),
                ("tabulate", ctypes.c_int)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_SO)
    d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
    P = ctypes.POINTER
    lib.ref_default_params.argtypes = [P(RefParams)]
    lib.ref_E1.restype = d; lib.ref_E1.argtypes = [d]
    lib.ref_trans_exact.restype = d; lib.ref_trans_exact.argtypes = [d]
    lib.ref_tab_one_minus_trans.restype = d; lib.ref_tab_one_minus_trans.argtypes = [d]
    lib.ref_tab_planck_bin.restype = d; lib.ref_tab_planck_bin.argtypes = [d, d, d]
    lib.ref_diffusivity_exact.restype = d; lib.ref_diffusivity_exact.argtypes = [d]
    lib.ref_gauss_legendre.argtypes = [i, vp, vp]
    lib.ref_planck_bin.restype = d; lib.ref_planck_bin.argtypes = [d, d, d]
    lib.ref_grid.argtypes = [P(RefAtm), vp, vp, vp, vp]
    lib.ref_point_temperatures.argtypes = [i, vp, vp]
    lib.ref_table_coord.argtypes = [d, d, d, i, P(ctypes.c_int), P(ctypes.c_double)]
    lib.ref_interp_opacity.argtypes = [P(RefAtm), vp, vp, vp, vp]
    lib.ref_boundary_spectra.argtypes = [P(RefAtm), vp, vp]
    lib.ref_layer_twostream.argtypes = [d, d, d, d, d, d, d, P(RefParams), P(ctypes.c_double), P(ctypes.c_double)]
    lib.ref_layer_exact.argtypes = [d, d, d, d, d, d, P(ctypes.c_double), P(ctypes.c_double)]
    lib.ref_flux_sweep.restype = i
    lib.ref_flux_sweep.argtypes = [P(RefAtm), P(RefParams), vp, i, i, vp, i, vp, vp, vp, vp, vp]
    lib.ref_flux_direct.restype = i
    lib.ref_flux_direct.argtypes = [P(RefAtm), P(RefParams), vp, i, vp, vp, vp]
    lib.ref_layer_affine.restype = None
    lib.ref_layer_affine.argtypes = [d, d, d, d, d, P(RefParams), vp]
    lib.ref_rayleigh_kappa.restype = d
    lib.ref_rayleigh_kappa.argtypes = [d, d, d]
    lib.ref_flux_sweep_iso.restype = i
    lib.ref_flux_sweep_iso.argtypes = [P(RefAtm), P(RefParams), vp, i, vp, vp, vp]
    lib.ref_temp_update.restype = i
    lib.ref_temp_update.argtypes = [P(RefAtm), P(RefParams), vp, vp, vp, vp, vp, vp, vp, vp]
    lib.ref_solve_re.restype = i
    lib.ref_solve_re.argtypes = [P(RefAtm), P(RefParams), vp, vp, vp, vp, vp, vp, vp]
    lib.ref_passes.restype = i
    lib.ref_passes.argtypes = [P(RefAtm), P(RefParams)]
    lib.ref_set_threads.restype = None
    lib.ref_set_threads.argtypes = [i]
    lib.ref_max_threads.restype = i
    lib.ref_max_threads.argtypes = []
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def params(**overrides) -> RefParams:
    p = RefParams()
    _load().ref_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


class Atm:
    """An oracle view of one synthetic atmosphere (keeps its arrays alive)."""

    def __init__(self, atm, table, grey: bool = False, kappa64=None, rayleigh: bool = False):
        self.src = atm
        self.nu = np.ascontiguousarray(atm.nu_edges, dtype=np.float64)
        self.w0 = np.ascontiguousarray(atm.omega0, dtype=np.float64)
        self.g0 = np.ascontiguousarray(atm.g0, dtype=np.float64)
        k = table.kappa_for_oracle() if kappa64 is None else kappa64
        self.kappa = np.ascontiguousarray(k, dtype=np.float64)
        s = RefAtm()
        s.n, s.L, s.G = atm.n_layers, atm.n_bins, table.G
        s.P_top_bar, s.P_bot_bar = atm.P_top_bar, atm.P_bot_bar
        s.grav, s.T_irr, s.T_int, s.T_star = atm.grav, atm.T_irr, atm.T_int, atm.T_star
        s.nu_edges, s.omega0, s.g0 = self.nu.ctypes.data, self.w0.ctypes.data, self.g0.ctypes.data
        s.nP, s.nT, s.L_table = table.nP, table.nT, table.L
        s.log10P0, s.dlog10P, s.T0, s.dT = table.log10P0, table.dlog10P, table.T0, table.dT
        s.kappa = self.kappa.ctypes.data
        s.grey = 1 if grey else 0
        s.rayleigh = 1 if rayleigh else 0
        self.s = s
        self.n, self.L, self.G = atm.n_layers, atm.n_bins, table.G

    @classmethod
    def from_workload(cls, wl, a: int = 0, **kw):
        """Atmosphere a of a workload; a species mixture (eq. 34) gets its mixed table."""
        atm = wl.atms[a]
        species = getattr(atm, "species", None)
        if species and "kappa64" not in kw:
            kw["kappa64"] = mixed_kappa(wl.tables, species)
        return cls(atm, wl.tables[atm.table_id], grey=wl.grey, **kw)


def mixed_kappa(tables, species) -> np.ndarray:
    """Eq. (34): the opacity of a mixture is sum_j X_j kappa_j over its species.  The species'
    tables share one (P, T) grid and bilinear interpolation is linear, so the oracle mixes the
    tables element-wise (float32 values widened to float64) and interpolates the result."""
    k = np.zeros(tables[0].kappa32.shape)
    for t, w in species:
        k += float(w) * tables[t].kappa32.astype(np.float64)
    return k


# ---------------------------------------------------------------------------
# thin functional wrappers
# ---------------------------------------------------------------------------
def E1(x: float) -> float:
    return _load().ref_E1(x)


def trans_exact(x: float) -> float:
    return _load().ref_trans_exact(x)


# the tables of Sect. 2.6 (ref_params.tabulate): nodes of 1 - e^-x and of the Planck function
TAB_X0, TAB_NX, TAB_DT, TAB_NT = -8.05, 102, 10.0, 601


def tab_one_minus_trans(x: float) -> float:
    """1 - e^-x from the table of Sect. 2.6 (linear in x between 0.1-dex nodes)."""
    return _load().ref_tab_one_minus_trans(x)


def tab_planck_bin(nu_lo: float, nu_hi: float, T: float) -> float:
    """The Planck intensity of a bin from the table of Sect. 2.6 (linear in T between 10 K nodes)."""
    return _load().ref_tab_planck_bin(nu_lo, nu_hi, T)


def diffusivity_exact(x: float) -> float:
    return _load().ref_diffusivity_exact(x)


def gauss_legendre(G: int):
    x = np.empty(G); w = np.empty(G)
    _load().ref_gauss_legendre(G, x.ctypes.data, w.ctypes.data)
    return x, w


def planck_bin(nu_lo: float, nu_hi: float, T: float) -> float:
    return _load().ref_planck_bin(nu_lo, nu_hi, T)


def grid(atm: Atm):
    n = atm.n
    lp = np.empty(2 * n + 1); P = np.empty(2 * n + 1); dm = np.empty(2 * n); Pl = np.empty(n)
    _load().ref_grid(ctypes.byref(atm.s), lp.ctypes.data, P.ctypes.data, dm.ctypes.data, Pl.ctypes.data)
    return lp, P, dm, Pl


def point_temperatures(T: np.ndarray) -> np.ndarray:
    T = np.ascontiguousarray(T, dtype=np.float64)
    out = np.empty(2 * len(T) + 1)
    _load().ref_point_temperatures(len(T), T.ctypes.data, out.ctypes.data)
    return out


def table_coord(x: float, x0: float, dx: float, nx: int):
    i = ctypes.c_int(); w = ctypes.c_double()
    _load().ref_table_coord(x, x0, dx, nx, ctypes.byref(i), ctypes.byref(w))
    return i.value, w.value


def interp_opacity(atm: Atm, T: np.ndarray, want_kappa: bool = True):
    n = atm.n; np_ = 2 * n + 1
    T = np.ascontiguousarray(T, dtype=np.float64)
    kap = np.empty((np_, atm.L, atm.G)) if want_kappa else None
    idx = np.empty((np_, 2), dtype=np.int32)
    w = np.empty((np_, 2))
    _load().ref_interp_opacity(ctypes.byref(atm.s), T.ctypes.data, _ptr(kap), idx.ctypes.data, w.ctypes.data)
    return kap, idx, w


def boundary_spectra(atm: Atm):
    toa = np.empty(atm.L); bint = np.empty(atm.L)
    _load().ref_boundary_spectra(ctypes.byref(atm.s), toa.ctypes.data, bint.ctypes.data)
    return toa, bint


def layer_twostream(F1up, F2dn, B1, B2, dtau, w0, g0, p: RefParams = None):
    p = p or params()
    u = ctypes.c_double(); dn = ctypes.c_double()
    _load().ref_layer_twostream(F1up, F2dn, B1, B2, dtau, w0, g0, ctypes.byref(p), ctypes.byref(u), ctypes.byref(dn))
    return u.value, dn.value


def layer_exact(F1up, F2dn, B1, B2, dtau, dtau_iso=1e-4):
    u = ctypes.c_double(); dn = ctypes.c_double()
    _load().ref_layer_exact(F1up, F2dn, B1, B2, dtau, dtau_iso, ctypes.byref(u), ctypes.byref(dn))
    return u.value, dn.value


def passes(atm: Atm, p: RefParams = None) -> int:
    p = p or params()
    return _load().ref_passes(ctypes.byref(atm.s), ctypes.byref(p))


def flux_sweep(atm: Atm, T: np.ndarray, n_passes: int = None, p: RefParams = None, exact: bool = False,
               warm: np.ndarray = None, warm_valid: bool = False, spectra: bool = False):
    """One flux evaluation.  Returns dict(Fup, Fdn, toa[, up_spec, dn_spec])."""
    p = p or params()
    if n_passes is None:
        n_passes = passes(atm, p)
    n = atm.n; np_ = 2 * n + 1
    T = np.ascontiguousarray(T, dtype=np.float64)
    Fu = np.empty(n + 1); Fd = np.empty(n + 1); toa = np.empty(atm.L)
    us = np.empty((atm.L, np_)) if spectra else None
    ds = np.empty((atm.L, np_)) if spectra else None
    rc = _load().ref_flux_sweep(ctypes.byref(atm.s), ctypes.byref(p), T.ctypes.data, n_passes, 1 if exact else 0,
                                _ptr(warm), 1 if warm_valid else 0, Fu.ctypes.data, Fd.ctypes.data,
                                toa.ctypes.data, _ptr(us), _ptr(ds))
    out = {"Fup": Fu, "Fdn": Fd, "toa": toa, "rc": rc}
    if spectra:
        out["up_spec"] = us; out["dn_spec"] = ds
    return out


def flux_sweep_iso(atm: Atm, T: np.ndarray, n_passes: int = None, p: RefParams = None):
    """One flux evaluation on the isothermal-layer grid (ref_flux_sweep_iso).
    Returns dict(Fup, Fdn, toa)."""
    p = p or params()
    if n_passes is None:
        n_passes = passes(atm, p)
    n = atm.n
    T = np.ascontiguousarray(T, dtype=np.float64)
    Fu = np.empty(n + 1); Fd = np.empty(n + 1); toa = np.empty(atm.L)
    rc = _load().ref_flux_sweep_iso(ctypes.byref(atm.s), ctypes.byref(p), T.ctypes.data, n_passes,
                                    Fu.ctypes.data, Fd.ctypes.data, toa.ctypes.data)
    return {"Fup": Fu, "Fdn": Fd, "toa": toa, "rc": rc}


def flux_direct(atm: Atm, T: np.ndarray, iso: bool = False, p: RefParams = None):
    """Exact solution of the coupled two-stream column equations (ref_flux_direct): the limit of
    infinitely many scattering passes.  Returns dict(Fup, Fdn, toa)."""
    p = p or params()
    n = atm.n
    T = np.ascontiguousarray(T, dtype=np.float64)
    Fu = np.empty(n + 1); Fd = np.empty(n + 1); toa = np.empty(atm.L)
    rc = _load().ref_flux_direct(ctypes.byref(atm.s), ctypes.byref(p), T.ctypes.data, 1 if iso else 0,
                                 Fu.ctypes.data, Fd.ctypes.data, toa.ctypes.data)
    return {"Fup": Fu, "Fdn": Fd, "toa": toa, "rc": rc}


def rayleigh_kappa(nu_lo, nu_hi, mbar_mp=2.4):
    """H2 Rayleigh opacity (cm^2/g) of the bin [nu_lo, nu_hi] cm^-1 (eqs. 16-17)."""
    return _load().ref_rayleigh_kappa(nu_lo, nu_hi, mbar_mp)


def layer_affine(B1, B2, dtau, w0, g0, p: RefParams = None):
    p = p or params()
    c = np.empty(6)
    _load().ref_layer_affine(B1, B2, dtau, w0, g0, ctypes.byref(p), c.ctypes.data)
    return c


class State:
    """Iteration state of one atmosphere: T, timestep multipliers, sign history, warm fluxes."""

    def __init__(self, atm: Atm, T0: np.ndarray):
        n = atm.n
        self.T = np.array(T0, dtype=np.float64)
        self.mult = np.ones(n)
        self.hist = np.zeros(n, dtype=np.int32)
        self.nhist = np.zeros(n, dtype=np.int32)
        self.warm = np.zeros(atm.L * atm.G * (2 * n + 1))

    def copy(self):
        s = object.__new__(State)
        s.T, s.mult, s.hist, s.nhist, s.warm = (self.T.copy(), self.mult.copy(), self.hist.copy(),
                                                 self.nhist.copy(), self.warm.copy())
        return s


def temp_update(atm: Atm, st: State, Fup: np.ndarray, Fdn: np.ndarray, p: RefParams = None):
    p = p or params()
    metric = ctypes.c_double()
    dT = np.empty(atm.n)
    Fup = np.ascontiguousarray(Fup, dtype=np.float64); Fdn = np.ascontiguousarray(Fdn, dtype=np.float64)
    rc = _load().ref_temp_update(ctypes.byref(atm.s), ctypes.byref(p), Fup.ctypes.data, Fdn.ctypes.data,
                                 st.T.ctypes.data, st.mult.ctypes.data, st.hist.ctypes.data,
                                 st.nhist.ctypes.data, ctypes.byref(metric), dT.ctypes.data)
    return rc, metric.value, dT


def set_threads(n: int) -> None:
    """Host threads of the oracle's OpenMP loops over bins (timing on 1 core and on all)."""
    _load().ref_set_threads(int(n))


def max_threads() -> int:
    return int(_load().ref_max_threads())


def solve_re(atm: Atm, st: State, p: RefParams = None):
    """Iterate to radiative equilibrium in place; returns (status, iterations, final metric)."""
    p = p or params()
    iters = ctypes.c_int(); metric = ctypes.c_double()
    rc = _load().ref_solve_re(ctypes.byref(atm.s), ctypes.byref(p), st.T.ctypes.data, st.mult.ctypes.data,
                              st.hist.ctypes.data, st.nhist.ctypes.data, st.warm.ctypes.data,
                              ctypes.byref(iters), ctypes.byref(metric))
    return rc, iters.value, metric.value
