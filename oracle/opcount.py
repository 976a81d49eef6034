"""Algorithmic operation counts of one flux evaluation, from the op-counting build of the oracle
(opcount.cpp: the oracle's own source with a counting floating-point type).  TEST AND
MEASUREMENT INFRASTRUCTURE ONLY: the benchmark's roofline figures divide these counts by the
measured time of the CUDA sweep; nothing on the product path calls it.

Every operation is counted as the oracle's formulas perform it, split by whether its result
depends on the radiation field (the fluxes; flagged from T_irr, T_int and the warm start) or not
(the layer coefficients, Planck values, opacities).  The oracle recomputes a sublayer's
coefficients inside every call of its layer solution and computes both outgoing streams in both
sweeps; the method needs them once per evaluation and one stream per sweep.  Two evaluations with
1 and 2 passes separate what a pass repeats from what an evaluation does once:
  per-pass coefficient work (oracle) = U2 - U1 = two layer calls' worth -> once: (U2 - U1) / 2
  per-pass flux work (oracle)        = F2 - F1 = two calls x both streams -> per pass: (F2 - F1) / 2
  algorithmic(K) = [U1 - (U2 - U1)] + (U2 - U1)/2 + [F1 - (F2 - F1)] + K (F2 - F1)/2
with the set-up that does not scale with the work (Gauss-Legendre nodes, the pressure grid, the
boundary spectra, the table coordinates of the points) counted by calling those functions alone
and taken out.

Instruction estimates (FP32 pipe, SFU): a quotient is a reciprocal (SFU) and a multiply; an
exponential, square root or logarithm is one SFU operation and one multiply (argument scaling);
a power is a logarithm and an exponential.  Multiplies and additions pair into fused
multiply-adds as far as their counts allow: FP32 instructions >= max(adds, multiplies) + the
multiplies above.  That lower bound is what a roofline of the FP32 pipe divides by.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_helios_opcount.so")
_lib = None

CATS = ("add", "mul", "div", "exp", "sqrt", "log", "pow")
CN = np.dtype({"names": ["v", "f"], "formats": ["f8", "u1"], "offsets": [0, 8], "itemsize": 16})


class _CNum(ctypes.Structure):
    _fields_ = [("v", ctypes.c_double), ("f", ctypes.c_ubyte), ("pad", ctypes.c_ubyte * 7)]


def _cn(x, flag=0):
    c = _CNum()
    c.v, c.f = float(x), flag
    return c


class _AtmC(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("L", ctypes.c_int), ("G", ctypes.c_int),
                ("P_top_bar", _CNum), ("P_bot_bar", _CNum), ("grav", _CNum), ("T_irr", _CNum),
                ("T_int", _CNum), ("T_star", _CNum),
                ("nu_edges", ctypes.c_void_p), ("omega0", ctypes.c_void_p), ("g0", ctypes.c_void_p),
                ("nP", ctypes.c_int), ("nT", ctypes.c_int), ("L_table", ctypes.c_int),
                ("log10P0", _CNum), ("dlog10P", _CNum), ("T0", _CNum), ("dT", _CNum),
                ("kappa", ctypes.c_void_p), ("grey", ctypes.c_int), ("rayleigh", ctypes.c_int)]


class _ParamsC(ctypes.Structure):
    _fields_ = [(k, _CNum) for k in ("D", "dtau_iso", "w0_pure", "tol", "fpre_num", "fpre_exp", "osc_down",
                                      "osc_up", "mult_max", "T_floor", "mbar_mp", "n_dof")] + \
               [("n_scat", ctypes.c_int), ("max_iter", ctypes.c_int), ("printed_gradient", ctypes.c_int),
                ("tabulate", ctypes.c_int)]


def build(force: bool = False) -> str:
    srcs = [os.path.join(_HERE, f) for f in ("opcount.cpp", "helios_ref.c", "helios_ref.h")]
    newest = max(os.path.getmtime(f) for f in srcs)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                               "-I", _HERE, "-o", tmp, srcs[0], "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        vp, i = ctypes.c_void_p, ctypes.c_int
        P = ctypes.POINTER
        lib.ref_opcount_get.argtypes = [vp]
        lib.ref_opcount_reset.argtypes = []
        lib.ref_default_params.argtypes = [P(_ParamsC)]
        lib.ref_flux_sweep.restype = i
        lib.ref_flux_sweep.argtypes = [P(_AtmC), P(_ParamsC), vp, i, i, vp, i, vp, vp, vp, vp, vp]
        lib.ref_gauss_legendre.argtypes = [i, vp, vp]
        lib.ref_grid.argtypes = [P(_AtmC), vp, vp, vp, vp]
        lib.ref_boundary_spectra.argtypes = [P(_AtmC), vp, vp]
        lib.ref_point_temperatures.argtypes = [i, vp, vp]
        lib.ref_table_coord.argtypes = [_CNum, _CNum, _CNum, i, P(ctypes.c_int), P(_CNum)]
        _lib = lib
    return _lib


def _arr(x, flag=0):
    a = np.zeros(np.size(x), dtype=CN)
    a["v"] = np.asarray(x, np.float64).ravel()
    a["f"] = flag
    return a


def _counts():
    out = np.zeros(2 * len(CATS), dtype=np.int64)
    _load().ref_opcount_get(out.ctypes.data)
    return {"coef": dict(zip(CATS, out[:len(CATS)].tolist())), "flux": dict(zip(CATS, out[len(CATS):].tolist()))}


def _sub(a, b, scale=1.0):
    return {k: a[k] - scale * b[k] for k in a}


def _add(a, b, scale=1.0):
    return {k: a[k] + scale * b[k] for k in a}


class _Atm:
    """The op-counting build's view of one synthetic atmosphere (arrays kept alive)."""

    def __init__(self, atm, table, kappa64=None, rayleigh=False):
        self.nu = _arr(atm.nu_edges)
        self.w0 = _arr(atm.omega0)
        self.g0 = _arr(atm.g0)
        k = table.kappa32.astype(np.float64) if kappa64 is None else kappa64
        self.kappa = _arr(k)
        s = _AtmC()
        s.n, s.L, s.G = atm.n_layers, atm.n_bins, table.G
        s.P_top_bar, s.P_bot_bar, s.grav = _cn(atm.P_top_bar), _cn(atm.P_bot_bar), _cn(atm.grav)
        s.T_irr, s.T_int = _cn(atm.T_irr, 1), _cn(atm.T_int, 1)      # the radiation field's sources
        s.T_star = _cn(atm.T_star)
        s.nu_edges, s.omega0, s.g0 = self.nu.ctypes.data, self.w0.ctypes.data, self.g0.ctypes.data
        s.nP, s.nT, s.L_table = table.nP, table.nT, table.L
        s.log10P0, s.dlog10P, s.T0, s.dT = _cn(table.log10P0), _cn(table.dlog10P), _cn(table.T0), _cn(table.dT)
        s.kappa = self.kappa.ctypes.data
        s.grey, s.rayleigh = 0, 1 if rayleigh else 0
        self.s = s
        self.n, self.L, self.G = atm.n_layers, atm.n_bins, table.G


def _params(n_scat=4):
    p = _ParamsC()
    _load().ref_default_params(ctypes.byref(p))
    p.n_scat = n_scat
    return p


def _eval_counts(a: _Atm, p, T, n_passes):
    lib = _load()
    n, np_ = a.n, 2 * a.n + 1
    Tc = _arr(T)
    Fu, Fd, toa = _arr(np.zeros(n + 1)), _arr(np.zeros(n + 1)), _arr(np.zeros(a.L))
    # the coupled stream starts from zero (a cold start), given as a warm start of flagged zeros so
    # that the first pass is counted like every other
    warm = _arr(np.zeros(a.L * a.G * np_), flag=1)
    lib.ref_opcount_reset()
    rc = lib.ref_flux_sweep(ctypes.byref(a.s), ctypes.byref(p), Tc.ctypes.data, n_passes, 0, warm.ctypes.data, 1,
                            Fu.ctypes.data, Fd.ctypes.data, toa.ctypes.data, None, None)
    if rc != 0:
        raise RuntimeError("op-counting flux evaluation failed")
    return _counts()


def _setup_counts(a: _Atm, T):
    """Operations of the per-evaluation set-up that does not scale with bins x points x g."""
    lib = _load()
    n, np_, G = a.n, 2 * a.n + 1, a.G
    lib.ref_opcount_reset()
    x, w = _arr(np.zeros(G)), _arr(np.zeros(G))
    lib.ref_gauss_legendre(G, x.ctypes.data, w.ctypes.data)
    lp, P, dm, Pl = _arr(np.zeros(np_)), _arr(np.zeros(np_)), _arr(np.zeros(np_ - 1)), _arr(np.zeros(n))
    lib.ref_grid(ctypes.byref(a.s), lp.ctypes.data, P.ctypes.data, dm.ctypes.data, Pl.ctypes.data)
    tb, bi = _arr(np.zeros(a.L)), _arr(np.zeros(a.L))
    lib.ref_boundary_spectra(ctypes.byref(a.s), tb.ctypes.data, bi.ctypes.data)
    Tp = _arr(np.zeros(np_))
    Tc = _arr(T)
    lib.ref_point_temperatures(n, Tc.ctypes.data, Tp.ctypes.data)
    idx, wt = ctypes.c_int(), _CNum()
    s = a.s
    for q in range(np_):
        lib.ref_table_coord(_cn(lp["v"][q]), s.log10P0, s.dlog10P, s.nP, ctypes.byref(idx), ctypes.byref(wt))
        lib.ref_table_coord(_cn(Tp["v"][q]), s.T0, s.dT, s.nT, ctypes.byref(idx), ctypes.byref(wt))
    return _counts()


def flux_evaluation(atm, table, T, n_passes, kappa64=None, rayleigh=False, n_scat=4):
    """Algorithmic operation counts of one flux evaluation of `atm` (a synthetic atmosphere) at
    the temperatures T with n_passes passes.  Returns a dict with
      coef: operations of the layer coefficients, Planck values and opacities (once per evaluation)
      flux: operations of the n_passes recurrences and the Gauss-point and bin sums
      cells: n L G; fp32, sfu: instruction estimates of the whole evaluation (module docstring);
      per_cell: fp32, sfu divided by the cells."""
    a = _Atm(atm, table, kappa64=kappa64, rayleigh=rayleigh)
    p = _params(n_scat)
    c1 = _eval_counts(a, p, T, 1)
    c2 = _eval_counts(a, p, T, 2)
    st = _setup_counts(a, T)
    pass_coef = _sub(c2["coef"], c1["coef"])                # two layer calls' coefficients per sublayer
    pass_flux = _sub(c2["flux"], c1["flux"])                # two calls x both streams per sublayer
    coef = _add(_sub(_sub(c1["coef"], pass_coef), st["coef"]), pass_coef, 0.5)
    flux = _add(_sub(_sub(c1["flux"], pass_flux), st["flux"]), pass_flux, 0.5 * n_passes)
    tot = _add(coef, flux)
    mul_extra = tot["div"] + tot["exp"] + tot["sqrt"] + tot["log"] + 2 * tot["pow"]
    fp32 = max(tot["add"], tot["mul"]) + mul_extra
    sfu = tot["div"] + tot["exp"] + tot["sqrt"] + tot["log"] + 2 * tot["pow"]
    cells = a.n * a.L * a.G
    return {"coef": coef, "flux": flux, "cells": cells, "fp32": fp32, "sfu": sfu,
            "per_cell": {"fp32": fp32 / cells, "sfu": sfu / cells}, "passes": n_passes}
