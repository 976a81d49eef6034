"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the CPU oracle's tests, the GPU tests, ``bench.py``
and the smoke test.  It holds none of the method's arithmetic: it draws
random numbers and lays out the inputs (pressure range, wavenumber bin edges,
scattering parameters, correlated-k tables, stellar and internal
temperatures).  Everything the method computes from these inputs (grids,
optical depths, Planck functions, boundary spectra, Gauss weights, fluxes,
temperature steps) is done separately by the oracle and by the CUDA library.

Randomness is a counter-based splitmix64 stream (integer-only, so numpy and
the C helper in ``synth_gen.c`` agree bit for bit).  Seeds are
``SEED_BASE + config``; every quantity draws from its own named stream.

Workload shapes follow the paper's set-up: bins equal in wavenumber
(Sect. 3, default set-up), a k-table on a (log P, T) grid with 20 Gauss
points per bin (Sect. 2.3), layers log-spaced in pressure (Sect. 2.2.1).
The opacities themselves are synthetic: log10(kappa) uniform in [-6, 2]
cm^2/g, sorted over g so each bin's k-distribution is monotone.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

SEED_BASE = 1606054740
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_synth_gen.so")
_lib = None

# named streams
STREAM_TABLE = 1000      # + table index
STREAM_ATM = 2           # per-atmosphere scalars
STREAM_G0 = 3            # per-bin asymmetry factors
STREAM_MIX = 4           # learned-initialiser parameters


# ----------------------------------------------------------------------------
# splitmix64 (numpy, vectorised)
# ----------------------------------------------------------------------------
def _mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> int:
    with np.errstate(over="ignore"):
        z = np.uint64(seed) ^ (np.uint64(stream) * _GOLDEN)
    return int(_mix64(np.array([z], dtype=np.uint64))[0])


def uniform(key: int, first: int, count: int) -> np.ndarray:
    """u_i = (splitmix64(key + (i+1)*golden) >> 11) * 2^-53 for i in [first, first+count)."""
    i = np.arange(first, first + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(key) + (i + np.uint64(1)) * _GOLDEN
    return (_mix64(z) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# ----------------------------------------------------------------------------
# C helper for large tables
# ----------------------------------------------------------------------------
def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "synth_gen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.synth_stream_key.restype = ctypes.c_uint64
        lib.synth_stream_key.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.synth_uniform.restype = ctypes.c_double
        lib.synth_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.synth_uniform_fill.restype = None
        lib.synth_uniform_fill.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
        lib.synth_ktable.restype = None
        lib.synth_ktable.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
        _lib = lib
    return _lib


def c_uniform(key: int, first: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    _load().synth_uniform_fill(ctypes.c_uint64(key), ctypes.c_uint64(first), count, out.ctypes.data)
    return out


# ----------------------------------------------------------------------------
# data containers
# ----------------------------------------------------------------------------
@dataclass
class KTable:
    """Correlated-k table kappa[nP][nT][L][G] in cm^2/g on a (log10 P[bar], T[K]) grid."""
    nP: int
    nT: int
    L: int
    G: int
    log10P0: float       # log10 of the first pressure node, bar
    dlog10P: float
    T0: float            # first temperature node, K
    dT: float
    kappa32: np.ndarray  # float32 [nP, nT, L, G]
    kappa64: Optional[np.ndarray] = None

    def kappa_for_oracle(self) -> np.ndarray:
        """The values the GPU receives (float32), widened to float64."""
        return self.kappa32.astype(np.float64)


@dataclass
class Atmosphere:
    n_layers: int
    P_top_bar: float     # pressure of the top layer centre
    P_bot_bar: float     # pressure of the bottom layer centre
    grav: float          # cm s^-2
    T_irr: float         # K, total incident diffuse flux is sigma*T_irr^4
    T_int: float         # K, internal flux sigma*T_int^4
    T_star: float        # K, stellar blackbody temperature
    nu_edges: np.ndarray  # float64 [L+1], cm^-1, increasing
    omega0: np.ndarray   # float32 [L]
    g0: np.ndarray       # float32 [L]
    table_id: int
    T_init: np.ndarray   # float64 [n_layers], bottom layer first
    species: Optional[list] = None   # [(table index, mass mixing ratio)] to mix tables, or None
    params: Optional[dict] = None    # generator parameters (for the learned initialiser's features)

    @property
    def n_bins(self) -> int:
        return len(self.nu_edges) - 1


@dataclass
class Workload:
    name: str
    atms: List[Atmosphere]
    tables: List[KTable]
    n_scat: int = 4               # extra scattering passes per temperature step
    grey: bool = False
    meta: dict = field(default_factory=dict)

    @property
    def G(self) -> int:
        return self.tables[0].G

    @property
    def cells(self) -> int:
        """(atmosphere, layer, bin, g) cells of one flux evaluation."""
        return int(sum(a.n_layers * a.n_bins for a in self.atms) * self.G)


# ----------------------------------------------------------------------------
# builders
# ----------------------------------------------------------------------------
NU_MIN = 1.0e4 / 200.0        # 200 um
NU_MAX = 1.0e4 / 0.3          # 0.3 um


def make_ktable(seed: int, index: int, L: int, G: int, log10P_lo: float, log10P_hi: float,
                nP: int = 20, nT: int = 20, T_lo: float = 200.0, T_hi: float = 3000.0,
                want64: bool = False) -> KTable:
    key = stream_key(seed, STREAM_TABLE + index)
    k32 = np.empty((nP, nT, L, G), dtype=np.float32)
    k64 = np.empty((nP, nT, L, G), dtype=np.float64) if want64 else None
    _load().synth_ktable(ctypes.c_uint64(key), nP, nT, L, G, -6.0, 2.0,
                         k64.ctypes.data if want64 else None, k32.ctypes.data)
    return KTable(nP=nP, nT=nT, L=L, G=G, log10P0=log10P_lo,
                  dlog10P=(log10P_hi - log10P_lo) / (nP - 1), T0=T_lo,
                  dT=(T_hi - T_lo) / (nT - 1), kappa32=k32, kappa64=k64)


def nu_edges(L: int, nu_min: float = NU_MIN, nu_max: float = NU_MAX) -> np.ndarray:
    return np.linspace(nu_min, nu_max, L + 1)


def rayleigh_like_omega0(edges: np.ndarray) -> np.ndarray:
    """Single-scattering albedo falling as lambda^-4 from the 0.5 um value 0.9, capped at 0.9."""
    nu_c = 0.5 * (edges[:-1] + edges[1:])
    lam_um = 1.0e4 / nu_c
    return np.minimum(0.9, 0.9 * (0.5 / lam_um) ** 4).astype(np.float32)


def config1(grey: bool = False) -> Workload:
    """Plain method, single atmosphere: 50 layers 1e-6..1e2 bar, 30 bins x 8 g, pure absorption."""
    seed = SEED_BASE + 1
    L, G, n = 30, 8, 50
    tab = make_ktable(seed, 0, L, G, -6.0, 2.0, want64=True)
    e = nu_edges(L)
    atm = Atmosphere(n_layers=n, P_top_bar=1e-6, P_bot_bar=1e2, grav=1000.0, T_irr=1200.0, T_int=100.0,
                     T_star=5000.0, nu_edges=e, omega0=np.zeros(L, np.float32), g0=np.zeros(L, np.float32),
                     table_id=0, T_init=np.full(n, 1000.0))
    return Workload(name="plain-single-50x30x8", atms=[atm], tables=[tab], n_scat=0)


def config2(L: int = 3000, n: int = 100) -> Workload:
    """Full-size single atmosphere: 100 layers 1e-6..1e3 bar, 3000 bins x 20 g, Rayleigh-like scattering."""
    seed = SEED_BASE + 2
    G = 20
    tab = make_ktable(seed, 0, L, G, -6.0, 3.0)
    e = nu_edges(L)
    g0 = (0.5 * uniform(stream_key(seed, STREAM_G0), 0, L)).astype(np.float32)
    atm = Atmosphere(n_layers=n, P_top_bar=1e-6, P_bot_bar=1e3, grav=1000.0, T_irr=1200.0, T_int=100.0,
                     T_star=5000.0, nu_edges=e, omega0=rayleigh_like_omega0(e), g0=g0,
                     table_id=0, T_init=np.full(n, 1000.0))
    return Workload(name=f"full-single-{n}x{L}x{G}", atms=[atm], tables=[tab], n_scat=4)


def _atm_scalars(seed: int, a: int):
    key = stream_key(seed, STREAM_ATM)
    u = uniform(key, 8 * a, 8)
    n = 50 + int(u[0] * 151)                      # U{50..200}
    L = 300 + int(u[1] * 2701)                    # U{300..3000}
    T_irr = 500.0 + 2500.0 * u[2]
    T_int = 50.0 + 350.0 * u[3]
    grav = 100.0 * 10.0 ** (0.5 + u[4])           # log10(g / m s^-2) in [0.5, 1.5], in cm s^-2
    return n, L, T_irr, T_int, grav, u


def config3(A: int = 4096, n_tables: int = 64, L_table: int = 3000, atm_ids=None) -> Workload:
    """Batched ragged atmospheres sharing a seeded pool of k-tables (atmosphere a uses table a mod pool)."""
    seed = SEED_BASE + 3
    G = 20
    ids = list(range(A)) if atm_ids is None else list(atm_ids)
    used = sorted({a % n_tables for a in ids})
    tabs = {t: make_ktable(seed, t, L_table, G, -6.0, 3.0) for t in used}
    remap = {t: i for i, t in enumerate(used)}
    g0_all = (0.5 * uniform(stream_key(seed, STREAM_G0), 0, L_table)).astype(np.float32)
    atms = []
    for a in ids:
        n, L, T_irr, T_int, grav, _ = _atm_scalars(seed, a)
        e = nu_edges(L)
        atms.append(Atmosphere(n_layers=n, P_top_bar=1e-6, P_bot_bar=1e3, grav=grav, T_irr=T_irr,
                               T_int=T_int, T_star=5000.0, nu_edges=e, omega0=rayleigh_like_omega0(e),
                               g0=g0_all[:L].copy(), table_id=remap[a % n_tables],
                               T_init=np.full(n, T_irr)))
    return Workload(name=f"batched-{len(ids)}-ragged", atms=atms, tables=[tabs[t] for t in used], n_scat=4,
                    meta={"atm_ids": ids, "pool": n_tables})


def config5(A: int = 64, L: int = 30000, n: int = 200, atm_ids=None) -> Workload:
    """High-resolution precision stress: 200 layers x 30000 bins x 20 g with scattering, one shared table."""
    seed = SEED_BASE + 5
    G = 20
    tab = make_ktable(seed, 0, L, G, -6.0, 3.0)
    e = nu_edges(L)
    g0 = (0.5 * uniform(stream_key(seed, STREAM_G0), 0, L)).astype(np.float32)
    ids = list(range(A)) if atm_ids is None else list(atm_ids)
    atms = []
    for a in ids:
        _, _, T_irr, T_int, grav, _ = _atm_scalars(seed, a)
        atms.append(Atmosphere(n_layers=n, P_top_bar=1e-6, P_bot_bar=1e3, grav=grav, T_irr=T_irr,
                               T_int=T_int, T_star=5000.0, nu_edges=e, omega0=rayleigh_like_omega0(e),
                               g0=g0, table_id=0, T_init=np.full(n, T_irr)))
    return Workload(name=f"precision-{len(ids)}x{n}x{L}x{G}", atms=atms, tables=[tab], n_scat=4)


def small_scattering(L: int = 60, n: int = 40, G: int = 20, seed_offset: int = 7) -> Workload:
    """A scattering atmosphere small enough for the oracle to finish quickly (several lane tiles, ragged tail)."""
    seed = SEED_BASE + seed_offset
    tab = make_ktable(seed, 0, L, G, -6.0, 3.0)
    e = nu_edges(L)
    g0 = (0.5 * uniform(stream_key(seed, STREAM_G0), 0, L)).astype(np.float32)
    atm = Atmosphere(n_layers=n, P_top_bar=1e-6, P_bot_bar=1e3, grav=1000.0, T_irr=1200.0, T_int=100.0,
                     T_star=5000.0, nu_edges=e, omega0=rayleigh_like_omega0(e), g0=g0,
                     table_id=0, T_init=np.full(n, 1000.0))
    return Workload(name=f"scat-small-{n}x{L}x{G}", atms=[atm], tables=[tab], n_scat=4)


def perturbed_profile(atm: Atmosphere, seed: int, amp: float = 300.0) -> np.ndarray:
    """A smooth, seeded non-isothermal temperature profile around the atmosphere's start value."""
    u = uniform(stream_key(seed, 99), 0, 4)
    n = atm.n_layers
    x = np.linspace(0.0, 1.0, n)
    T = atm.T_init + amp * (u[0] - 0.5) + amp * np.sin(np.pi * (x * (1.0 + 2.0 * u[1]) + u[2])) * 0.5 \
        + amp * (1.0 - x) * u[3]
    return np.maximum(T, 150.0)


def grey_two_band(n: int = 50, gamma: float = 0.25, kappa_th: float = 1e-2, T_irr: float = 1200.0,
                  T_int: float = 100.0, P_bot_bar: float = 1e2) -> Workload:
    """Two bins, one Gauss point: a visible band (stellar only) and a thermal band (sigma T^4 source)."""
    tab = KTable(nP=2, nT=2, L=2, G=1, log10P0=-6.0, dlog10P=8.0, T0=200.0, dT=2800.0,
                 kappa32=np.empty((2, 2, 2, 1), np.float32))
    k = np.empty((2, 2, 2, 1))
    k[:, :, 0, 0] = gamma * kappa_th
    k[:, :, 1, 0] = kappa_th
    tab.kappa32[...] = k.astype(np.float32)
    tab.kappa64 = k
    e = np.array([NU_MIN, 0.5 * (NU_MIN + NU_MAX), NU_MAX])
    atm = Atmosphere(n_layers=n, P_top_bar=1e-6, P_bot_bar=P_bot_bar, grav=1000.0, T_irr=T_irr, T_int=T_int,
                     T_star=5000.0, nu_edges=e, omega0=np.zeros(2, np.float32), g0=np.zeros(2, np.float32),
                     table_id=0, T_init=np.full(n, 1000.0))
    return Workload(name=f"grey-two-band-{n}", atms=[atm], tables=[tab], n_scat=0, grey=True,
                    meta={"gamma": gamma, "kappa_th": kappa_th})


def learned_dataset(n_samples: int, L: int = 300, n: int = 100, first: int = 0) -> Workload:
    """Planet parameters for the learned initialiser, on the full-size atmosphere's geometry
    (100 layers, 1e-6..1e3 bar, 20 g, Rayleigh-like scattering) with L bins.

    Per sample: T_irr ~ U[500, 3000] K, T_int ~ U[50, 400] K, log10(g / m s^-2) ~ U[0.5, 1.5],
    [M/H] ~ U[-1, 1], C/O ~ U[0.3, 1.5].  The opacity mixes two seeded tables A and B:
    kappa = 10^[M/H] (kappa_A/(1 + C/O) + kappa_B (C/O)/(1 + C/O)) -- a synthetic stand-in
    (not a chemistry model) that makes [M/H] and C/O matter.  Start: isothermal at T_irr."""
    seed = SEED_BASE + 4
    G = 20
    tabA = make_ktable(seed, 0, L, G, -6.0, 3.0)
    tabB = make_ktable(seed, 1, L, G, -6.0, 3.0)
    e = nu_edges(L)
    w0 = rayleigh_like_omega0(e)
    g0 = (0.5 * uniform(stream_key(seed, STREAM_G0), 0, L)).astype(np.float32)
    meanA, meanB = float(tabA.kappa32.astype(np.float64).mean()), float(tabB.kappa32.astype(np.float64).mean())
    key = stream_key(seed, STREAM_MIX)
    atms = []
    for i in range(first, first + n_samples):
        u = uniform(key, 8 * i, 8)
        T_irr = 500.0 + 2500.0 * u[0]
        T_int = 50.0 + 350.0 * u[1]
        lg = 0.5 + u[2]
        mh = -1.0 + 2.0 * u[3]
        co = 0.3 + 1.2 * u[4]
        cA = 10.0 ** mh / (1.0 + co)
        cB = 10.0 ** mh * co / (1.0 + co)
        atms.append(Atmosphere(n_layers=n, P_top_bar=1e-6, P_bot_bar=1e3, grav=100.0 * 10.0 ** lg, T_irr=T_irr,
                               T_int=T_int, T_star=5000.0, nu_edges=e, omega0=w0, g0=g0, table_id=0,
                               T_init=np.full(n, T_irr), species=[(0, cA), (1, cB)],
                               params={"T_irr": T_irr, "T_int": T_int, "log10g": lg, "MH": mh, "CO": co,
                                       "log10_mean_kappa": float(np.log10(cA * meanA + cB * meanB))}))
    return Workload(name=f"learned-{n_samples}x{n}x{L}x{G}", atms=atms, tables=[tabA, tabB], n_scat=4)

