"""B300-native radiative-equilibrium hot path of HELIOS (Malik et al. 2016, arXiv:1606.05474).

Python binding of the C ABI in ``include/helios.h``: argument marshalling only.
Every step of the method runs in the CUDA kernels of ``libhelios.so``;
PyTorch supplies device memory and streams.  There is no CPU fallback: the
package raises if the library or a CUDA device is missing.
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np

from . import _lib
from ._lib import (ATM_ACTIVE, ATM_CONVERGED, ATM_NONFINITE, ATM_NOT_CONVERGED, ATM_OUT_OF_RANGE, HeliosError,  # noqa: F401
                   check)

__all__ = ["Context", "Plan", "MLP", "default_params", "autotune", "flux_sweep_noalloc", "HeliosError", "build"]


def build(force: bool = False) -> str:
    from ._build import build as _b
    return _b(force=force)


DIRECT = _lib.HELIOS_DIRECT


def default_params(**overrides) -> _lib.Params:
    p = _lib.Params()
    _lib.load().helios_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("paper_1606_05474_b300 needs a CUDA device; there is no CPU path")
    return torch


def _stream_ptr(stream) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t):
    return None if t is None else t.data_ptr()


class Context:
    """A library context on one CUDA device."""

    def __init__(self, device: int = 0):
        _torch()
        self.lib = _lib.load()
        self.device = device
        h = ctypes.c_void_p()
        check(self.lib.helios_create(ctypes.byref(h), device))
        self.h = h

    def close(self):
        if self.h:
            self.lib.helios_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def flux_sweep_noalloc(atm, table, kappa, T, out, n_passes=0, params=None, stream=None):
    """One cold-start flux evaluation of a single atmosphere without a plan and without any
    allocation inside the library (helios_flux_sweep_noalloc).  For callers that cannot
    allocate device memory: all outputs are caller-provided tensors in `out` = (Fup_bol
    [n+1] float64, Fdn_bol [n+1] float64, Fup_toa [L] float32 or None)."""
    torch = _torch()
    lib = _lib.load()
    p = params if params is not None else default_params()
    host = {
        "n_layers": np.array([atm.n_layers], np.int32), "n_bins": np.array([atm.n_bins], np.int32),
        "table_id": np.zeros(1, np.int32), "P_top_bar": np.array([atm.P_top_bar], np.float64),
        "P_bot_bar": np.array([atm.P_bot_bar], np.float64), "grav": np.array([atm.grav], np.float64),
        "T_irr": np.array([atm.T_irr], np.float64), "T_int": np.array([atm.T_int], np.float64),
        "T_star": np.array([atm.T_star], np.float64),
        "nu_edges": np.ascontiguousarray(atm.nu_edges, np.float64),
        "omega0": np.ascontiguousarray(atm.omega0, np.float32), "g0": np.ascontiguousarray(atm.g0, np.float32)}
    b = _lib.Batch()
    b.A = 1
    for k, v in host.items():
        setattr(b, k, v.ctypes.data)
    if not (kappa.is_cuda and kappa.dtype == torch.float32 and kappa.is_contiguous()):
        raise ValueError("the k-table must be a contiguous float32 CUDA tensor")
    t = _lib.KTable()
    t.nP, t.nT, t.L, t.G = table.nP, table.nT, table.L, table.G
    t.log10P0, t.dlog10P, t.T0, t.dT = table.log10P0, table.dlog10P, table.T0, table.dT
    t.kappa = kappa.data_ptr()
    Fu, Fd, toa = out
    check(lib.helios_flux_sweep_noalloc(ctypes.byref(b), ctypes.byref(t), ctypes.byref(p), T.data_ptr(),
                                        int(n_passes), Fu.data_ptr(), Fd.data_ptr(), _ptr(toa), _stream_ptr(stream)))
    return Fu, Fd, toa


def _cat(arrays, dtype):
    # an empty batch passes empty arrays on, for the library to reject
    return np.ascontiguousarray(np.concatenate([np.asarray(x, dtype) for x in arrays]) if arrays else
                                np.zeros(1, dtype))


def _marshal(atms, tables, kappa):
    """Host arrays of a helios_batch_t and the helios_ktable_t descriptors (kept alive by the caller)."""
    torch = _torch()
    host = {
        "n_layers": np.array([a.n_layers for a in atms], dtype=np.int32),
        "n_bins": np.array([a.n_bins for a in atms], dtype=np.int32),
        "table_id": np.array([a.table_id for a in atms], dtype=np.int32),
        "P_top_bar": np.array([a.P_top_bar for a in atms], dtype=np.float64),
        "P_bot_bar": np.array([a.P_bot_bar for a in atms], dtype=np.float64),
        "grav": np.array([a.grav for a in atms], dtype=np.float64),
        "T_irr": np.array([a.T_irr for a in atms], dtype=np.float64),
        "T_int": np.array([a.T_int for a in atms], dtype=np.float64),
        "T_star": np.array([a.T_star for a in atms], dtype=np.float64),
        "nu_edges": _cat([a.nu_edges for a in atms], np.float64),
        "omega0": _cat([a.omega0 for a in atms], np.float32),
        "g0": _cat([a.g0 for a in atms], np.float32),
    }
    if any(getattr(a, "species", None) for a in atms):
        # eq. (34) mixing: (table, mass mixing ratio) pairs per atmosphere; plain atmospheres
        # contribute their own table with weight 1
        pairs = [list(a.species) if getattr(a, "species", None) else [(a.table_id, 1.0)] for a in atms]
        host["species_off"] = np.concatenate([[0], np.cumsum([len(p) for p in pairs])]).astype(np.int32)
        host["species_table"] = np.array([t for p in pairs for t, _ in p], dtype=np.int32)
        host["species_weight"] = np.array([w for p in pairs for _, w in p], dtype=np.float64)
    b = _lib.Batch()
    b.A = len(atms)
    for k, v in host.items():
        setattr(b, k, v.ctypes.data)
    for k in kappa:
        if not (k.is_cuda and k.dtype == torch.float32 and k.is_contiguous()):
            raise ValueError("k-tables must be contiguous float32 CUDA tensors")
    tabs = (_lib.KTable * len(tables))()
    for i, (t, k) in enumerate(zip(tables, kappa)):
        tabs[i].nP, tabs[i].nT, tabs[i].L, tabs[i].G = t.nP, t.nT, t.L, t.G
        tabs[i].log10P0, tabs[i].dlog10P, tabs[i].T0, tabs[i].dT = t.log10P0, t.dlog10P, t.T0, t.dT
        tabs[i].kappa = k.data_ptr()
    return b, tabs, host


def measure_peaks(ctx):
    """(FP32 TFLOP/s, MUFU ex2 T op/s) measured on the context's device (helios_measure_peaks)."""
    f, u = ctypes.c_double(), ctypes.c_double()
    check(ctx.lib.helios_measure_peaks(ctx.h, ctypes.byref(f), ctypes.byref(u)))
    return f.value, u.value


def device_recip(x, stream=None):
    """1/x by the device reciprocal of the two-stream coefficients (helios_device_recip); x: a
    float32 CUDA tensor.  Returns a new tensor."""
    torch = _torch()
    if x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous():
        raise ValueError("x must be a contiguous float32 CUDA tensor")
    y = torch.empty_like(x)
    check(_lib.load().helios_device_recip(x.data_ptr(), y.data_ptr(), x.numel(), _stream_ptr(stream)))
    return y


def autotune(ctx, atms, tables, kappa, params=None, cache_path=None):
    """Pick bins_per_item and the launch mode for this batch (helios_autotune); returns tuned params."""
    base = params if params is not None else default_params()
    b, tabs, _host = _marshal(atms, tables, kappa)
    out = _lib.Params()
    check(ctx.lib.helios_autotune(ctx.h, ctypes.byref(b), tabs, len(tables), ctypes.byref(base),
                                  cache_path.encode() if cache_path else None, ctypes.byref(out)))
    return out


class Plan:
    """A validated batch of atmospheres with its device workspace.

    atms: objects with n_layers, n_bins, table_id, P_top_bar, P_bot_bar, grav, T_irr,
    T_int, T_star, nu_edges, omega0, g0.  tables: objects with nP, nT, L, G, log10P0,
    dlog10P, T0, dT.  kappa: one float32 CUDA tensor [nP, nT, L, G] per table.
    """

    def __init__(self, ctx: Context, atms: Sequence, tables: Sequence, kappa: Sequence, params=None):
        torch = _torch()
        self.ctx, self.lib = ctx, ctx.lib
        self.params = params if params is not None else default_params()
        self.A = len(atms)
        self.n = np.array([a.n_layers for a in atms], dtype=np.int32)
        self.L = np.array([a.n_bins for a in atms], dtype=np.int32)
        b, tabs, self._host = _marshal(atms, tables, kappa)
        self.kappa = list(kappa)
        h = ctypes.c_void_p()
        check(self.lib.helios_plan_create(ctx.h, ctypes.byref(b), tabs, len(tables), ctypes.byref(self.params),
                                          ctypes.byref(h)))
        self.h = h
        info = _lib.PlanInfo()
        check(self.lib.helios_plan_info(h, ctypes.byref(info)))
        self.info = info
        self.G = tables[0].G
        self.lay_off = np.concatenate([[0], np.cumsum(self.n)]).astype(np.int64)
        self.if_off = np.concatenate([[0], np.cumsum(self.n + 1)]).astype(np.int64)
        self.pt_off = np.concatenate([[0], np.cumsum(2 * self.n + 1)]).astype(np.int64)
        self.bin_off = np.concatenate([[0], np.cumsum(self.L)]).astype(np.int64)
        self.dev = torch.device("cuda", ctx.device)

    def close(self):
        if getattr(self, "h", None):
            self.lib.helios_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- helpers
    def _empty(self, n, dtype):
        return _torch().empty(int(n), dtype=dtype, device=self.dev)

    def _check_T(self, T):
        torch = _torch()
        if not (T.is_cuda and T.dtype == torch.float64 and T.is_contiguous() and T.numel() == self.info.layers):
            raise ValueError(f"T_layer must be a contiguous float64 CUDA tensor of {self.info.layers} values")

    # ---- the four calls of the hot path
    def interp_opacity(self, T, want_kappa=True, stream=None):
        torch = _torch()
        self._check_T(T)
        nk = sum((2 * int(n) + 1) * int(L) for n, L in zip(self.n, self.L)) * int(self.G)
        kap = self._empty(nk, torch.float32) if want_kappa else None
        idx = self._empty(2 * self.info.points, torch.int32)
        w = self._empty(2 * self.info.points, torch.float64)
        check(self.lib.helios_interp_opacity(self.h, T.data_ptr(), _ptr(kap), idx.data_ptr(), w.data_ptr(),
                                             _stream_ptr(stream)))
        return kap, idx.view(-1, 2), w.view(-1, 2)

    def flux_sweep(self, T, n_passes=0, warm=False, want_toa=True, out=None, stream=None, warm_buf=None,
                   spec=None):
        """One flux evaluation (helios_flux_sweep); returns (Fup_bol, Fdn_bol, Fup_toa).
        warm_buf: optional caller-owned float32 warm-start tensor of info.warm_floats values (the
        plan's own buffer otherwise).  spec: optional float32 tensor of info.spec_floats values
        that receives every bin's fluxes at every point (see split_spec)."""
        torch = _torch()
        self._check_T(T)
        if out is None:
            out = (self._empty(self.info.interfaces, torch.float64), self._empty(self.info.interfaces, torch.float64),
                   self._empty(self.info.bins, torch.float32) if want_toa else None)
        Fu, Fd, toa = out
        for buf, size, name in ((warm_buf, self.info.warm_floats, "warm_buf"), (spec, self.info.spec_floats, "spec")):
            if buf is not None and not (buf.is_cuda and buf.dtype == torch.float32 and buf.is_contiguous()
                                        and buf.numel() == size):
                raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of {size} values")
        check(self.lib.helios_flux_sweep(self.h, T.data_ptr(), int(n_passes), 1 if warm else 0, _ptr(warm_buf),
                                         Fu.data_ptr(), Fd.data_ptr(), _ptr(toa), _ptr(spec), _stream_ptr(stream)))
        return Fu, Fd, toa

    def split_spec(self, spec):
        """The per-bin flux output of flux_sweep as one (Fup [L, 2n+1], Fdn [L, 2n+1]) numpy pair
        per atmosphere."""
        v = spec.cpu().numpy() if hasattr(spec, "cpu") else np.asarray(spec)
        out, off = [], 0
        for n, L in zip(self.n, self.L):
            np_ = 2 * int(n) + 1
            blk = v[off:off + 2 * int(L) * np_].reshape(int(L), 2, np_)
            out.append((blk[:, 0, :], blk[:, 1, :]))
            off += 2 * int(L) * np_
        return out

    def emission_spectrum(self, T, n_passes=81, stream=None):
        """Emergent spectrum of converged temperatures T (Sect. 3: computed as a post-processing
        step, on a plan made with iso_layers=1 and the spectrum's bins; Sect. 2.2.3: 80
        additional scattering passes, or n_passes=DIRECT for their limit).  One cold-start
        evaluation; returns (Fup_toa per bin, Fup_bol, Fdn_bol)."""
        Fu, Fd, toa = self.flux_sweep(T, n_passes=n_passes, warm=False, want_toa=True, stream=stream)
        return toa, Fu, Fd

    def new_state(self):
        torch = _torch()
        L = int(self.info.layers)
        return {"mult": torch.ones(L, dtype=torch.float64, device=self.dev),
                "hist": torch.zeros(L, dtype=torch.uint8, device=self.dev),
                "nhist": torch.zeros(L, dtype=torch.uint8, device=self.dev),
                "status": torch.zeros(self.A, dtype=torch.int32, device=self.dev),
                "iters": torch.zeros(self.A, dtype=torch.int32, device=self.dev),
                "metric": torch.zeros(self.A, dtype=torch.float64, device=self.dev)}

    def temp_update(self, Fup, Fdn, T, state, stream=None):
        self._check_T(T)
        s = state
        check(self.lib.helios_temp_update(self.h, Fup.data_ptr(), Fdn.data_ptr(), T.data_ptr(), s["mult"].data_ptr(),
                                          s["hist"].data_ptr(), s["nhist"].data_ptr(), s["status"].data_ptr(),
                                          _ptr(s.get("iters")), _ptr(s.get("metric")), _stream_ptr(stream)))
        return state

    def re_step(self, T, state, warm=True, out=None, stream=None):
        """One radiative-equilibrium iteration of every atmosphere in place (helios_re_step):
        the flux evaluation with the plan's default passes and the temperature step.  out:
        optional (Fup_bol, Fdn_bol) tensors for this step's bolometric fluxes."""
        self._check_T(T)
        s = state
        Fu, Fd = out if out is not None else (None, None)
        check(self.lib.helios_re_step(self.h, T.data_ptr(), 1 if warm else 0, s["mult"].data_ptr(),
                                      s["hist"].data_ptr(), s["nhist"].data_ptr(), s["status"].data_ptr(),
                                      _ptr(s.get("iters")), _ptr(s.get("metric")), _ptr(Fu), _ptr(Fd),
                                      _stream_ptr(stream)))
        return state

    def re_step_host(self, T_host, T_dev, state, status_host, warm=True, stream=None):
        """helios_re_step_host: one iteration with the temperatures in host memory.  T_host: a
        float64 CPU tensor (pinned for asynchronous copies), updated in place; T_dev: a float64
        CUDA scratch tensor of the same size; status_host: an int32 CPU tensor of A values.  The
        host tensors hold the result once the stream has reached this call."""
        torch = _torch()
        n = int(self.info.layers)
        if not (T_host.dtype == torch.float64 and not T_host.is_cuda and T_host.is_contiguous() and T_host.numel() == n):
            raise ValueError(f"T_host must be a contiguous float64 CPU tensor of {n} values")
        if not (status_host.dtype == torch.int32 and not status_host.is_cuda and status_host.numel() == self.A):
            raise ValueError(f"status_host must be an int32 CPU tensor of {self.A} values")
        self._check_T(T_dev)
        s = state
        check(self.lib.helios_re_step_host(self.h, T_host.data_ptr(), T_dev.data_ptr(), 1 if warm else 0,
                                           s["mult"].data_ptr(), s["hist"].data_ptr(), s["nhist"].data_ptr(),
                                           s["status"].data_ptr(), _ptr(s.get("iters")), _ptr(s.get("metric")),
                                           status_host.data_ptr(), _stream_ptr(stream)))
        return state

    def solve_re(self, T, stream=None, raise_on_noconv=False):
        """Iterate to radiative equilibrium in place; returns (iters, status) CUDA tensors."""
        torch = _torch()
        self._check_T(T)
        iters = self._empty(self.A, torch.int32)
        status = self._empty(self.A, torch.int32)
        rc = self.lib.helios_solve_re(self.h, T.data_ptr(), iters.data_ptr(), status.data_ptr(), _stream_ptr(stream))
        if rc != _lib.HELIOS_OK and (raise_on_noconv or rc != _lib.HELIOS_ENOCONV):
            check(rc)
        return iters, status

    # ---- measurement
    def set_timing(self, slots=1):
        """Record CUDA events around the sweep kernels of the last `slots` evaluations (0: off)."""
        check(self.lib.helios_plan_set_timing(self.h, int(slots)))

    def sweep_times(self, max_n=65536):
        buf = np.zeros(max_n, dtype=np.float32)
        n = ctypes.c_int()
        check(self.lib.helios_plan_sweep_times(self.h, buf.ctypes.data, max_n, ctypes.byref(n)))
        return buf[:n.value].copy()

    def last_sweep_ms(self) -> float:
        v = ctypes.c_float()
        check(self.lib.helios_plan_last_sweep_ms(self.h, ctypes.byref(v)))
        return v.value

    # ---- packing helpers
    def export_state(self, out=None, stream=None):
        """Checkpoint of the plan's own iteration state (helios_plan_state_export): a uint8 tensor
        (device by default, or `out`, host or device) that import_state restores."""
        torch = _torch()
        n = ctypes.c_int64()
        check(self.lib.helios_plan_state_bytes(self.h, ctypes.byref(n)))
        buf = out if out is not None else torch.empty(n.value, dtype=torch.uint8, device=self.dev)
        if buf.dtype != torch.uint8 or buf.numel() != n.value or not buf.is_contiguous():
            raise ValueError(f"the checkpoint buffer must be a contiguous uint8 tensor of {n.value} bytes")
        check(self.lib.helios_plan_state_export(self.h, buf.data_ptr(), _stream_ptr(stream)))
        return buf

    def import_state(self, buf, stream=None):
        """Restore a checkpoint made by export_state of a plan of the same shape
        (helios_plan_state_import); the next re_step with warm=True continues from it."""
        torch = _torch()
        if buf.dtype != torch.uint8 or not buf.is_contiguous():
            raise ValueError("the checkpoint must be a contiguous uint8 tensor")
        check(self.lib.helios_plan_state_import(self.h, buf.data_ptr(), _stream_ptr(stream)))

    def split_layers(self, x):
        return [x[self.lay_off[a]:self.lay_off[a + 1]] for a in range(self.A)]

    def split_interfaces(self, x):
        return [x[self.if_off[a]:self.if_off[a + 1]] for a in range(self.A)]

    def split_bins(self, x):
        return [x[self.bin_off[a]:self.bin_off[a + 1]] for a in range(self.A)]


class _DeviceView:
    """__cuda_array_interface__ over library-owned device memory (no copy, no allocation)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": "<f4", "data": (int(ptr), False), "version": 3}


class MLP:
    """The learned initialiser's network (helios_mlp_*): n_in -> hidden_layers x n_hidden (SiLU) -> n_out."""

    def __init__(self, ctx: Context, n_in=6, n_hidden=256, hidden_layers=3, n_out=100, seed=0, max_batch=4096):
        torch = _torch()
        self.ctx, self.lib = ctx, ctx.lib
        self.dims = [n_in] + [n_hidden] * hidden_layers + [n_out]
        self.max_batch = max_batch
        h = ctypes.c_void_p()
        check(self.lib.helios_mlp_create(ctx.h, n_in, n_hidden, hidden_layers, n_out, seed, max_batch, ctypes.byref(h)))
        self.h = h
        p, g, n = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_longlong()
        check(self.lib.helios_mlp_params(h, ctypes.byref(p), ctypes.byref(g), ctypes.byref(n)))
        dev = torch.device("cuda", ctx.device)
        self.params = torch.as_tensor(_DeviceView(p.value, n.value), device=dev)
        self.grads = torch.as_tensor(_DeviceView(g.value, n.value), device=dev)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)

    def close(self):
        if getattr(self, "h", None):
            self.lib.helios_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params_changed(self):
        """Declare that the parameters were written through `params` (helios_mlp_params_changed):
        the BF16 weight tiles of the matrix products are rebuilt before the next product."""
        check(self.lib.helios_mlp_params_changed(self.h))

    def layer_views(self):
        """[(W_l [in, out], b_l [out])] views into the parameter buffer (after writing through them,
        call params_changed)."""
        out, o = [], 0
        for a, b in zip(self.dims[:-1], self.dims[1:]):
            W = self.params[o:o + a * b].view(a, b); o += a * b
            bb = self.params[o:o + b]; o += b
            out.append((W, bb))
        return out

    def forward(self, x, out=None, stream=None):
        torch = _torch()
        x = x.contiguous()
        y = out if out is not None else torch.empty(x.shape[0], self.dims[-1], dtype=torch.float32, device=x.device)
        check(self.lib.helios_mlp_forward(self.h, x.data_ptr(), y.data_ptr(), x.shape[0], _stream_ptr(stream)))
        return y

    def grad(self, x, target, stream=None):
        check(self.lib.helios_mlp_grad(self.h, x.contiguous().data_ptr(), target.contiguous().data_ptr(), x.shape[0],
                                       self.loss.data_ptr(), _stream_ptr(stream)))
        return self.loss

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        check(self.lib.helios_mlp_adam(self.h, lr, beta1, beta2, eps, _stream_ptr(stream)))

    def error(self):
        """1 if a tensor-core product of this network gave up waiting (its results invalid), else 0
        (helios_mlp_error; synchronous)."""
        f = ctypes.c_int()
        check(self.lib.helios_mlp_error(self.h, ctypes.byref(f)))
        return f.value

    def train_step(self, x, target, lr=1e-3, stream=None):
        check(self.lib.helios_mlp_train_step(self.h, x.contiguous().data_ptr(), target.contiguous().data_ptr(),
                                             x.shape[0], lr, self.loss.data_ptr(), _stream_ptr(stream)))
        return self.loss

    def initial_profiles(self, plan, feats, x_mu, x_sd, y_mu, y_sd, T_fallback, T_min=50.0, T_max=8000.0, out=None,
                         stream=None):
        """helios_mlp_initial_profiles: start profiles of every atmosphere of `plan` (a float64 CUDA
        tensor of plan.info.layers values) and which ones kept the network's profile (int32 [A]).
        feats: float32 CUDA [A, n_in] (raw); x_mu, x_sd, y_mu, y_sd: float32 CUDA statistics;
        T_fallback: float64 CUDA [layers]."""
        torch = _torch()
        T = out if out is not None else torch.empty(int(plan.info.layers), dtype=torch.float64, device=T_fallback.device)
        used = torch.empty(plan.A, dtype=torch.int32, device=T_fallback.device)
        args = [feats, x_mu, x_sd, y_mu, y_sd]
        if any(a.dtype != torch.float32 or not a.is_cuda or not a.is_contiguous() for a in args):
            raise ValueError("features and statistics must be contiguous float32 CUDA tensors")
        if feats.numel() != plan.A * self.dims[0]:
            raise ValueError(f"feats must hold {plan.A} x {self.dims[0]} values")
        plan._check_T(T_fallback)
        check(self.lib.helios_mlp_initial_profiles(self.h, plan.h, feats.data_ptr(), x_mu.data_ptr(), x_sd.data_ptr(),
                                                   y_mu.data_ptr(), y_sd.data_ptr(), T_fallback.data_ptr(), T_min,
                                                   T_max, T.data_ptr(), used.data_ptr(), _stream_ptr(stream)))
        return T, used
