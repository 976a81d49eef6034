"""Learned initialiser of the radiative-equilibrium iteration.

The iteration of Sect. 2.2.3 may start from any profile; the number of flux evaluations it
needs depends on how far that start is from equilibrium.  This module maps six planet
parameters (T_irr, T_int, log10 g, [M/H], C/O, log10 of the mean opacity) to a 100-point
temperature profile (bottom to top, evenly spaced in log P over the model's range) with the
library's MLP (BF16 tensor-core products, FP32 accumulation, trained with Adam on the solver's
own converged solutions).  Every arithmetic step runs in the library: the training data's
statistics and standardisation (helios_column_stats, helios_standardize), training
(helios_mlp_train_step) and the start profiles (helios_mlp_initial_profiles: standardisation,
the network, de-standardisation, interpolation in log P to each atmosphere's layers, and the
fallback to the isothermal start for an invalid prediction).  The plain iteration still decides
every result: the solver iterates to eq. (29) from the predicted start.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import MLP, Context, _ptr, _stream_ptr, _torch, check


def column_stats(x, eps, stream=None):
    """(mu, sd + eps) of every column of a float32 CUDA tensor [B, n] (helios_column_stats)."""
    torch = _torch()
    x = x.contiguous()
    B, n = x.shape
    mu = torch.empty(n, dtype=torch.float32, device=x.device)
    sd = torch.empty(n, dtype=torch.float32, device=x.device)
    from . import _lib
    check(_lib.load().helios_column_stats(x.data_ptr(), B, n, float(eps), mu.data_ptr(), sd.data_ptr(),
                                          _stream_ptr(stream)))
    return mu, sd


def standardize(x, mu, sd, stream=None):
    """(x - mu) / sd column-wise in float32 (helios_standardize); a new tensor."""
    torch = _torch()
    x = x.contiguous()
    out = torch.empty_like(x)
    from . import _lib
    check(_lib.load().helios_standardize(x.data_ptr(), mu.data_ptr(), sd.data_ptr(), x.shape[0], x.shape[1],
                                         out.data_ptr(), _stream_ptr(stream)))
    return out


class LearnedInitializer:
    def __init__(self, ctx: Context, n_points: int = 100, n_hidden: int = 256, hidden_layers: int = 3, seed: int = 0,
                 max_batch: int = 4096):
        self.net = MLP(ctx, n_in=6, n_hidden=n_hidden, hidden_layers=hidden_layers, n_out=n_points, seed=seed,
                       max_batch=max_batch)
        self.n_points = n_points
        self.dev = self.net.params.device
        self.x_mu = self.x_sd = self.y_mu = self.y_sd = None     # float32 CUDA tensors after fit()

    # ---- training
    def fit(self, feats: np.ndarray, profiles: np.ndarray, epochs: int = 300, batch: int = 256, lr: float = 1e-3,
            seed: int = 0, lr_final: float = 1e-5):
        """Train on (features [N, 6], converged profiles [N, n_points] in K); returns the loss per epoch.
        The statistics and the standardised data are formed on the device by the library; the
        host only draws the epoch's order of the samples."""
        torch = _torch()
        F = torch.from_numpy(np.asarray(feats, np.float32)).to(self.dev)
        Yk = torch.from_numpy(np.asarray(profiles, np.float32)).to(self.dev)
        self.x_mu, self.x_sd = column_stats(F, 1e-12)
        self.y_mu, self.y_sd = column_stats(Yk, 1e-6)
        X, Y = standardize(F, self.x_mu, self.x_sd), standardize(Yk, self.y_mu, self.y_sd)
        n = X.shape[0]
        rng = np.random.default_rng(seed)
        batch = min(batch, n, self.net.max_batch)
        losses = []
        steps = max(1, epochs * ((n + batch - 1) // batch))
        k = 0
        for _ in range(epochs):
            perm = torch.from_numpy(rng.permutation(n)).to(self.dev)
            tot = torch.zeros((), dtype=torch.float64, device=self.dev)
            for s in range(0, n, batch):
                idx = perm[s:s + batch]
                rate = lr * (lr_final / lr) ** (k / steps)          # geometric decay
                loss = self.net.train_step(X[idx], Y[idx], lr=rate)
                tot += loss[0].double() * idx.numel()
                k += 1
            losses.append(float(tot.item()) / n)
        return losses

    # ---- inference
    def statistics(self):
        """The standardisation statistics (x_mu, x_sd, y_mu, y_sd), float32 CUDA tensors."""
        return self.x_mu, self.x_sd, self.y_mu, self.y_sd

    def initial_profiles_device(self, plan, feats, fallback, T_min=50.0, T_max=8000.0):
        """Start profiles for every atmosphere of `plan` (helios_mlp_initial_profiles), with
        `fallback` (the isothermal start) where the prediction is invalid.  Returns (T float64 CUDA
        tensor of the plan's layers, used: numpy bool [A])."""
        torch = _torch()
        f = torch.from_numpy(np.asarray(feats, np.float32)).to(self.dev)
        fb = torch.from_numpy(np.concatenate([np.asarray(x, np.float64) for x in fallback])).to(self.dev)
        T, used = self.net.initial_profiles(plan, f, *self.statistics(), fb, T_min=T_min, T_max=T_max)
        return T, used.cpu().numpy().astype(bool)

    def initial_profiles(self, plan, feats, fallback, T_min=50.0, T_max=8000.0):
        """The same start profiles as a list of numpy arrays (one per atmosphere) and `used`."""
        T, used = self.initial_profiles_device(plan, feats, fallback, T_min, T_max)
        return plan.split_layers(T.cpu().numpy()), used


def features(atms) -> np.ndarray:
    """[T_irr, T_int, log10 g (m s^-2), [M/H], C/O, log10 mean kappa] per atmosphere (from its generator
    parameters)."""
    return np.array([[a.params["T_irr"], a.params["T_int"], a.params["log10g"], a.params["MH"], a.params["CO"],
                      a.params["log10_mean_kappa"]] for a in atms], dtype=np.float64)
