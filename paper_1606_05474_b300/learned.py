"""Learned initialiser of the radiative-equilibrium iteration.

The iteration of Sect. 2.2.3 may start from any profile; the number of flux evaluations it
needs depends on how far that start is from equilibrium.  This module maps six planet
parameters (T_irr, T_int, log10 g, [M/H], C/O, log10 of the mean opacity) to a 100-point
temperature profile (bottom to top, evenly spaced in log P over the model's range) with the
library's MLP (BF16 tensor-core products, FP32 accumulation, trained with Adam on the solver's
own converged solutions), interpolates it to each atmosphere's layers and validates it; an
invalid prediction falls back to the isothermal start, and the plain iteration still decides
every result (the solver iterates to eq. 29 from the predicted start).
"""
from __future__ import annotations

import numpy as np

from . import MLP, Context, _torch


class LearnedInitializer:
    def __init__(self, ctx: Context, n_points: int = 100, n_hidden: int = 256, hidden_layers: int = 3, seed: int = 0,
                 max_batch: int = 4096):
        self.net = MLP(ctx, n_in=6, n_hidden=n_hidden, hidden_layers=hidden_layers, n_out=n_points, seed=seed,
                       max_batch=max_batch)
        self.n_points = n_points
        self.dev = self.net.params.device
        self.x_mu = self.x_sd = self.y_mu = self.y_sd = None

    # ---- training
    def fit(self, feats: np.ndarray, profiles: np.ndarray, epochs: int = 300, batch: int = 256, lr: float = 1e-3,
            seed: int = 0, lr_final: float = 1e-5):
        """Train on (features [N, 6], converged profiles [N, n_points] in K); returns the loss per epoch."""
        torch = _torch()
        feats = np.asarray(feats, np.float64)
        prof = np.asarray(profiles, np.float64)
        self.x_mu, self.x_sd = feats.mean(0), feats.std(0) + 1e-12
        self.y_mu, self.y_sd = prof.mean(0), prof.std(0) + 1e-6
        X = torch.from_numpy(((feats - self.x_mu) / self.x_sd).astype(np.float32)).to(self.dev)
        Y = torch.from_numpy(((prof - self.y_mu) / self.y_sd).astype(np.float32)).to(self.dev)
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
    def predict(self, feats: np.ndarray) -> np.ndarray:
        """Profiles [N, n_points] in K (bottom first) for features [N, 6]."""
        torch = _torch()
        X = torch.from_numpy(((np.asarray(feats, np.float64) - self.x_mu) / self.x_sd).astype(np.float32)).to(self.dev)
        out = []
        for s in range(0, X.shape[0], self.net.max_batch):
            out.append(self.net.forward(X[s:s + self.net.max_batch]).double().cpu().numpy())
        return np.concatenate(out) * self.y_sd + self.y_mu

    def initial_profiles(self, feats, n_layers, fallback, T_min=50.0, T_max=8000.0):
        """Start profiles for atmospheres of n_layers[i] layers: the predicted profile interpolated
        linearly in the normalised log-P coordinate, or fallback[i] (the isothermal start) when the
        prediction is not finite or leaves [T_min, T_max].  Returns (profiles, used_prediction)."""
        pred = self.predict(feats)
        s_out = np.linspace(0.0, 1.0, self.n_points)
        profiles, used = [], []
        for i, n in enumerate(n_layers):
            T = np.interp(np.linspace(0.0, 1.0, n), s_out, pred[i])
            ok = bool(np.all(np.isfinite(T)) and T.min() > T_min and T.max() < T_max)
            profiles.append(T if ok else np.asarray(fallback[i], np.float64))
            used.append(ok)
        return profiles, np.array(used)


def features(atms) -> np.ndarray:
    """[T_irr, T_int, log10 g (m s^-2), [M/H], C/O, log10 mean kappa] per atmosphere (from its generator
    parameters)."""
    return np.array([[a.params["T_irr"], a.params["T_int"], a.params["log10g"], a.params["MH"], a.params["CO"],
                      a.params["log10_mean_kappa"]] for a in atms], dtype=np.float64)
