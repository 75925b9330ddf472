"""Learned cardinality estimator on top of the cube (BF16 weights, FP32 accumulate).

The paper estimates a host's cardinality with Thm. 2 from the zero bits of
its union column.  In a cube whose arrays saturate, the estimate degrades;
this module trains a 16-64-64-1 network, on the GPU with libcbaa's own
forward / gradient / Adam kernels, to map what the cube shows about an
address (cbaa_host_features) to a correction y of ln(1 + Thm. 2 estimate):
the learned cardinality is exp(ln(1 + est) + y) - 1.  The last layer starts
at zero, so an untrained network reproduces Thm. 2 exactly.  Training pairs are
(features, exact cardinality) that the caller obtains from the same kind of
traffic (the exact baseline of Section V.A).  Thm. 2 stays the fallback:
cbaa_learned_decide uses it wherever the network output is not finite.

Marshalling only: features, forward, gradients, optimiser and decision all
run in libcbaa's kernels; torch supplies device memory.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import cbaa as C

IN, HID, N_PARAMS = 16, 64, 5313


def _ptr(t) -> int:
    return t.data_ptr()


def features(cube: "C.Cube", theta: int, ips, stream=None):
    """float32 [n, 16] device features of device uint32/int32 addresses ``ips``."""
    torch = C._torch()
    g = cube.geometry
    S, A = 1 << g["r"], g["n_ra"] + g["n_va"]
    dev = cube.memory.device
    za = torch.zeros(S * A, dtype=torch.int64, device=dev)
    eps = torch.zeros(S, dtype=torch.float64, device=dev)
    C._check(C.lib().cbaa_column_stats(cube.handle, theta, None, _ptr(za), _ptr(eps), None, C._stream_ptr(stream)),
             "column_stats")
    n = int(ips.numel())
    out = torch.empty((max(n, 1), IN), dtype=torch.float32, device=dev)
    C._check(C.lib().cbaa_host_features(cube.handle, _ptr(za), _ptr(eps), _ptr(ips), n, _ptr(out),
                                        C._stream_ptr(stream)), "host_features")
    return out[:n]


class LearnedEstimator:
    """The network's FP32 master weights, Adam moments and the BF16 copy the kernels read."""

    def __init__(self, device="cuda", seed: int = 0):
        torch = C._torch()
        gen = torch.Generator().manual_seed(seed)
        w1 = torch.randn(HID, IN, generator=gen) * math.sqrt(2.0 / IN)
        w2 = torch.randn(HID, HID, generator=gen) * math.sqrt(2.0 / HID)
        w3 = torch.zeros(HID)                     # start as the identity correction (y = 0)
        flat = torch.cat([w1.reshape(-1), torch.zeros(HID), w2.reshape(-1), torch.zeros(HID), w3, torch.zeros(1)])
        assert flat.numel() == N_PARAMS
        self.device = device
        self.master = flat.to(device=device, dtype=torch.float32).contiguous()
        self.m = torch.zeros_like(self.master)
        self.v = torch.zeros_like(self.master)
        self.wb = torch.zeros(N_PARAMS, dtype=torch.int16, device=device)
        self.grad = torch.zeros_like(self.master)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.step_count = 0
        C._check(C.lib().cbaa_mlp_to_bf16(_ptr(self.master), _ptr(self.wb), C._stream_ptr(None)), "mlp_to_bf16")

    # ------------------------------------------------------------------ kernels
    def predict(self, X):
        torch = C._torch()
        n = int(X.shape[0])
        y = torch.empty(max(n, 1), dtype=torch.float32, device=X.device)
        C._check(C.lib().cbaa_mlp_forward(_ptr(self.wb), _ptr(X), n, _ptr(y), C._stream_ptr(None)), "mlp_forward")
        return y[:n]

    def loss_grad(self, X, t, scale: float = 1.0):
        """(sum of squared errors, gradient of scale * SSE) at the current BF16 weights."""
        self.grad.zero_()
        self.loss.zero_()
        C._check(C.lib().cbaa_mlp_grad(_ptr(self.wb), _ptr(X), _ptr(t), int(X.shape[0]), ctypes.c_float(scale),
                                       _ptr(self.grad), _ptr(self.loss), C._stream_ptr(None)), "mlp_grad")
        return self.loss, self.grad

    def adam(self, lr: float = 1e-3, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
        self.step_count += 1
        C._check(C.lib().cbaa_mlp_adam(_ptr(self.master), _ptr(self.grad), _ptr(self.m), _ptr(self.v),
                                       _ptr(self.wb), ctypes.c_float(lr), ctypes.c_float(b1), ctypes.c_float(b2),
                                       ctypes.c_float(eps), self.step_count, C._stream_ptr(None)), "mlp_adam")

    def decide(self, y, X, log2_g: int, theta: float):
        torch = C._torch()
        n = int(y.numel())
        card = torch.empty(max(n, 1), dtype=torch.float32, device=y.device)
        dec = torch.empty(max(n, 1), dtype=torch.uint8, device=y.device)
        C._check(C.lib().cbaa_learned_decide(_ptr(y), _ptr(X), n, log2_g, ctypes.c_float(theta), _ptr(card),
                                             _ptr(dec), C._stream_ptr(None)), "learned_decide")
        return card[:n], dec[:n]

    # ------------------------------------------------------------------ training loop
    def train(self, X, t, epochs: int = 30, batch: int = 1 << 14, lr: float = 2e-3, seed: int = 0):
        """Mini-batch Adam on mean squared error; returns the mean loss of each epoch."""
        torch = C._torch()
        n = int(X.shape[0])
        gen = torch.Generator(device=X.device).manual_seed(seed)
        losses = []
        for ep in range(epochs):
            perm = torch.randperm(n, device=X.device, generator=gen)
            Xp, tp = X[perm].contiguous(), t[perm].contiguous()
            tot = 0.0
            for b0 in range(0, n, batch):
                xb, tb = Xp[b0:b0 + batch], tp[b0:b0 + batch]
                loss, _ = self.loss_grad(xb, tb, scale=1.0 / xb.shape[0])
                self.adam(lr=lr * (0.5 * (1 + math.cos(math.pi * ep / epochs))))
                tot += float(loss.item())
            losses.append(tot / n)
        return losses

    @staticmethod
    def balanced_indices(counts, seed: int = 0):
        """Training rows with every address of non-zero cardinality repeated so that the real hosts
        weigh as much as the phantoms (restored addresses that never appeared), which dominate the
        candidates of a saturated cube."""
        counts = np.asarray(counts)
        real = np.nonzero(counts > 0)[0]
        ph = np.nonzero(counts == 0)[0]
        rep = max(1, int(round(len(ph) / max(1, len(real)))))
        idx = np.concatenate([ph, np.repeat(real, rep)])
        np.random.default_rng(seed).shuffle(idx)
        return idx

    @staticmethod
    def target(X, counts):
        """Training target for exact cardinalities ``counts`` (device): ln(1 + c) - ln(1 + est), computed by
        cbaa_learned_target."""
        torch = C._torch()
        n = int(X.shape[0])
        c = counts.to(torch.float32).contiguous()
        t = torch.empty(max(n, 1), dtype=torch.float32, device=X.device)
        C._check(C.lib().cbaa_learned_target(_ptr(X), _ptr(c), n, _ptr(t), C._stream_ptr(None)), "learned_target")
        return t[:n]

    @staticmethod
    def training_set(cand_ips, cand_counts, ips, counts, n_samples: int, seed: int = 0):
        """Addresses (uint32) and exact cardinalities for training, n_samples of them: up to half are the
        candidates the detector restores at its looser bound, the real hosts among them repeated to
        weigh as much as the phantoms (which dominate the candidates of an undersized cube); the rest
        are present sources drawn in equal numbers from each octave of cardinality -- stratified, so
        the octaves around theta weigh as much as the crowded low ones."""
        cand_ips = np.asarray(cand_ips, dtype=np.uint32)
        cand_counts = np.asarray(cand_counts, dtype=np.int64)
        ips = np.asarray(ips, dtype=np.uint32)
        counts = np.asarray(counts, dtype=np.int64)
        bal = LearnedEstimator.balanced_indices(cand_counts, seed)[: n_samples // 2]
        take_ips, take_cnt = [cand_ips[bal]], [cand_counts[bal]]
        room = n_samples - bal.size
        keep = ~np.isin(ips, cand_ips) & (counts > 0)
        ips, counts = ips[keep], counts[keep]
        octave = np.floor(np.log2(np.maximum(counts, 1))).astype(np.int64)
        groups = [np.nonzero(octave == b)[0] for b in np.unique(octave)]
        rng = np.random.default_rng(seed)
        groups.sort(key=len)                      # small octaves first: what they cannot fill, others get
        for k, grp in enumerate(groups):
            quota = room // (len(groups) - k)
            pick = grp if grp.size <= quota else rng.choice(grp, size=quota, replace=False)
            take_ips.append(ips[pick])
            take_cnt.append(counts[pick])
            room -= pick.size
        return np.concatenate(take_ips), np.concatenate(take_cnt)

    @staticmethod
    def choose_threshold(card, counts, theta: float, max_fnr: float | None = None, factors=None) -> float:
        """Decision threshold factor f (decide card >= f theta), a margin chosen on the training window's
        candidates (Eq. 2, Eq. 3 over these addresses: H = cardinality >= theta): the f that minimises
        FNR + FPR, or with max_fnr the largest f whose FNR stays within max_fnr (fewer missed super
        hosts bought with more false positives)."""
        card = np.asarray(card, dtype=np.float64)
        counts = np.asarray(counts, dtype=np.float64)
        H = counts >= theta
        nH = max(1, int(H.sum()))
        grid = factors if factors is not None else np.exp(np.linspace(np.log(0.1), np.log(4.0), 81))
        best = (float("inf"), float(grid[0]))
        for f in grid:
            D = card >= f * theta
            fnr = np.count_nonzero(H & ~D) / nH
            if max_fnr is not None:
                if fnr <= max_fnr:
                    best = (0.0, float(f))                    # the grid ascends: keep the largest
                continue
            err = fnr + np.count_nonzero(D & ~H) / nH
            if err < best[0] - 1e-12:
                best = (err, float(f))
        return best[1]

    def weights_bf16(self) -> np.ndarray:
        return self.wb.cpu().numpy().view(np.uint16).copy()
