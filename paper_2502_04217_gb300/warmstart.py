"""Training and use of the learned warm start (a 3D conv network over the slot
grid, see include/sdft_ipm.h, "learned warm start").

Everything numerical runs in the CUDA library: the instances are drawn by the
seeded generator, solved by the library's own IPM (the targets are its
solutions), and the network is trained by the library's forward/backward
kernels (``ws_train_step``).  This module only orchestrates.

    python -m paper_2502_04217_gb300.warmstart --side 128 --count 2000 --epochs 8 \
        --out paper_2502_04217_gb300/weights/warmstart.f32
"""

import argparse
import os
import time

import numpy as np

from . import binding
from .synth import lattice_mask, make_problem

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "weights", "warmstart.f32")
# mu0 = MU_SCALE lambda^2 of the predicted start point, chosen on held-out 512^3
# instances (1 to 5 of the 512^3 workload; mixed precision, 1e-6 gap, the library's
# defaults): of {0.1, 0.2, 0.3, 0.5, 0.8} every value takes 6 IPM iterations (the cold
# start 8 to 10), and 0.3 the fewest PCG iterations (18 on three of the five instances,
# 19 on the others; the rest 19 to 20).
MU_SCALE = 0.3

# (stored cin, stored cout, real cin, real cout) of the four convolutions
LAYERS = [(16, 32, 8, 32), (32, 32, 32, 32), (32, 32, 32, 32), (32, 8, 32, 4)]


def instance(side, i, seed=0):
    """Instance i of the training distribution: a side^3 grid drawn like the
    256^3 / 512^3 workloads (0.25 % occupied frequencies at 128^3 scale,
    noise 0.01, Bragg-ball mask with random period 8..16, radius 1..2 and offsets)."""
    dims = (side,) * 3
    k = max(1, round(100000 * side ** 3 / 512 ** 3))
    w = make_problem("custom", dims=dims, k=k, missing=0.0, noise=0.01, seed=50000 + seed + i)
    rng = np.random.default_rng(90000 + seed + i)
    per = int(rng.integers(8, 17))
    rad = int(rng.integers(1, 3))
    w.mask = lattice_mask(dims, per, rad * rad, rng.integers(0, per, size=3))
    w.lam_rel = 0.05
    return w


class Dataset:
    """Instances on the host and their IPM solutions on the device; one handle
    per grid shape is reused for every instance (ipm_set_problem)."""

    def __init__(self, side, count, seed=0, gap_tol=1e-8, stream=None, log=None):
        import torch
        self.side = side
        self.items = []
        opt = binding.default_options(precision=binding.IPM_MIXED, lambda_relative=1, gap_tol=gap_tol)
        self.h = None
        for i in range(count):
            w = instance(side, i, seed)
            if self.h is None:
                self.h = binding.ipm_create(w.dims, w.mask, w.y, w.lam_rel, opt, stream=stream)
            else:
                binding.ipm_set_problem(self.h, w.mask, w.y, w.lam_rel)
            res = binding.ipm_solve(self.h)
            H, n = binding.ipm_sizes(self.h)
            pt = [torch.empty(2 * H, dtype=torch.float64, device="cuda") for _ in range(6)]
            binding.ipm_get_point(self.h, pt)
            self.items.append((w, pt[0], res))
            if log and (i + 1) % max(1, count // 10) == 0:
                log(f"solved {i + 1}/{count}: {res['ipm_iters']} IPM iterations")

    def load(self, i):
        w, bstar, _ = self.items[i]
        binding.ipm_set_problem(self.h, w.mask, w.y, w.lam_rel)
        return bstar

    def close(self):
        if self.h is not None:
            binding.ipm_destroy(self.h)
            self.h = None


def train(net, data, epochs, lr=1e-3, seed=0, log=None):
    """Adam over shuffled single instances; the learning rate decays linearly to
    a tenth of lr over the epochs (Adam alone showed occasional loss spikes)."""
    rng = np.random.default_rng(seed)
    hist = []
    for ep in range(epochs):
        lr_ep = lr * (1.0 - 0.9 * ep / max(1, epochs - 1))
        losses = []
        for i in rng.permutation(len(data.items)):
            bstar = data.load(int(i))
            losses.append(binding.ws_train_step(net, data.h, bstar, lr_ep))
        hist.append(float(np.mean(losses)))
        if log:
            log(f"epoch {ep}: mean loss {hist[-1]:.4g}")
    return hist


def save(net, path):
    p = np.empty(binding.ws_num_params(net), dtype=np.float32)
    binding.ws_get_params(net, p)
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    p.tofile(path)


def load(path=DEFAULT_WEIGHTS, seed=0, stream=None):
    net = binding.ws_create(seed=seed, stream=stream)
    p = np.fromfile(path, dtype=np.float32)
    if p.size != binding.ws_num_params(net):
        binding.ws_destroy(net)
        raise ValueError(f"{path}: {p.size} parameters, the network has {binding.ws_num_params(net)}")
    binding.ws_set_params(net, p)
    return net


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--side", type=int, default=128)
    ap.add_argument("--count", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    args = ap.parse_args()
    t0 = time.time()
    log = lambda m: print(f"[{time.time() - t0:7.1f} s] {m}", flush=True)
    data = Dataset(args.side, args.count, log=log)
    net = binding.ws_create(seed=1)
    try:
        train(net, data, args.epochs, args.lr, log=log)
        save(net, args.out)
        log(f"saved {args.out}")
    finally:
        binding.ws_destroy(net)
        data.close()


if __name__ == "__main__":
    main()
