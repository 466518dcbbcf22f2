"""Focal-field surrogate for parameter sweeps: data from the solver, training
and evaluation with the library's network kernels (psatd_fno_*).

Six pulse parameters (CEP, ellipticity, polarisation angle, f-number, cycles,
edge width) map to the real electric field (Ex, Ey, Ez) on a P^3 patch around
the focus at t = R0/c.  Training targets come from the one-shot solver path
(one exact step of T on the mapped grid of the f = 1 tight-focus geometry,
then P planes sampled from the held spectrum); the solver stays the judge of the
surrogate's error and the fallback for parameters outside the trained ranges.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import workloads as W

PARAM_NAMES = ("cep", "ellipticity", "pol_angle", "fnumber", "n_cycles", "eps")
RANGES = np.array([[0.0, 2 * math.pi], [0.0, 1.0], [0.0, math.pi], [1.0, 2.0], [1.5, 3.0], [0.1, 0.3]])


def sample_params(n: int, seed: int) -> np.ndarray:
    """n x 6 physical parameter values, uniform in RANGES (seeded PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random((n, len(PARAM_NAMES)))
    return RANGES[:, 0] + u * (RANGES[:, 1] - RANGES[:, 0])


def normalise(p: np.ndarray) -> np.ndarray:
    """Map physical parameters to [-1, 1]."""
    return (2 * (p - RANGES[:, 0]) / (RANGES[:, 1] - RANGES[:, 0]) - 1).astype(np.float32)


def in_range(p: np.ndarray) -> np.ndarray:
    """Rows inside the trained ranges (others go to the solver)."""
    return np.all((p >= RANGES[:, 0]) & (p <= RANGES[:, 1]), axis=1)


def pulse_for(p) -> tuple:
    """(PulseSpec, MappingSpec, T) of one parameter row on the f = 1 geometry."""
    lam = W.LAMBDA0
    cep, ell, psi, f, ncyc, eps = p
    R0 = 20 * lam
    L = 4.5 * ncyc * lam
    pulse = W.PulseSpec(kind=W.GAUSSIAN, lam=lam, theta=math.atan(1.0 / (2.0 * f)), eps=float(eps), P0=1e7,
                        n_cycles=float(ncyc), cep=float(cep), ellipticity=float(ell), pol_angle=float(psi),
                        div_project=1)
    return pulse, W.MappingSpec(R0, L), R0 / W.C_CGS


class SolverPatch:
    """Solver side: focal patch [3][P][P][P] (z, y, x) of Re E at t = R0/c."""

    def __init__(self, N: int = 128, patch: int = 64, half_width_lam: float = 2.0, precision: int = 32):
        import torch
        from . import psatd
        g, m, _, n_steps, _ = W.tight_focus_workload(N=N)
        self.grid, self.P = g, patch
        self.ctx = psatd.Context(g, m, (m.R0 / g.c) / n_steps, precision)
        h = half_width_lam * W.LAMBDA0
        self.h = h
        self.xs = -h + 2 * h * np.arange(patch) / patch
        dt = torch.complex64 if precision == 32 else torch.complex128
        self.plane = torch.empty((3, patch, patch), dtype=dt, device="cuda")

    def __call__(self, p, out):
        """Fill out[3][P][P][P] (float32 CUDA) for parameter row p."""
        pulse, mapping, T = pulse_for(p)
        P, h = self.P, self.h
        self.ctx.set_mapping(mapping)
        self.ctx.focal_one_shot(pulse, T, float(self.xs[0]), P, P, -h, h, -h, h, comps=(0, 1, 2), out=self.plane)
        out[:, :, :, 0] = self.plane.real
        for i in range(1, P):
            self.ctx.sample_focal_plane(float(self.xs[i]), P, P, -h, h, -h, h, comps=(0, 1, 2), out=self.plane)
            out[:, :, :, i] = self.plane.real

    def close(self):
        self.ctx.close()


def make_dataset(n: int, seed: int, N: int = 128, patch: int = 64):
    """Parameters (normalised, CUDA) and solver patches (CUDA float32), plus the
    solver's time per sample in seconds."""
    import torch
    phys = sample_params(n, seed)
    sp = SolverPatch(N, patch)
    tgt = torch.empty((n, 3, patch, patch, patch), dtype=torch.float32, device="cuda")
    sp(phys[0], tgt[0])                                       # warm-up (tables, buffers)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(n):
        sp(phys[i], tgt[i])
    torch.cuda.synchronize()
    t_solver = (time.perf_counter() - t0) / n
    sp.close()
    prm = torch.tensor(normalise(phys), device="cuda")
    return phys, prm, tgt, t_solver


def train(net, prm, tgt, steps: int, batch: int, lr: float, seed: int = 0, log_every: int = 0):
    """Adam on the mean squared error; learning rate decays linearly to lr/10."""
    import torch
    n = prm.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    order = rng.permutation(n)
    hist = []
    pos = 0
    for it in range(steps):
        if pos + batch > n:
            order = rng.permutation(n)
            pos = 0
        idx = torch.tensor(order[pos:pos + batch], device="cuda")
        pos += batch
        loss = net.loss_backward(prm.index_select(0, idx).contiguous(), tgt.index_select(0, idx).contiguous(),
                                 want_loss=(log_every and it % log_every == 0) or it == steps - 1)
        if loss is not None:
            hist.append((it, loss))
        net.adam_step(lr * (1 - 0.9 * it / max(steps - 1, 1)))
    return hist


def evaluate(net, prm, tgt, batch: int, repeats: int = 5):
    """Per-sample relative L2 error of the surrogate against the solver patch,
    and the surrogate's inference time per sample in seconds (forward passes
    only, CUDA events on the model's stream, after one warm-up pass)."""
    import torch
    n = prm.shape[0]
    errs = []
    for s in range(0, n, batch):
        k = min(batch, n - s)
        out = net.forward(prm[s:s + k].contiguous())
        d = (out - tgt[s:s + k]).flatten(1).norm(dim=1) / tgt[s:s + k].flatten(1).norm(dim=1)
        errs.append(d.clone())
    chunks = [prm[s:s + batch].contiguous() for s in range(0, n, batch)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(net.stream)
    for _ in range(repeats):
        for c in chunks:
            net.forward(c)
    e1.record(net.stream)
    torch.cuda.synchronize()
    return torch.cat(errs).cpu().numpy(), e0.elapsed_time(e1) / 1e3 / (n * repeats)


def study(n_train: int = 2000, n_test: int = 200, N: int = 128, patch: int = 64, width: int = 32, layers: int = 4,
          modes: int = 12, hidden: int = 64, batch: int = 8, steps: int = 4000, lr: float = 2e-3, seed: int = 0):
    """Solver-generated data set, training and held-out evaluation; returns a
    summary dict (errors relative L2 over the patch, times per focal patch)."""
    import torch
    from . import psatd
    t0 = time.perf_counter()
    phys, prm, tgt, t_solver = make_dataset(n_train + n_test, seed, N, patch)
    t_data = time.perf_counter() - t0
    scale = tgt.abs().amax()
    tgt /= scale
    net = psatd.Fno(len(PARAM_NAMES), width=width, layers=layers, patch=patch, modes=modes, hidden=hidden,
                    out_channels=3, max_batch=batch, seed=seed)
    t0 = time.perf_counter()
    hist = train(net, prm[:n_train], tgt[:n_train], steps, batch, lr, seed=seed + 1, log_every=max(steps // 20, 1))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    errs, t_net = evaluate(net, prm[n_train:], tgt[n_train:], batch)
    mean = tgt[:n_train].mean(0, keepdim=True)
    base = ((mean - tgt[n_train:]).flatten(1).norm(dim=1) / tgt[n_train:].flatten(1).norm(dim=1)).cpu().numpy()
    net.close()
    return {"n_train": n_train, "n_test": n_test, "grid": N, "patch": patch, "width": width, "layers": layers,
            "modes": modes, "hidden": hidden, "batch": batch, "steps": steps,
            "rel_l2_mean": float(errs.mean()), "rel_l2_median": float(np.median(errs)),
            "rel_l2_p90": float(np.quantile(errs, 0.9)), "mean_field_rel_l2": float(base.mean()),
            "solver_s_per_patch": t_solver, "surrogate_s_per_patch": t_net,
            "speedup": t_solver / t_net, "data_s": t_data, "train_s": t_train,
            "loss_history": [(int(i), float(v)) for i, v in hist]}


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description=study.__doc__)
    for k, v in (("n_train", 2000), ("n_test", 200), ("N", 128), ("patch", 64), ("width", 32), ("layers", 4),
                 ("modes", 12), ("hidden", 64), ("batch", 8), ("steps", 4000), ("seed", 0)):
        ap.add_argument("--" + k.replace("_", "-"), type=int, default=v)
    ap.add_argument("--lr", type=float, default=2e-3)
    a = ap.parse_args()
    print(json.dumps(study(**vars(a))))
