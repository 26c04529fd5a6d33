"""Learned warm start: train the network on factors the solver produces, then compare starts.

Orchestration only: every numerical step (kernel matrix aside, which is input
generation) is a call into the CUDA library: the range finder gives the
sketch X Omega with one Omega shared by all instances (fixed Philox key), the
LAI solver gives converged factors H*, and the network's forward / backward /
Adam steps are the library's kernels.

Instances follow the warm-start workload: n points of a c-component Gaussian
mixture in R^d with Dirichlet(1) weights, X = exp(-||x_i - x_j||^2 / sigma^2),
sigma the median pairwise distance.
"""

from __future__ import annotations

import time

import numpy as np
import torch

from . import MLP, SRC_LAI, SRC_X, Solver, gaussian

OMEGA_SEED = 0x5EED0F0E6A


def instance_points(n, d, c, seed):
    """The seeded points of one instance and its kernel width (host side, numpy)."""
    from synth import gmm_points, median_pair_distance

    pts, labels = gmm_points(n, d, c, seed=seed, weights="dirichlet")
    return pts, median_pair_distance(pts, seed=seed), labels


def instance_matrix(pts, sigma, device, math_dtype=None):
    """(X float32, X bfloat16 padded to 8 columns) of one instance on the device."""
    from synth import kernel_matrix_torch

    n = pts.shape[0]
    Xf = kernel_matrix_torch(pts, sigma, device, math_dtype=math_dtype)
    ld = (n + 7) // 8 * 8
    Xb = torch.zeros((n, ld), dtype=torch.bfloat16, device=device)
    Xb[:, :n] = Xf.to(torch.bfloat16)
    return Xf, Xb


def make_instance(n, d, c, seed, device, math_dtype=None):
    """Kernel matrix of one seeded instance on the device: (X float32, X bfloat16 padded to 8 columns).

    Distances are formed in `math_dtype` (default float64, as the oracle forms them; float32 is
    enough for training instances and much faster on this part's FP64 units)."""
    pts, sigma, labels = instance_points(n, d, c, seed)
    Xf, Xb = instance_matrix(pts, sigma, device, math_dtype)
    return Xf, Xb, labels


def training_set(n, d, c, k, l, q, sweeps, seeds, omega, device, math_dtype=None, workers=8):
    """(features, H*) of every seed: the instance solved by the library (sketch with the shared
    Omega, LAI sweeps, 2 full-X sweeps).  The host draws the next instances' points on a thread
    pool while the device solves the current one."""
    from concurrent.futures import ThreadPoolExecutor

    data = []
    seeds = list(seeds)
    window = 2 * workers  # instances drawn ahead (bounded host memory)
    with ThreadPoolExecutor(max_workers=workers) as pool:
        futs = [pool.submit(instance_points, n, d, c, s) for s in seeds[:window]]
        for i, s in enumerate(seeds):
            if i + window < len(seeds):
                futs.append(pool.submit(instance_points, n, d, c, seeds[i + window]))
            pts, sigma, _ = futs[i].result()
            futs[i] = None
            Xf, Xb = instance_matrix(pts, sigma, device, math_dtype)
            sv, feats, _ = solve(Xb, Xf, k, l, q, sweeps, seed=s, omega=omega)
            H, _ = sv.factors()
            data.append((feats.clone(), H.clone()))
            sv.close()
            del Xf, Xb
    return data


def solve(Xb, Xf, k, l, q, sweeps, refine=2, seed=1, net=None, omega=None, record=False):
    """Sketch + LAI sweeps + full-X refinement; returns (solver, features, objectives).

    The start is the network's output on the sketch features when `net` is
    given, else the scaled Philox uniform start.
    """
    n = Xf.shape[0]
    s = Solver(Xb[:, :n] if Xb.shape[1] == n else Xb, k, max_width=l, seed=seed, x_hi=Xf)
    if omega is None:
        omega = gaussian(n, l, OMEGA_SEED)
    s.lai_sketch(l, q, omega)
    feats = s.sketch_features()
    if net is not None:
        net.warm_start(s, feats)
    else:
        s.init_random(True)
    objs = s.sweep(sweeps, source=SRC_LAI, record=record) if sweeps else None
    if refine:
        s.sweep(refine, source=SRC_X, record=False)
    return s, feats, objs


def sweeps_to_target(objs, target):
    """First sweep (1-based) whose objective is <= target, or None."""
    idx = np.nonzero(np.asarray(objs) <= target)[0]
    return int(idx[0]) + 1 if idx.size else None


def train(net, data, epochs, lr=1e-3, log=None):
    """Adam on (features, H*) pairs, one instance per step, shuffled each epoch."""
    rng = np.random.default_rng(0)
    for ep in range(epochs):
        order = rng.permutation(len(data))
        tot = 0.0
        for i in order:
            x, hs = data[i]
            tot += net.loss_grad(x, hs)
            net.adam(lr)
        if log is not None:
            log.append(tot / len(data))
    return net


def experiment(n=50000, d=64, c=32, k=32, l=74, q=2, sweeps=200, n_train=200, n_test=10, epochs=5,
               lr=1e-3, device="cuda", train_seeds=1000, test_seeds=0):
    """Train on `n_train` solved instances, compare warm vs random starts on `n_test` held-out ones.

    For each held-out instance, the target is the LAI objective the random start
    reaches after `sweeps` sweeps; reported are the sweeps and seconds each start
    needs to reach it, and both final residuals against X.
    """
    dev = torch.device(device)
    omega = gaussian(n, l, OMEGA_SEED)
    data = []
    t0 = time.time()
    for i in range(n_train):
        Xf, Xb, _ = make_instance(n, d, c, train_seeds + i, dev)
        s, feats, _ = solve(Xb, Xf, k, l, q, sweeps, seed=train_seeds + i, omega=omega)
        H, _ = s.factors()
        data.append((feats.clone(), H.clone()))
        s.close()
        del Xf, Xb
    t_gen = time.time() - t0
    net = MLP((l, 256, 256, k), seed=7)
    losses = []
    t0 = time.time()
    train(net, data, epochs, lr, losses)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    rows = []
    for j in range(n_test):
        Xf, Xb, _ = make_instance(n, d, c, test_seeds + j, dev)
        res = {}
        for name, m in (("random", None), ("learned", net)):
            torch.cuda.synchronize()
            a = time.perf_counter()
            s, _, objs = solve(Xb, Xf, k, l, q, sweeps, refine=0, seed=test_seeds + j, net=m, omega=omega, record=True)
            torch.cuda.synchronize()
            el = time.perf_counter() - a
            nr, _ = s.residual(SRC_X)
            res[name] = dict(objs=np.asarray(objs), seconds=el, nr=nr)
            s.close()
        target = res["random"]["objs"][-1]
        row = {}
        for name in ("random", "learned"):
            sw = sweeps_to_target(res[name]["objs"], target * (1 + 1e-6))
            o = res[name]["objs"]
            row[name] = dict(sweeps_to_target=sw, obj0=float(o[0]), obj5=float(o[min(4, len(o) - 1)]),
                             obj10=float(o[min(9, len(o) - 1)]), obj_final=float(o[-1]), nr=res[name]["nr"],
                             seconds=res[name]["seconds"])
        rows.append(row)
        del Xf, Xb
    return dict(t_generate_solve=t_gen, t_train=t_train, losses=losses, rows=rows)
