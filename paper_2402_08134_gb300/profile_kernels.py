"""Run one kernel family of the library on a seeded synthetic case (for profilers such as ncu).

    python -m paper_2402_08134_gb300.profile_kernels xf_tc --n 16384 --width 50
    python -m paper_2402_08134_gb300.profile_kernels lai_engine --n 20000 --k 20 --l 50 --sweeps 10
    python -m paper_2402_08134_gb300.profile_kernels lai_engine_u --n 50000 --k 32 --l 74 --sweeps 10
    python -m paper_2402_08134_gb300.profile_kernels sketch_u --n 50000 --l 74
    python -m paper_2402_08134_gb300.profile_kernels csr_sweep --n 200000 --k 64
    python -m paper_2402_08134_gb300.profile_kernels lvs --n 200000 --k 64
    python -m paper_2402_08134_gb300.profile_kernels batched --nprob 16

Each case runs `--reps` times after one warm-up and prints a one-line summary.
Sweeps run without graph replay so that every kernel is a separate launch.
"""

from __future__ import annotations

import argparse
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["xf_tc", "xf_fp8", "xf_simt", "lai_engine", "lai_kernels", "full_sweep",
                                     "lai_engine_u", "sketch_u", "csr_sweep", "lvs", "batched", "mlp"])
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--k", type=int, default=20)
    ap.add_argument("--l", type=int, default=50)
    ap.add_argument("--width", type=int, default=50)
    ap.add_argument("--sweeps", type=int, default=10)
    ap.add_argument("--nprob", type=int, default=16)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--time", action="store_true", help="print the mean time per run (CUDA events)")
    a = ap.parse_args(argv)

    import torch

    import paper_2402_08134_gb300 as S

    dev = torch.device("cuda:0")
    g = torch.Generator(device=dev).manual_seed(0)
    n = a.n
    out = None
    if a.case in ("xf_tc", "xf_fp8", "xf_simt"):
        Xf = torch.rand((n, n), device=dev, generator=g)
        F = torch.rand((n, a.width), device=dev, generator=g)
        if a.case == "xf_tc":
            X = Xf.to(torch.bfloat16)
            del Xf
            run = lambda: S.dense_xf(X, F, gemm=S.GEMM_TC)  # noqa: E731
        elif a.case == "xf_fp8":
            x8, rs = S.quantize_fp8(Xf)
            del Xf
            run = lambda: S.dense_xf(x8, F, row_scale=rs, gemm=S.GEMM_TC)  # noqa: E731
        else:
            run = lambda: S.dense_xf(Xf, F, gemm=S.GEMM_SIMT)  # noqa: E731
    elif a.case in ("lai_engine", "lai_kernels", "full_sweep"):
        from synth import gmm_points, kernel_matrix_torch, median_pair_distance

        pts, _ = gmm_points(n, 50, 20, seed=0)
        Xf = kernel_matrix_torch(pts, median_pair_distance(pts, seed=0), dev)
        Xb = Xf.to(torch.bfloat16)
        s = S.Solver(Xb, a.k, max_width=a.l, seed=1, x_hi=Xf, use_graph=False,
                     lai_mode=(0 if a.case == "lai_engine" else 1))
        s.init_random(True)
        s.lai_sketch(a.l, 2)
        if a.case == "full_sweep":
            run = lambda: s.sweep(a.sweeps, source=S.SRC_X, record=False)  # noqa: E731
        else:
            run = lambda: s.sweep(a.sweeps, source=S.SRC_LAI, record=False)  # noqa: E731
    elif a.case in ("lai_engine_u", "sketch_u"):
        # the sweeps and the range finder's orthonormalisation on a tiny identity X (CSR): a random
        # orthonormal U (given through set_lai) for the sweeps, X Omega = Omega for the sketch
        rp = torch.arange(n + 1, device=dev, dtype=torch.int64)
        col = torch.arange(n, device=dev, dtype=torch.int32)
        val = torch.ones(n, device=dev, dtype=torch.float32)
        s = S.Solver(csr=(rp, col, val), k=a.k, n=n, max_width=a.l, seed=1, use_graph=False, alpha=1.0)
        if a.case == "sketch_u":
            run = lambda: s.lai_sketch(a.l, 2)  # noqa: E731
        else:
            import numpy as np

            Q, _ = np.linalg.qr(np.random.default_rng(0).standard_normal((n, a.l)))
            lam = [50.0 * 0.9 ** i for i in range(a.l)]
            s.set_lai(torch.tensor(Q, dtype=torch.float32, device=dev), lam)
            s.set_factors(torch.rand((n, a.k), device=dev, generator=g) * 0.1)
            run = lambda: s.sweep(a.sweeps, source=S.SRC_LAI, record=False)  # noqa: E731
    elif a.case in ("csr_sweep", "lvs"):
        from synth import lvs_sample_count, sbm_csr

        gr = sbm_csr(n=n, c=64, avg_deg=30, ratio=20, seed=0)
        rp = torch.tensor(gr["row_ptr"], device=dev)
        col = torch.tensor(gr["col"], device=dev)
        val = torch.tensor(gr["val"], device=dev)
        s = S.Solver(csr=(rp, col, val), k=a.k, n=n, seed=3, use_graph=False)
        s.init_random(True)
        sc = lvs_sample_count(a.k)
        if a.case == "lvs":
            run = lambda: s.lvs_iterate(1, 1.0 / sc, sc)  # noqa: E731
        else:
            run = lambda: s.sweep(1, record=False)  # noqa: E731
    elif a.case == "batched":
        from synth import batched_problem_specs

        specs = batched_problem_specs(a.nprob, seed=0)
        Xs = []
        for p, sp_ in enumerate(specs):
            m = sp_["n"]
            A = torch.rand((m, m), device=dev, generator=torch.Generator(device=dev).manual_seed(p))
            lab = torch.arange(m, device=dev) % sp_["k"]
            P = torch.where(lab[:, None] == lab[None, :], 0.3, 0.015)
            M = torch.triu(A < P, 1)
            M = M | M.T
            M.fill_diagonal_(True)
            ld = (m + 7) // 8 * 8
            buf = torch.zeros((m, ld), dtype=torch.bfloat16, device=dev)
            buf[:, :m] = M.to(torch.bfloat16)
            Xs.append(buf)
        b = S.Batch(Xs, [sp_["k"] for sp_ in specs], restarts=4)
        b.init_random(True)
        run = lambda: b.sweep(1, record=False)  # noqa: E731  (one eager sweep: no graph replay)
    else:  # mlp
        net = S.MLP((a.l, 256, 256, a.k), seed=0)
        x = torch.rand((n, a.l), device=dev, generator=g)
        Hs = torch.rand((n, a.k), device=dev, generator=g)
        run = lambda: (net.loss_grad(x, Hs), net.adam(1e-3))  # noqa: E731
    run()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(a.reps):
        out = run()
    t1.record()
    torch.cuda.synchronize()
    if a.time:
        print(f"{a.case} n={n} k={a.k}: {t0.elapsed_time(t1) * 1e3 / max(a.reps, 1):.0f} us per run", flush=True)
    print(f"{a.case} n={n} done ({type(out).__name__}); launches={S.launch_count()}", flush=True)
    return 0 if math.isfinite(0.0) else 1


if __name__ == "__main__":
    sys.exit(main())
