"""Host logic of bench.py's multi-process (replica) path, on CPU ranks over gloo."""

import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    # each rank's step time; every rank must come out with the slowest one
    mine = 10.0 + 3.5 * rank
    got = bench.max_over_ranks(mine, w, torch.device("cpu"))
    dist.barrier()
    out[rank] = got
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_step_time_is_the_max_over_ranks(world):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert sorted(out.keys()) == list(range(world))
    assert all(v == 10.0 + 3.5 * (world - 1) for v in out.values())


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(7.25, 1, torch.device("cpu")) == 7.25


def test_reference_arm_runs_on_rank_zero_only():
    # a non-zero rank of a torchrun launch exits 0 at once, printing nothing
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


class _FakeLib:
    SRC_X, SRC_LAI, SRC_XHI = 0, 1, 2


class _FakeSolver:
    """Residual falls by a fixed factor per sweep; records what the driver asked for."""

    def __init__(self, nr0, rate):
        self.nr, self.rate, self.log = nr0, rate, []

    def init_random(self, scaled):
        self.log.append(("init", scaled))

    def lai_sketch(self, l, q, omega=None):
        self.log.append(("sketch", l, q))

    def sweep(self, m, source, record):
        self.log.append(("sweep", m, source))
        self.nr *= self.rate ** m

    def residual(self, src):
        self.log.append(("check", src))
        return self.nr, 0.0

    def sweep_to_target(self, target, *, source, check, chunk, max_sweeps):
        # the contract of symnmf_sweep_to_target: chunks of `chunk` (the last one cut to max_sweeps),
        # a check after each, stop after the first check at or below the target
        done = checks = 0
        nr = float("inf")
        while done < max_sweeps:
            m = min(chunk, max_sweeps - done)
            self.sweep(m, source, False)
            done += m
            nr = self.residual(check)[0]
            checks += 1
            if nr <= target:
                break
        return {"sweeps": done, "checks": checks, "nr": nr}


def test_solve_to_target_stops_at_the_first_check_below_target():
    sys.path.insert(0, ROOT)
    import bench

    s = _FakeSolver(1.0, 0.9)
    r = bench.solve_to_target(_FakeLib, s, 0.9 ** 35, _FakeLib.SRC_X, lai=True, refine_src=_FakeLib.SRC_X)
    # checks after 10, 20, 30, 40 LAI sweeps; 0.9^40 is the first at or below 0.9^35
    assert r["reached"] and r["sweeps"] == 40 and r["checks"] == 4 and r["refine_sweeps"] == 0
    assert s.log[:2] == [("init", True), ("sketch", bench.L, bench.Q)]
    assert all(e[2] == _FakeLib.SRC_LAI for e in s.log if e[0] == "sweep")


def test_solve_to_target_refines_with_full_x_when_lai_stalls():
    sys.path.insert(0, ROOT)
    import bench

    s = _FakeSolver(1.0, 1.0)  # the LAI sweeps make no progress
    r = bench.solve_to_target(_FakeLib, s, 0.5, _FakeLib.SRC_X, lai=True, refine_src=_FakeLib.SRC_X)
    assert r["sweeps"] == bench.SWEEPS and not r["reached"]
    assert r["refine_sweeps"] == bench.MAX_IR
    assert r["checks"] == bench.SWEEPS // bench.CHECK_EVERY + bench.MAX_IR // bench.IR_CHUNK
    refine = [e for e in s.log if e[0] == "sweep" and e[2] == _FakeLib.SRC_X]
    assert len(refine) == bench.MAX_IR // bench.IR_CHUNK
