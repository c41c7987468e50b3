"""Multi-process paths on CPU with the gloo backend, world size 2.

1. The replica aggregation used by bench.py under torchrun: the job time is the
   slowest rank's and the throughput counts every rank's cells.
2. A strip decomposition of one periodic grid over two ranks that exchange halos of
   4 rows (two RK stages of stencil radius 2) by point-to-point messages before each
   step, with the CPU oracle as the per-strip stepper: the result must equal the
   undivided run bit for bit (each cell's arithmetic only sees its stencil).
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

HALO = 4


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _replica_worker(rank, world, port, q):
    dist = _init(rank, world, port)
    from paper_2502_16818_gb300 import replicas
    ms = [12.0, 17.5][rank]
    m = replicas.max_over_ranks(ms)
    v = replicas.job_throughput(1000.0, world, m * 1e-3)
    q.put((rank, m, v))
    dist.destroy_process_group()


def test_replica_timing_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in out:
        assert m == 17.5
        assert v == pytest.approx(1000.0 * 2 / 17.5e-3)


def _strip_worker(rank, world, port, steps, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    dist = _init(rank, world, port)
    import oracle
    from paper_2502_16818_gb300 import workloads as W
    w = W.random_blocks(24, 20, seed=7, dt=4e-4, tau=1e-3)          # periodic both axes
    rows = np.array_split(np.arange(w.ny), world)[rank]
    lo, hi = rows[0], rows[-1] + 1
    nloc = hi - lo
    m_full = oracle.Model(nx=w.nx, ny=w.ny, dx=w.dx, dy=w.dy, dt=w.dt, tau=w.tau, I=w.I, vg=w.vg, eg=w.eg,
                          threads=1)
    f_full = oracle.init(m_full, w.rho, w.ux, w.uy, w.T)
    f = np.ascontiguousarray(f_full[:, lo:hi, :])                    # this rank's strip
    m_pad = oracle.Model(nx=w.nx, ny=nloc + 2 * HALO, dx=w.dx, dy=w.dy, dt=w.dt, tau=w.tau, I=w.I, vg=w.vg,
                         eg=w.eg, bc_x=0, bc_y=1, threads=1)
    up, down = (rank + 1) % world, (rank - 1) % world
    for _ in range(steps):
        # halo exchange: my top rows go up, my bottom rows go down
        top = torch.from_numpy(np.ascontiguousarray(f[:, -HALO:, :]))
        bot = torch.from_numpy(np.ascontiguousarray(f[:, :HALO, :]))
        from_down = torch.empty_like(top)
        from_up = torch.empty_like(bot)
        reqs = [dist.isend(top, up), dist.isend(bot, down), dist.irecv(from_down, down), dist.irecv(from_up, up)]
        for r in reqs:
            r.wait()
        pad = np.concatenate([from_down.numpy(), f, from_up.numpy()], axis=1)
        pad = oracle.step(m_pad, pad, 1)
        f = np.ascontiguousarray(pad[:, HALO:HALO + nloc, :])
    q.put((rank, lo, hi, f))
    dist.destroy_process_group()


def test_strip_decomposition_equals_undivided_run():
    import oracle
    from paper_2502_16818_gb300 import workloads as W
    steps = 6
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_strip_worker, args=(r, 2, port, steps, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = W.random_blocks(24, 20, seed=7, dt=4e-4, tau=1e-3)
    m = oracle.Model(nx=w.nx, ny=w.ny, dx=w.dx, dy=w.dy, dt=w.dt, tau=w.tau, I=w.I, vg=w.vg, eg=w.eg, threads=1)
    ref = oracle.step(m, oracle.init(m, w.rho, w.ux, w.uy, w.T), steps)
    got = np.concatenate([p[3] for p in parts], axis=1)
    assert np.array_equal(got, ref)
