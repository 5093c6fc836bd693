"""Multi-rank logic on CPU (gloo, world size 2): point partition, the all-reduce of partial
boundary adjoints (at fixed lambda and through the lambda search), and the all-gather of
per-point solve results, with the FP64 oracle standing in for each rank's GPU compute."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1306_1122_gb300.shard import partition, sharded_solve, sharded_vjp
    rng = np.random.default_rng(0)
    nx, ny = 12, 9
    g = oracle.Grid(nx, ny)
    bd = oracle.Boundary(g, *(rng.normal(0, 50, (ny, nx)).astype(np.float32) for _ in range(3)))
    n = 23
    xyz = torch.from_numpy(np.stack([rng.uniform(0, 11, n), rng.uniform(0, 8, n),
                                     rng.uniform(0.5, 5, n)], 1))
    lam = torch.from_numpy(rng.uniform(-0.3, 0.3, (n, 3)))
    gB = torch.from_numpy(rng.normal(0, 1, (n, 3)))

    def vjp_fn(x, l, gb):
        return torch.from_numpy(oracle.vjp(bd, x.numpy(), l.numpy(), gb.numpy(), nthreads=1))

    full = sharded_vjp(vjp_fn, xyz, lam, gB)
    ref = oracle.vjp(bd, xyz.numpy(), lam.numpy(), gB.numpy(), nthreads=1)

    # the gradient through the lambda search is a sum over points too: same all-reduce
    def ivjp_fn(x, l, gb):
        return torch.from_numpy(oracle.implicit_vjp(bd, x.numpy(), l.numpy(), gb.numpy(),
                                                    1.0 / 6.0, nthreads=1)[0])

    ifull = sharded_vjp(ivjp_fn, xyz, lam, gB)
    iref = oracle.implicit_vjp(bd, xyz.numpy(), lam.numpy(), gB.numpy(), 1.0 / 6.0, nthreads=1)[0]
    ierr = float(np.abs(ifull.numpy() - iref).max() / np.abs(iref).max())

    def solve_fn(x):
        r = oracle.solve(bd, x.numpy(), oracle.Options(max_iter=8), nthreads=1)
        return {"lam": torch.from_numpy(r["lam"]), "B": torch.from_numpy(r["B"]),
                "iters": torch.from_numpy(r["iters"])}

    sol = sharded_solve(solve_fn, xyz)
    sref = oracle.solve(bd, xyz.numpy(), oracle.Options(max_iter=8), nthreads=1)
    q.put((rank, max(float(np.abs(full.numpy() - ref).max() / np.abs(ref).max()), ierr),
           bool(np.array_equal(sol["lam"].numpy(), sref["lam"])),
           bool(np.array_equal(sol["iters"].numpy(), sref["iters"])),
           partition(n, world)))
    dist.destroy_process_group()


def test_partition_balanced():
    from paper_1306_1122_gb300.shard import partition
    assert partition(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert partition(0, 2) == [(0, 0), (0, 0)]
    p = partition(6, 2, weights=[1, 1, 1, 1, 4, 4])
    assert p[0][0] == 0 and p[-1][1] == 6 and p[0][1] == p[1][0]


def test_two_rank_adjoint_and_solve_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, err, lam_eq, it_eq, parts in res:
        assert err < 1e-12, err           # summed partial adjoints == full adjoint
        assert lam_eq and it_eq           # gathered per-point results == unsharded solve
        assert parts == [(0, 12), (12, 23)]
