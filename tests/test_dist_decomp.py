"""The phi-slab decomposition of the method (oracle/decomp.py) on CPU ranks (gloo, world sizes 2
and 4) against the single-rank oracle: RKL2 + PTL and BE + PCG under PTL cycling, for conduction
and viscosity.  The decomposed STS + PTL run must reproduce the single-rank schedule (cycle
lengths, stage counts, the PTL location k) and state exactly: the halo makes every owned point's
F the single-rank value, and the reductions that decide (max, MAXLOC, min) are exact.  PCG sums
its dot products in another order, so fixed-iteration BE agrees to 1e-13 and converged BE to the
solver tolerance, with the same schedule and iteration counts within one."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from gpu_common import tc_problem, visc_problem
from oracle import advance

CASES = [("tc", (16, 12, 16)), ("visc", (12, 10, 8))]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem(kind, shape):
    return tc_problem(*shape, noise=0.05) if kind == "tc" else visc_problem(*shape)


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import decomp
    res = {}
    for kind, shape in CASES:
        g, inp, op, u = _problem(kind, shape)
        so = decomp.SlabOperator(op, rank, world)
        dt = 100.0 * so.dt_explicit()
        uo, log = decomp.sts_advance(so, so.take(u), dt)
        res[(kind, "sts")] = (so.gather(uo).tobytes(), log.dt_c, log.s, log.k)
        uo, log = decomp.be_advance(so, so.take(u), dt, use_ptl=False, fixed_iters=25)
        res[(kind, "be_fixed")] = (so.gather(uo).tobytes(), log.dt_c, log.iters, log.k)
        uo, log = decomp.be_advance(so, so.take(u), dt, use_ptl=True, rtol=1e-10)
        res[(kind, "be_ptl")] = (so.gather(uo).tobytes(), log.dt_c, log.iters, log.k)
        res[(kind, "dtE")] = so.dt_explicit()
    if rank == 0:
        out.update(res)
    dist.barrier()
    dist.destroy_process_group()


@pytest.fixture(scope="module", params=[2, 4])
def decomposed(request):
    world = request.param
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
        return world, dict(out)


@pytest.mark.parametrize("kind,shape", CASES)
def test_decomposed_sts_ptl_equals_single_rank(decomposed, kind, shape):
    world, res = decomposed
    g, inp, op, u = _problem(kind, shape)
    assert res[(kind, "dtE")] == op.dt_explicit()
    dt = 100.0 * op.dt_explicit()
    uo, log = advance.sts_advance(op, u, dt)
    got, dt_c, s, k = res[(kind, "sts")]
    assert log.cycles > 1
    assert dt_c == log.dt_c and s == log.s and k == log.k
    np.testing.assert_array_equal(np.frombuffer(got), uo)


@pytest.mark.parametrize("kind,shape", CASES)
def test_decomposed_be_pcg(decomposed, kind, shape):
    world, res = decomposed
    g, inp, op, u = _problem(kind, shape)
    dt = 100.0 * op.dt_explicit()
    uo, _ = advance.be_advance(op, u, dt, use_ptl=False, fixed_iters=25)
    got = np.frombuffer(res[(kind, "be_fixed")][0])
    assert np.linalg.norm(got - uo) <= 1e-13 * np.linalg.norm(uo)
    uo, log = advance.be_advance(op, u, dt, use_ptl=True, rtol=1e-10)
    got, dt_c, iters, k = res[(kind, "be_ptl")]
    assert len(dt_c) == log.cycles and k == log.k
    np.testing.assert_allclose(dt_c, log.dt_c, rtol=1e-12)
    assert all(abs(a - b) <= 1 for a, b in zip(iters, log.iters))
    assert np.linalg.norm(np.frombuffer(got) - uo) <= 1e-9 * np.linalg.norm(uo)


def test_slab_partition_covers_every_plane_once():
    from oracle.decomp import slab
    for n_phi in (3, 8, 13, 64):
        for world in (1, 2, 3, 4):
            if world > n_phi:
                continue
            planes = [k for r in range(world) for k in range(*slab(n_phi, r, world))]
            assert planes == list(range(n_phi))
            sizes = [slab(n_phi, r, world)[1] - slab(n_phi, r, world)[0] for r in range(world)]
            assert max(sizes) - min(sizes) <= 1
