"""The multi-GPU path of the benchmark on CPU: 'replicas only' (one FMM
evaluation has no exchange-free split, so every rank evaluates its own
instance and only the timing is combined).  Two gloo ranks exercise the
rank setup, the barrier and the max-over-ranks reduction that bench.py uses
under torchrun, and the per-rank instances differ."""
import multiprocessing as mp
import os
import socket
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    os.environ.update(WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W

    world, r, local, pg = bench.dist_setup(types.SimpleNamespace(impl="reference"))
    bench.barrier(pg)
    slowest = bench.max_over_ranks(pg, 1.0 + 0.5 * rank)  # this rank's "step time"
    w = W.uniform_random(1 << 10, 2 + rank, 2.0 / 32)     # the instance of this rank
    q.put((r, world, slowest, float(w.x[:8].sum())))
    pg.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[2] == 1.5 for o in out)  # every rank sees the max
    assert out[0][3] != out[1][3]         # independent instances (seed + rank)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench

    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        world, rank, local, pg = bench.dist_setup(types.SimpleNamespace(impl="ours"))
        assert (world, rank, local, pg) == (1, 0, 0, None)
        assert bench.max_over_ranks(None, 3.25) == 3.25
    finally:
        os.environ.update(env)


def test_near_field_peak_is_the_pipe_bound():
    """The near-field roofline: 8 FP32 lane operations, one ex2 and one rcp
    per pair (Eq. 6 in the 2^-q2 form), 6 issue slots with packed FP32 pairs,
    on 128 FP32 lanes, a MUFU pipe of 30 ex2 or 15 rcp lanes and 128 issue
    lanes per SM: the MUFU pipe binds at 1 / (1/30 + 1/15) = 10 pairs per SM
    per clock, 3146 Gpair/s at 2070 MHz on 152 SMs."""
    sys.path.insert(0, ROOT)
    import bench

    per_sm_clock = bench.p2p_peak_pairs_per_s(1.0) / (bench.N_SMS * 1e6)
    assert abs(per_sm_clock - 10.0) < 1e-12
    assert abs(bench.p2p_peak_pairs_per_s(2070.0) / 1e9 - 3146.4) < 1e-6
