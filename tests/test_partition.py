"""The split of one evaluation over ranks (contiguous Morton-key ranges of
leaves): the exchange plan's index sets against a brute-force enumeration
from the definitions of the local list and the interaction list (Sec.
3.3.1), and two gloo ranks that each plan their own side of the exchange and
agree with each other."""
import itertools
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_0809_1810_gb300 import partition as PT  # noqa: E402


def _xy(key):
    """Coordinates of a Morton key, bit by bit (independent of the module)."""
    ix = iy = 0
    for b in range(16):
        ix |= ((key >> (2 * b)) & 1) << b
        iy |= ((key >> (2 * b + 1)) & 1) << b
    return ix, iy


def _key(ix, iy):
    k = 0
    for b in range(16):
        k |= ((ix >> b) & 1) << (2 * b) | ((iy >> b) & 1) << (2 * b + 1)
    return k


def _owner(key, bounds):
    for r in range(len(bounds) - 1):
        if bounds[r] <= key < bounds[r + 1]:
            return r
    raise AssertionError(key)


def brute_force(bounds, L, reach):
    """{(q, r): (set of leaves, set of (level, box))} from the definitions."""
    R = len(bounds) - 1
    nleaf = 4 ** L
    out = {(q, r): (set(), set()) for q in range(R) for r in range(R) if q != r}
    for t in range(nleaf):
        r = _owner(t, bounds)
        tx, ty = _xy(t)
        # local list (and the cutoff ring): leaves within Chebyshev distance
        for s in range(nleaf):
            q = _owner(s, bounds)
            if q == r:
                continue
            sx, sy = _xy(s)
            if max(abs(sx - tx), abs(sy - ty)) <= reach:
                out[(q, r)][0].add(s)
        # interaction lists of the leaf's boxes at every level >= 2: children
        # of the parent's neighbours that are not neighbours of the box
        for level in range(2, L + 1):
            sh = L - level
            Tx, Ty = tx >> sh, ty >> sh
            side = 1 << level
            for Sx, Sy in itertools.product(range(side), repeat=2):
                if max(abs((Sx >> 1) - (Tx >> 1)), abs((Sy >> 1) - (Ty >> 1))) > 1:
                    continue
                if max(abs(Sx - Tx), abs(Sy - Ty)) < 2:
                    continue
                S = _key(Sx, Sy)
                lo, hi = S << (2 * sh), (S + 1) << (2 * sh)
                for q in {_owner(k, bounds) for k in range(lo, hi)}:
                    if q != r:
                        out[(q, r)][1].add((level, S))
    return out


def _as_sets(entry):
    leaves = set(int(k) for k in entry["leaves"])
    boxes = {(lev, int(k)) for lev, ks in entry["boxes"].items() for k in ks}
    return leaves, boxes


@pytest.mark.parametrize("L,R,reach,seed", [(3, 2, 1, 0), (3, 3, 2, 1), (4, 2, 1, 2),
                                            (4, 4, 2, 3), (2, 2, 1, 4)])
def test_exchange_plan_matches_brute_force(L, R, reach, seed):
    rng = np.random.default_rng(seed)
    counts = rng.poisson(5.0, 4 ** L)
    counts[rng.integers(0, 4 ** L, 4 ** L // 5)] = 0  # some empty leaves
    bounds = PT.leaf_bounds(counts, R)
    assert bounds[0] == 0 and bounds[-1] == 4 ** L and np.all(np.diff(bounds) >= 0)
    plan = PT.exchange_plan(bounds, L, reach)
    want = brute_force(bounds, L, reach)
    assert set(plan) == set(want)
    for key, entry in plan.items():
        assert _as_sets(entry) == want[key], key


def test_leaf_bounds_balance_particles():
    rng = np.random.default_rng(9)
    counts = rng.poisson(40.0, 4 ** 5)
    for R in (2, 3, 5):
        b = PT.leaf_bounds(counts, R)
        per = [counts[b[r]:b[r + 1]].sum() for r in range(R)]
        assert max(per) - min(per) <= 2 * counts.max()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    os.environ.update(WORLD_SIZE="2", RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_0809_1810_gb300 import partition as P

    dist.init_process_group("gloo", rank=rank, world_size=2)
    L, reach = 4, 2
    rng = np.random.default_rng(21)  # the same occupancy on both ranks
    counts = rng.poisson(6.0, 4 ** L)
    bounds = P.leaf_bounds(counts, 2)
    other = 1 - rank
    plan = P.exchange_plan(bounds, L, reach)
    sends = _as_sets(plan[(rank, other)])
    recvs = _as_sets(plan[(other, rank)])
    got = [None, None]
    dist.all_gather_object(got, {"sends": sends, "recvs": recvs})
    ok = got[other]["sends"] == recvs and got[other]["recvs"] == sends
    want = brute_force(bounds, L, reach)
    ok = ok and sends == want[(rank, other)] and recvs == want[(other, rank)]
    q.put((rank, ok, len(sends[0]), len(sends[1])))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_exchange():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] for o in out)
    assert all(o[2] > 0 and o[3] > 0 for o in out)  # both send halo leaves and multipoles
