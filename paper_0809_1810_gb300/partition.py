"""One FMM evaluation split over ranks by contiguous Morton-key ranges.

The leaves of the uniform quadtree (Sec. 3.3) in Morton order form a
space-filling curve; rank r owns the leaves with keys in
[bounds[r], bounds[r + 1]) and the particles in them.  Every box of a coarser
level covers a contiguous key range of leaves, so a rank's boxes at each
level are a contiguous range of box keys too.  What a rank needs from the
others (host-side index sets; the data moves by peer copies or NCCL):

* Near field (Eq. 10 over the local list of Sec. 3.3.1): the particles of
  every leaf within Chebyshev distance 1 of an owned leaf -- 2 when the cutoff
  a of Sec. 4.1 is on, the ring its correction reaches.  These are the halo
  leaves; their owners send the particles.
* Far field (Eq. 22 over the interaction lists): the complete multipole
  expansion of every box in the interaction list of a box that holds an
  owned leaf.  A multipole expansion is linear in the particles (Eq. 20), so
  each rank owning leaves under such a source box sends its partial
  expansion of that box, and the receiver adds them to its own.  M2L, L2L and
  L2P then run on the receiver exactly as in one evaluation.

This module is the plan (which leaves and which boxes each rank sends and
receives); `split_evaluate` runs the split with the library's two partial
entry points, fmm2d_multipoles and fmm2d_velocity_from_multipoles.
"""
from __future__ import annotations

import numpy as np


def morton_key(ix, iy):
    """Interleave the bits of ix (even bits) and iy (odd bits)."""
    ix = np.asarray(ix, dtype=np.uint64)
    iy = np.asarray(iy, dtype=np.uint64)

    def spread(v):
        v = v & np.uint64(0xFFFF)
        v = (v | (v << np.uint64(8))) & np.uint64(0x00FF00FF)
        v = (v | (v << np.uint64(4))) & np.uint64(0x0F0F0F0F)
        v = (v | (v << np.uint64(2))) & np.uint64(0x33333333)
        v = (v | (v << np.uint64(1))) & np.uint64(0x55555555)
        return v

    return spread(ix) | (spread(iy) << np.uint64(1))


def morton_xy(key):
    """(ix, iy) of Morton keys."""
    key = np.asarray(key, dtype=np.uint64)

    def compact(v):
        v = v & np.uint64(0x55555555)
        v = (v | (v >> np.uint64(1))) & np.uint64(0x33333333)
        v = (v | (v >> np.uint64(2))) & np.uint64(0x0F0F0F0F)
        v = (v | (v >> np.uint64(4))) & np.uint64(0x00FF00FF)
        v = (v | (v >> np.uint64(8))) & np.uint64(0x0000FFFF)
        return v

    return compact(key).astype(np.int64), compact(key >> np.uint64(1)).astype(np.int64)


def leaf_bounds(leaf_counts, ranks):
    """Split the leaves (counts in Morton order) into `ranks` contiguous key
    ranges of about equal particle count: bounds[0] = 0, bounds[ranks] =
    number of leaves, rank r owns [bounds[r], bounds[r + 1])."""
    counts = np.asarray(leaf_counts, dtype=np.int64)
    nleaf = counts.size
    total = int(counts.sum())
    cum = np.concatenate([[0], np.cumsum(counts)])
    bounds = [0]
    for r in range(1, ranks):
        # first leaf boundary at or past r/ranks of the particles
        k = int(np.searchsorted(cum, r * total / ranks, side="left"))
        bounds.append(min(max(k, bounds[-1]), nleaf))
    bounds.append(nleaf)
    return np.asarray(bounds, dtype=np.int64)


def owner_of(keys, bounds):
    """Rank owning each leaf key."""
    return np.searchsorted(np.asarray(bounds), np.asarray(keys, dtype=np.int64), side="right") - 1


def owned_boxes(bounds, r, L, level):
    """Box keys at `level` that hold at least one leaf of rank r (a
    contiguous range in Morton order); empty when r owns no leaf."""
    lo, hi = int(bounds[r]), int(bounds[r + 1])
    if hi <= lo:
        return np.zeros(0, dtype=np.int64)
    sh = 2 * (L - level)
    return np.arange(lo >> sh, ((hi - 1) >> sh) + 1, dtype=np.int64)


def box_owners(bounds, L, level, box):
    """Ranks owning leaves under box `box` of `level` (a contiguous range)."""
    sh = 2 * (L - level)
    lo, hi = int(box) << sh, (int(box) + 1) << sh
    first = int(owner_of(lo, bounds))
    last = int(owner_of(hi - 1, bounds))
    return [q for q in range(first, last + 1) if bounds[q + 1] > bounds[q]]


def halo_leaves(bounds, r, L, reach=1):
    """Leaf keys of other ranks within Chebyshev distance `reach` of a leaf
    of rank r: whole 3x3 (reach 1) or 5x5 (reach 2) blocks around each
    owned leaf, computed by offsetting the owned leaves' coordinates."""
    lo, hi = int(bounds[r]), int(bounds[r + 1])
    if hi <= lo:
        return np.zeros(0, dtype=np.int64)
    own = np.arange(lo, hi, dtype=np.int64)
    ix, iy = morton_xy(own)
    side = 1 << L
    found = []
    for dy in range(-reach, reach + 1):
        for dx in range(-reach, reach + 1):
            if dx == 0 and dy == 0:
                continue
            sx, sy = ix + dx, iy + dy
            ok = (sx >= 0) & (sy >= 0) & (sx < side) & (sy < side)
            found.append(morton_key(sx[ok], sy[ok]).astype(np.int64))
    keys = np.unique(np.concatenate(found)) if found else np.zeros(0, dtype=np.int64)
    return keys[(keys < lo) | (keys >= hi)]


# The 7 x 7 child offsets (dx, dy) of an interaction list, by target parity:
# children of the parent's 8 neighbours (and the parent itself) that are not
# adjacent to the target (Sec. 3.3.1).
def _il_offsets(px, py):
    out = []
    for dy in range(-2 - py, 4 - py):
        for dx in range(-2 - px, 4 - px):
            if max(abs(dx), abs(dy)) >= 2:
                out.append((dx, dy))
    return out


_IL = {(px, py): np.asarray(_il_offsets(px, py), dtype=np.int64) for px in (0, 1) for py in (0, 1)}


def needed_boxes(bounds, r, L):
    """{level: sorted box keys} in the interaction lists of rank r's boxes,
    levels 2..L (offsets of the source boxes by target parity)."""
    out = {}
    for level in range(2, L + 1):
        t = owned_boxes(bounds, r, L, level)
        if t.size == 0:
            out[level] = np.zeros(0, dtype=np.int64)
            continue
        tx, ty = morton_xy(t)
        side = 1 << level
        found = []
        for (px, py), offs in _IL.items():
            sel = ((tx & 1) == px) & ((ty & 1) == py)
            if not sel.any():
                continue
            bx, by = tx[sel][:, None] + offs[None, :, 0], ty[sel][:, None] + offs[None, :, 1]
            ok = (bx >= 0) & (by >= 0) & (bx < side) & (by < side)
            found.append(morton_key(bx[ok], by[ok]).astype(np.int64))
        out[level] = np.unique(np.concatenate(found)) if found else np.zeros(0, dtype=np.int64)
    return out


def exchange_plan(bounds, L, reach=1):
    """For every ordered pair of ranks (q, r), q != r: the leaves whose
    particles q sends to r (halo of r owned by q) and, per level, the boxes
    whose partial multipole expansions q sends to r (boxes r needs that hold
    leaves of q).  {(q, r): {"leaves": keys, "boxes": {level: keys}}}."""
    R = len(bounds) - 1
    plan = {}
    for r in range(R):
        halo = halo_leaves(bounds, r, L, reach)
        need = needed_boxes(bounds, r, L)
        halo_owner = owner_of(halo, bounds)
        for q in range(R):
            if q == r:
                continue
            boxes = {}
            for level, keys in need.items():
                sh = 2 * (L - level)
                lo_q, hi_q = int(bounds[q]), int(bounds[q + 1])
                if hi_q <= lo_q:
                    boxes[level] = np.zeros(0, dtype=np.int64)
                    continue
                # box key range of q at this level
                k0, k1 = lo_q >> sh, (hi_q - 1) >> sh
                boxes[level] = keys[(keys >= k0) & (keys <= k1)]
            plan[(q, r)] = {"leaves": halo[halo_owner == q], "boxes": boxes}
    return plan


def box_slot(L, level, keys, P):
    """Offsets (in reals) of boxes in the library's multipole array: levels
    2..L one after another, each as four parity planes (ix & 1, iy & 1) of a
    row-major (2^(level-1))^2 grid, 2P reals per box."""
    base = 0
    for lev in range(2, level):
        base += 4 ** lev
    ix, iy = morton_xy(keys)
    h = 1 << (level - 1)
    plane = ((iy & 1) << 1) | (ix & 1)
    return (base + (plane * h + (iy >> 1)) * h + (ix >> 1)) * 2 * P


def split_evaluate(plan_factory, xy, gamma, L, root, ranks, reach=1, exchange=None):
    """Evaluate one particle set as `ranks` partitions, one after another on
    the current device (the data paths of a multi-GPU run without the
    transport): each rank computes the multipoles of its own particles;
    rank r receives, per the exchange plan, the partial multipoles of the
    boxes it needs and the particles of its halo leaves, and evaluates its
    owned particles.  Returns the velocities of all particles (input order)
    and the plan.  plan_factory(n) returns a library Plan for up to n
    particles; `exchange(q, r, what, data)` may stand in for the transport."""
    import torch

    n = xy.shape[0]
    x0, y0, W = root
    side = 1 << L
    # leaf of every particle by the library's rule (floor, upper edge clamped)
    sc = side / W
    lx = torch.clamp(torch.floor((xy[:, 0].double() - x0) * sc), 0, side - 1).long().cpu().numpy()
    ly = torch.clamp(torch.floor((xy[:, 1].double() - y0) * sc), 0, side - 1).long().cpu().numpy()
    leaf = morton_key(lx, ly).astype(np.int64)
    counts = np.bincount(leaf, minlength=side * side)
    bounds = leaf_bounds(counts, ranks)
    own = owner_of(leaf, bounds)
    xplan = exchange_plan(bounds, L, reach)
    dev = xy.device
    # partial multipoles of every rank (its own particles only)
    partial = []
    for q in range(ranks):
        idx = torch.as_tensor(np.nonzero(own == q)[0], device=dev)
        with plan_factory(max(int(idx.numel()), 1)) as pl:
            partial.append(pl.multipoles(xy[idx].contiguous(), gamma[idx].contiguous()))
    uv = torch.zeros_like(xy)
    for r in range(ranks):
        me = partial[r].clone()
        P = me.numel() // (2 * sum(4 ** lev for lev in range(2, L + 1))) if L >= 2 else 0
        halo_idx = []
        for q in range(ranks):
            if q == r:
                continue
            ex = xplan[(q, r)]
            for level, keys in ex["boxes"].items():
                if keys.size == 0:
                    continue
                off = box_slot(L, level, keys, P)
                cols = torch.as_tensor(off[:, None] + np.arange(2 * P)[None, :], device=dev)
                data = partial[q][cols]
                if exchange is not None:
                    data = exchange(q, r, ("boxes", level), data)
                me[cols] += data
            if ex["leaves"].size:
                sel = np.nonzero(np.isin(leaf, ex["leaves"]) & (own == q))[0]
                halo_idx.append(sel)
        mine = np.nonzero(own == r)[0]
        halo = np.concatenate(halo_idx) if halo_idx else np.zeros(0, dtype=np.int64)
        idx = torch.as_tensor(np.concatenate([mine, halo]), device=dev)
        with plan_factory(max(int(idx.numel()), 1)) as pl:
            out = pl.velocity_from_multipoles(xy[idx].contiguous(), gamma[idx].contiguous(), me)
        uv[torch.as_tensor(mine, device=dev)] = out[: mine.size]
    return uv, xplan, bounds
