"""Learned (p, L) proposer: binding, training-row generation, training and
proposal.

The paper picks the expansion order p and the tree depth l by hand and
measures how the error moves with them (Sec. 5), explaining the floor that a
leaf small against the core size sigma puts under it (Sec. 4.1, Eqs. 26-29).
The proposer learns that error surface from the library's own measurements
and returns the cheapest (p, L) whose predicted max error meets a
tolerance, or a conservative fixed setting when none qualifies.

All network arithmetic (forward, backward, Adam) and the feature reduction
run in libfmm2d's kernels (fmm2d_mlp_*, fmm2d_features, fmm2d_propose); this
module marshals arrays, drives the FMM and its FP64 direct sum to produce
training rows, fits the linear cost model, and reads and writes checkpoints
(a JSON header plus the raw float32 parameters).
"""
from __future__ import annotations

import ctypes
import json
import math
import os

import numpy as np
import torch

from . import Plan, _check, _native, _ptr, _stream, cutoff_for

HERE = os.path.dirname(os.path.abspath(__file__))
CHECKPOINT = os.path.join(HERE, "data", "proposer")
FALLBACK_P = 20
# Every candidate runs with the cutoff of Sec. 4.1 set for this tolerance:
# a = sigma sqrt(2 ln(1/tol)) where the leaves are narrower (cutoff_for), so
# the error surface learned is that of the method with the cutoff.
CUTOFF_TOL = 1e-6
# log10(leaf / sigma) below which a candidate runs with the cutoff
CUTOFF_LOG10_LEAF = math.log10(math.sqrt(2.0 * math.log(1.0 / CUTOFF_TOL)))


def cutoff(sigma: float, root, L: int) -> float:
    """The cutoff a candidate at depth L runs with (0: none needed)."""
    return cutoff_for(sigma, root[2] / 2.0 ** L, CUTOFF_TOL)
ORDERS = tuple(range(4, 29))
N_IN, N_OUT, N_PARAMS = _native.MLP_INPUTS, _native.MLP_OUTPUTS, _native.MLP_PARAMS
FEATURE_NAMES = ("p", "L", "sigma_over_h", "log2_n", "log2_mean_per_leaf",
                 "count_cv", "count_max_over_mean", "sum_abs_leaf_sum_over_sum_abs",
                 "leaf_sum_std_over_A", "leaf_sum_max_over_A", "sum_over_sum_abs",
                 "log10_leaf_over_sigma")
LABEL_NAMES = ("log10_median_leaf_err", "log10_max_err")


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


class MLP:
    """The network of fmm2d_mlp_create: 12 -> 128 -> 128 -> 128 -> 2, BF16
    weights, FP32 accumulation, trained by the library's own kernels."""

    def __init__(self, max_rows: int = 4096, seed: int = 0):
        self._lib = _native.load()
        self.max_rows = int(max_rows)
        h = ctypes.c_void_p()
        _check(self._lib.fmm2d_mlp_create(ctypes.byref(h), self.max_rows, int(seed)),
               "mlp_create")
        self._h = h
        self.norm = (np.zeros(N_IN, np.float32), np.ones(N_IN, np.float32),
                     np.zeros(N_OUT, np.float32), np.ones(N_OUT, np.float32))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.fmm2d_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_normalization(self, in_mean, in_std, out_mean, out_std):
        norm = tuple(_f32(a) for a in (in_mean, in_std, out_mean, out_std))
        if [a.size for a in norm] != [N_IN, N_IN, N_OUT, N_OUT]:
            raise ValueError("normalisation arrays must hold 12, 12, 2, 2 values")
        _check(self._lib.fmm2d_mlp_set_normalization(
            self._h, *[a.ctypes.data_as(ctypes.c_void_p) for a in norm]), "mlp_set_normalization")
        self.norm = norm

    def params(self) -> np.ndarray:
        out = np.empty(N_PARAMS, np.float32)
        _check(self._lib.fmm2d_mlp_params(self._h, out.ctypes.data_as(ctypes.c_void_p), None),
               "mlp_params")
        return out

    def set_params(self, w):
        w = _f32(w)
        if w.size != N_PARAMS:
            raise ValueError(f"expected {N_PARAMS} parameters")
        _check(self._lib.fmm2d_mlp_params(self._h, None, w.ctypes.data_as(ctypes.c_void_p)),
               "mlp_params")

    def _rows(self, x):
        if not (x.is_cuda and x.dtype == torch.float32 and x.dim() == 2 and x.shape[1] == N_IN):
            raise TypeError("x must be a CUDA float32 tensor of shape (rows, 12)")
        return x.contiguous(), int(x.shape[0])

    def forward(self, x, stream=None):
        x, rows = self._rows(x)
        y = torch.empty((rows, N_OUT), dtype=torch.float32, device=x.device)
        _check(self._lib.fmm2d_mlp_forward(self._h, rows, _ptr(x), _ptr(y), _stream(stream)),
               "mlp_forward")
        return y

    def gradients(self, x, t, stream=None):
        """(gradient (34946,), loss ()) of the standardised mean squared
        error, as device tensors."""
        x, rows = self._rows(x)
        t = t.contiguous()
        g = torch.empty(N_PARAMS, dtype=torch.float32, device=x.device)
        loss = torch.empty((), dtype=torch.float32, device=x.device)
        _check(self._lib.fmm2d_mlp_gradients(self._h, rows, _ptr(x), _ptr(t), _ptr(g),
                                             _ptr(loss), _stream(stream)), "mlp_gradients")
        return g, loss

    def train_step(self, x, t, lr: float, loss_out=None, stream=None):
        """One Adam step; the loss before the step lands in loss_out (a
        device float32 scalar) when given."""
        x, rows = self._rows(x)
        _check(self._lib.fmm2d_mlp_train_step(self._h, rows, _ptr(x), _ptr(t.contiguous()),
                                              ctypes.c_float(lr), _ptr(loss_out),
                                              _stream(stream)), "mlp_train_step")

    # -- checkpoints -----------------------------------------------------------
    def save(self, prefix: str, meta: dict | None = None):
        os.makedirs(os.path.dirname(os.path.abspath(prefix)), exist_ok=True)
        self.params().astype("<f4").tofile(prefix + ".f32")
        head = {"format": "fmm2d-mlp", "dims": [N_IN, 128, 128, 128, N_OUT],
                "params": N_PARAMS, "layout": "per layer: W [out][in] row-major, then b [out]",
                "features": list(FEATURE_NAMES), "labels": list(LABEL_NAMES),
                "in_mean": self.norm[0].tolist(), "in_std": self.norm[1].tolist(),
                "out_mean": self.norm[2].tolist(), "out_std": self.norm[3].tolist()}
        head.update(meta or {})
        with open(prefix + ".json", "w") as f:
            json.dump(head, f, indent=1)

    @classmethod
    def load(cls, prefix: str, max_rows: int = 4096):
        with open(prefix + ".json") as f:
            head = json.load(f)
        if head.get("format") != "fmm2d-mlp" or head.get("params") != N_PARAMS:
            raise ValueError(f"{prefix}.json is not a checkpoint of this network")
        w = np.fromfile(prefix + ".f32", dtype="<f4")
        net = cls(max_rows=max_rows)
        net.set_params(w)
        net.set_normalization(head["in_mean"], head["in_std"], head["out_mean"],
                              head["out_std"])
        return net, head


# -- features and candidates ----------------------------------------------------

def features(xy, gamma, sigma: float, root, p: int, L: int, stream=None) -> np.ndarray:
    """The 12 features (fmm2d_features) of float32 device particles."""
    lib = _native.load()
    if not (xy.is_cuda and gamma.is_cuda and xy.dtype == torch.float32
            and gamma.dtype == torch.float32):
        raise TypeError("features take float32 CUDA tensors")
    xy, gamma = xy.contiguous(), gamma.contiguous()
    out = np.empty(N_IN, np.float32)
    _check(lib.fmm2d_features(int(gamma.shape[0]), _ptr(xy), _ptr(gamma), float(sigma),
                              float(root[0]), float(root[1]), float(root[2]), int(p), int(L),
                              out.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
           "features")
    return out


def depth_candidates(n: int):
    """Depths whose mean leaf occupancy lies between 4 and 2048 particles."""
    lo = max(0, math.ceil(math.log(max(n, 1) / 2048.0, 4)))
    hi = min(10, math.floor(math.log(max(n, 4) / 4.0, 4)))
    return list(range(lo, max(lo, hi) + 1))


def fallback(n: int, sigma: float, root) -> tuple:
    """The conservative plain setting: p = 20 and the depth that gives about
    64 particles per leaf, capped so that a leaf spans at least 6 sigma --
    the regularised and singular kernels then differ by less than
    exp(-18) beyond the near field (Sec. 4.1, Eq. 29)."""
    L_occ = int(round(math.log(max(n, 1) / 64.0, 4))) if n > 64 else 0
    L_floor = int(math.floor(math.log2(root[2] / (6.0 * sigma)))) if root[2] > 6 * sigma else 0
    return FALLBACK_P, max(0, min(10, L_occ, L_floor))


def cost_terms(feat) -> np.ndarray:
    """Regressors of the cost model for one candidate row: a constant, n
    (tree build), n p (P2M, L2P), boxes x P^2 with P the padded order of the
    translation kernels (M2M, M2L, L2L), the near-field pair estimate
    9 sum_b c_b^2 = 9 4^L mean^2 (1 + cv^2), and, for candidates that run
    with the cutoff (log10(leaf / sigma) below CUTOFF_LOG10_LEAF), the ring
    scan 16 sum_b c_b^2."""
    p, L = float(feat[0]), int(round(float(feat[1])))
    n = 2.0 ** float(feat[3])
    mean, cv = 2.0 ** float(feat[4]), float(feat[5])
    boxes = (4.0 ** (L + 1) - 1.0) / 3.0
    P = 16.0 if p <= 16 else 32.0
    sum_c2 = 4.0 ** L * mean * mean * (1.0 + cv * cv)
    ring = 16.0 * sum_c2 if float(feat[11]) < CUTOFF_LOG10_LEAF else 0.0
    return np.array([1.0, n, n * p, boxes * P * P, 9.0 * sum_c2, ring])


def fit_cost_model(feats, seconds) -> np.ndarray:
    """Non-negative least squares of measured seconds on cost_terms,
    weighted by 1/seconds (relative error)."""
    from scipy.optimize import nnls

    A = np.stack([cost_terms(f) for f in feats])
    s = np.asarray(seconds, np.float64)
    w = 1.0 / s
    scale = np.abs(A).max(axis=0)
    coef, _ = nnls(A / scale * w[:, None], s * w)
    return coef / scale


class Proposer:
    """A trained network, its cost model and the selection margin."""

    def __init__(self, net: MLP, cost_coef, margin: float = 0.5, meta: dict | None = None):
        self.net = net
        self.cost_coef = np.asarray(cost_coef, np.float64)
        self.margin = float(margin)
        self.meta = meta or {}

    @classmethod
    def load(cls, prefix: str = CHECKPOINT, max_rows: int = 4096):
        net, head = MLP.load(prefix, max_rows=max_rows)
        return cls(net, head["cost_coef"], head.get("margin", 0.5), head)

    def candidates(self, xy, gamma, sigma, root, orders=ORDERS, depths=None):
        n = int(gamma.shape[0])
        depths = depth_candidates(n) if depths is None else depths
        rows = []
        for L in depths:
            f = features(xy, gamma, sigma, root, 1, L)
            for p in orders:
                r = f.copy()
                r[0] = p
                rows.append(r)
        feats = np.stack(rows).astype(np.float32)
        cost = np.array([float(cost_terms(r) @ self.cost_coef) for r in feats])
        return feats, cost

    def _select(self, feats, cost, tol, margin, fb):
        lib = _native.load()
        p, L, choice = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        pred = np.empty((len(feats), N_OUT), np.float32)
        cost = np.ascontiguousarray(cost, np.float64)
        _check(lib.fmm2d_propose(self.net._h, len(feats), feats.ctypes.data_as(ctypes.c_void_p),
                                 cost.ctypes.data_as(ctypes.c_void_p), float(tol), float(margin),
                                 fb[0], fb[1], ctypes.byref(p), ctypes.byref(L),
                                 ctypes.byref(choice), pred.ctypes.data_as(ctypes.c_void_p)),
               "propose")
        return p.value, L.value, choice.value, pred

    def propose(self, xy, gamma, sigma, root, tol: float = 1e-6, margin: float | None = None,
                orders=ORDERS, depths=None, verify: int = 0, precision="fp32_tc",
                accept: float = 0.8, max_tries: int = 4, screen_margin: float = 0.1) -> dict:
        """(p, L) for these particles (fmm2d_propose) with the candidate table.

        verify = 0: the network's choice at `margin` decades below the
        tolerance (the checkpoint's validation margin by default).
        verify = S > 0: direct-sum sampling judges the choice.  Candidates
        pass the network at `screen_margin`; the cheapest is run through the
        FMM and its max error measured against the FP64 direct sum at S
        seeded particles; it is accepted at <= accept * tol, otherwise it is
        struck from the table and the next cheapest is tried (at most
        max_tries), before the fallback."""
        n = int(gamma.shape[0])
        feats, cost = self.candidates(xy, gamma, sigma, root, orders, depths)
        fb = fallback(n, sigma, root)
        out = {"fallback": fb, "features": feats, "cost": cost, "tries": []}
        if not verify:
            m = self.margin if margin is None else float(margin)
            p, L, ch, pred = self._select(feats, cost, tol, m, fb)
            out.update(p=p, L=L, cutoff=cutoff(sigma, root, L), choice=ch, predicted=pred)
            return out
        import workloads as W

        tgt = torch.tensor(W.sample_targets(n, int(verify), 7919), device=xy.device)
        with Plan(1, 0, sigma, "fp32", root=root, max_n=n) as yard:
            ref = yard.direct_sampled(xy, gamma, tgt, kernel=0)
        work = cost.copy()
        pred = None
        for _ in range(max_tries):
            p, L, ch, pred_k = self._select(feats, work, tol, screen_margin, fb)
            pred = pred_k if pred is None else pred
            if ch < 0:
                break
            a = cutoff(sigma, root, L)
            with Plan(p, L, sigma, precision, root=root, max_n=n, cutoff=a) as plan:
                uv = plan.velocity(xy, gamma)
                st = plan.error_stats(xy, uv, tgt, ref).cpu().numpy()
                plan.check()
            err = float(st[0] / st[1])
            out["tries"].append({"p": p, "L": L, "cutoff": a, "err": err,
                                 "predicted": float(pred_k[ch, 1])})
            if err <= accept * tol:
                out.update(p=p, L=L, cutoff=a, choice=ch, predicted=pred, verified_err=err)
                return out
            work[ch] = np.inf  # struck: the selection skips non-finite costs
        out.update(p=fb[0], L=fb[1], cutoff=cutoff(sigma, root, fb[1]), choice=-1, predicted=pred)
        return out


# -- training rows --------------------------------------------------------------

def label_set_specs(count: int, seed: int, sizes=(1 << 18, 1 << 19, 1 << 20)):
    """Particle sets for training rows: uniform, Lamb-Oseen lattice and
    clustered families in turn; n drawn from `sizes`, sigma/h log-uniform in
    [0.6, 3], patch counts 8..64 for the clustered family."""
    rng = np.random.Generator(np.random.PCG64(seed))
    kinds = ("uniform", "lamb_oseen", "clustered")
    out = []
    for i in range(count):
        out.append({"index": i, "kind": kinds[i % 3], "n": int(rng.choice(sizes)),
                    "sigma_over_h": float(math.exp(rng.uniform(math.log(0.6), math.log(3.0)))),
                    "npatch": int(rng.integers(8, 65)), "seed": int(seed * 1000003 + i)})
    return out


def make_set(spec):
    import workloads as W

    n, soh = spec["n"], spec["sigma_over_h"]
    if spec["kind"] == "lamb_oseen":
        side = int(round(math.sqrt(n)))
        return W.lamb_oseen_lattice(side, sigma_over_h=soh, dtype=np.float32)
    h = 2.0 / math.sqrt(n)
    if spec["kind"] == "uniform":
        return W.uniform_random(n, spec["seed"], h, sigma_over_h=soh)
    return W.clustered_patches(n, spec["seed"], npatch=spec["npatch"], h=h, sigma_over_h=soh)


def measure(w, orders=ORDERS, depths=None, targets: int = 1024, seed: int = 0,
            precision="fp32_tc", max_pairs: float = 3e10):
    """Training rows of one particle set: for every candidate (p, L), the
    features, the two labels (FMM velocities against the FP64 regularised
    direct sum at `targets` sampled particles, relative to the largest
    reference speed) and the replayed evaluation time in seconds.  Depths
    whose near-field pair estimate exceeds `max_pairs` (tens of
    milliseconds of near field: never the cheapest) are skipped."""
    import workloads as W

    dev = torch.device("cuda")
    xy = torch.tensor(np.stack([w.x, w.y], 1).astype(np.float32), device=dev)
    g = torch.tensor(w.gamma.astype(np.float32), device=dev)
    n = w.n
    depths = depth_candidates(n) if depths is None else depths
    base = {L: features(xy, g, w.sigma, w.root, 1, L) for L in depths}
    pairs = {L: cost_terms(base[L])[4] for L in depths}
    depths = [L for L in depths if pairs[L] <= max_pairs] or [max(depths)]
    tgt = torch.tensor(W.sample_targets(n, targets, seed), device=dev)
    ref = None
    rows = []
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for L in depths:
        for p in orders:
            with Plan(p, L, w.sigma, precision, root=w.root, max_n=n,
                      cutoff=cutoff(w.sigma, w.root, L)) as plan:
                if ref is None:
                    ref = plan.direct_sampled(xy, g, tgt, kernel=0)
                uv = plan.velocity(xy, g)
                start.record()
                uv = plan.velocity(xy, g, out=uv)
                stop.record()
                stats, leaf = plan.error_stats(xy, uv, tgt, ref, per_leaf=True)
                plan.check()
                secs = start.elapsed_time(stop) * 1e-3
                s = stats.cpu().numpy()
                le = leaf.cpu().numpy()
                le = le[le > 0]
            ref_max = s[1]  # largest sampled reference speed (Sec. 5.1 normalisation)
            emax = max(s[0] / ref_max, 1e-12)
            emed = max(float(np.median(le)) / ref_max if le.size else emax, 1e-12)
            f = base[L].copy()
            f[0] = p
            rows.append(np.concatenate([f, [math.log10(emed), math.log10(emax), secs]]))
    return np.stack(rows).astype(np.float64)


# -- training -------------------------------------------------------------------

def normalisation(X, Y):
    in_mean, in_std = X.mean(0), X.std(0)
    in_std = np.where(in_std > 1e-6, in_std, 1.0)
    out_mean, out_std = Y.mean(0), Y.std(0)
    out_std = np.where(out_std > 1e-6, out_std, 1.0)
    return in_mean, in_std, out_mean, out_std


def train(X, Y, epochs: int = 300, batch: int = 2048, lr: float = 2e-3, seed: int = 0,
          X_val=None, Y_val=None, log=None):
    """Fit the network to rows (X, Y) with the library's Adam kernel on
    shuffled mini-batches (cosine learning-rate decay).  Returns the network
    and the per-epoch (mean train loss, validation RMSE per label)."""
    X, Y = np.asarray(X, np.float32), np.asarray(Y, np.float32)
    if X_val is not None:
        X_val, Y_val = np.asarray(X_val, np.float32), np.asarray(Y_val, np.float32)
    batch = min(batch, len(X))
    net = MLP(max_rows=max(batch, len(X_val) if X_val is not None else 0), seed=seed)
    net.set_normalization(*normalisation(X, Y))
    rng = np.random.Generator(np.random.PCG64(seed))
    dev = torch.device("cuda")
    steps_per_epoch = len(X) // batch
    losses = torch.zeros(max(steps_per_epoch, 1), dtype=torch.float32, device=dev)
    total = epochs * steps_per_epoch
    hist = []
    step = 0
    xv = torch.tensor(X_val, device=dev) if X_val is not None else None
    for ep in range(epochs):
        perm = rng.permutation(len(X))
        xe = torch.tensor(X[perm], device=dev)
        ye = torch.tensor(Y[perm], device=dev)
        for b in range(steps_per_epoch):
            rate = lr * 0.5 * (1.0 + math.cos(math.pi * step / max(total, 1)))
            net.train_step(xe[b * batch:(b + 1) * batch], ye[b * batch:(b + 1) * batch],
                           max(rate, lr * 1e-3), loss_out=losses[b])
            step += 1
        rec = {"epoch": ep, "train_mse": float(losses.cpu().numpy().mean())}
        if xv is not None and (ep % 10 == 0 or ep == epochs - 1):
            pred = net.forward(xv).cpu().numpy()
            rec["val_rmse"] = np.sqrt(((pred - Y_val) ** 2).mean(0)).tolist()
        hist.append(rec)
        if log:
            log(rec)
    return net, hist
