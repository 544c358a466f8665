"""CPU FP64 oracle of the learned (p, L) proposer.

TEST INFRASTRUCTURE ONLY, under the same rule as the rest of this package:
only the test suite, the smoke check and the benchmark's CPU legs may import
it; it never imports the CUDA library and shares no code with it.

The proposer is not in the paper.  It learns the error surface whose trends
Sec. 5 measures (error against expansion order p and tree depth l) and whose
floor Sec. 4.1 explains (the kernel-substitution error of Eqs. 26-29 when
leaves are small against sigma), and picks (p, L).  This module writes out,
in float64 and plain numpy, every step the CUDA side computes:

* :func:`bf16_round` -- IEEE binary32 to bfloat16, round to nearest, ties to
  even (the storage format of the weights).
* :func:`forward` -- the network 12 -> 128 -> 128 -> 128 -> 2 with SiLU
  (x * sigmoid(x)) between layers, inputs standardised, outputs
  de-standardised.
* :func:`loss_and_grad` -- mean squared error on standardised outputs and
  its gradient by the chain rule, layer by layer, through the BF16 weights.
* :func:`adam` -- one step of Adam (Kingma & Ba 2015, Algorithm 1).
* :func:`features` -- the 12 input features, from their definitions.
* :func:`cost_terms` -- the regressors of the linear cost model.
* :func:`propose` -- the selection rule: the cheapest candidate whose
  predicted log10 max error is at most log10(tol) - margin, else a fallback.

Parameter layout (34946 floats): for each layer W as [out][in] row-major,
then its bias [out].

Pins (tests/test_proposer_oracle_pins.py): the gradient against central
finite differences, bfloat16 rounding against torch's conversion and worked
bit patterns, SiLU closed forms, the zero-weight network, Adam's first step
(which moves each weight by -lr * sign(g)), features of a hand-built set,
the selection rule on a worked table.
"""
from __future__ import annotations

import math

import numpy as np

DIMS = (12, 128, 128, 128, 2)
N_IN, N_OUT = DIMS[0], DIMS[-1]
N_PARAMS = sum(DIMS[i + 1] * DIMS[i] + DIMS[i + 1] for i in range(len(DIMS) - 1))


def bf16_round(x) -> np.ndarray:
    """float32 -> nearest bfloat16 (ties to even), returned as float64.
    bfloat16 keeps the sign, the 8 exponent bits and the top 7 mantissa bits
    of binary32, so rounding adds half of the dropped 16-bit field (minus one
    when the kept field is even, so that exact ties go to the even neighbour)
    and truncates.  Finite inputs only."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    keep_lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = (u + np.uint64(0x7FFF) + keep_lsb) & np.uint64(0xFFFF0000)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params):
    """Flat parameter vector -> [(W_l, b_l)] as float64 views (copies)."""
    params = np.asarray(params, dtype=np.float64)
    if params.shape != (N_PARAMS,):
        raise ValueError("parameter vector must hold %d values" % N_PARAMS)
    out, at = [], 0
    for i in range(len(DIMS) - 1):
        nin, nout = DIMS[i], DIMS[i + 1]
        W = params[at:at + nout * nin].reshape(nout, nin)
        at += nout * nin
        b = params[at:at + nout]
        at += nout
        out.append((W.copy(), b.copy()))
    return out


def pack(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def _layers_used(params, bf16: bool):
    """The weights the network computes with: BF16-rounded matrices (from the
    float32 master values) and float32 biases, or the plain values."""
    layers = unpack(params)
    if not bf16:
        return layers
    return [(bf16_round(W.astype(np.float32)), b.astype(np.float32).astype(np.float64))
            for W, b in layers]


def _run(layers, norm, x):
    in_mean, in_std, out_mean, out_std = (np.asarray(a, np.float64) for a in norm)
    h = (np.asarray(x, np.float64) - in_mean) / in_std
    inputs, zs = [h], []
    for l, (W, b) in enumerate(layers):
        z = h @ W.T + b
        zs.append(z)
        h = silu(z) if l < len(layers) - 1 else z
        inputs.append(h)
    return inputs, zs


def forward(params, norm, x, bf16: bool = True) -> np.ndarray:
    """Network outputs (rows, 2) in de-standardised units.  `norm` is
    (in_mean[12], in_std[12], out_mean[2], out_std[2])."""
    layers = _layers_used(params, bf16)
    inputs, _ = _run(layers, norm, x)
    out_mean, out_std = np.asarray(norm[2], np.float64), np.asarray(norm[3], np.float64)
    return inputs[-1] * out_std + out_mean


def loss_and_grad(params, norm, x, t, bf16: bool = True):
    """(loss, gradient) of mean((y_s - t_s)^2) over rows x outputs, with y_s
    the raw (standardised) network output and t_s = (t - out_mean)/out_std.
    The gradient is taken with respect to the weights the network computes
    with (the BF16 values when bf16 is set) and is laid out like params."""
    layers = _layers_used(params, bf16)
    inputs, zs = _run(layers, norm, x)
    out_mean, out_std = np.asarray(norm[2], np.float64), np.asarray(norm[3], np.float64)
    ts = (np.asarray(t, np.float64) - out_mean) / out_std
    rows = ts.shape[0]
    d = inputs[-1] - ts
    loss = float(np.sum(d * d) / (rows * N_OUT))
    dz = 2.0 * d / (rows * N_OUT)  # d loss / d output (the last layer is linear)
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        grads[l] = (dz.T @ inputs[l], dz.sum(axis=0))
        if l > 0:
            dz = (dz @ W) * silu_grad(zs[l - 1])
    return loss, pack(grads)


def adam(w, g, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015, Algorithm 1) at step count t >= 1;
    returns the new (w, m, v)."""
    w, g, m, v = (np.asarray(a, np.float64) for a in (w, g, m, v))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


def leaf_index(x, y, root, L):
    """Leaf column and row of each particle at depth L: floor((x - x0) 2^L / W)
    clamped to [0, 2^L - 1] (Sec. 3.3's uniform subdivision of the root box)."""
    x0, y0, W = root
    side = 2 ** L
    ix = np.floor((np.asarray(x, np.float64) - x0) * (side / W))
    iy = np.floor((np.asarray(y, np.float64) - y0) * (side / W))
    ix = np.clip(np.nan_to_num(ix, nan=0.0), 0, side - 1).astype(np.int64)
    iy = np.clip(np.nan_to_num(iy, nan=0.0), 0, side - 1).astype(np.int64)
    return ix, iy


def features(x, y, gamma, sigma, root, p, L) -> np.ndarray:
    """The 12 features of a particle set for candidate (p, L):
    0 p; 1 L; 2 sigma / h with h = W / sqrt(n); 3 log2 n; 4 log2 of the mean
    particle count per leaf; 5 std / mean and 6 max / mean of the counts;
    7 sum_b |S_b| / sum_i |Gamma_i|; 8 std_b S_b / A; 9 max_b |S_b| / A;
    10 sum Gamma / sum |Gamma|; 11 log10(leaf width / sigma).  S_b is the
    circulation sum of leaf b and A = sum |Gamma| / 4^L.  Means and standard
    deviations run over all 4^L leaves, empty ones included (population
    standard deviation)."""
    g = np.asarray(gamma, np.float64)
    n = g.shape[0]
    x0, y0, W = root
    side = 2 ** L
    ix, iy = leaf_index(x, y, root, L)
    leaf = iy * side + ix
    nleaf = side * side
    counts = np.bincount(leaf, minlength=nleaf).astype(np.float64)
    S = np.bincount(leaf, weights=g, minlength=nleaf)
    abs_total = np.abs(g).sum()
    if abs_total <= 0.0:
        abs_total = 1.0
    A = abs_total / nleaf
    cmean = counts.mean()
    f = np.empty(12)
    f[0] = p
    f[1] = L
    f[2] = sigma / (W / math.sqrt(n))
    f[3] = math.log2(n)
    f[4] = math.log2(max(cmean, 1e-3))
    f[5] = counts.std() / cmean if cmean > 0 else 0.0
    f[6] = counts.max() / cmean if cmean > 0 else 0.0
    f[7] = np.abs(S).sum() / abs_total
    f[8] = S.std() / A
    f[9] = np.abs(S).max() / A
    f[10] = g.sum() / abs_total
    f[11] = math.log10(W / side / sigma)
    return f


def cost_terms(feat) -> np.ndarray:
    """Regressors of the linear cost model for one candidate row: 1, n,
    n p, boxes P^2 (boxes = (4^(L+1) - 1)/3 of the full tree, P = 16 for
    p <= 16 else 32, the padded order of the translation kernels), the
    near-field pair estimate 9 sum_b c_b^2 = 9 4^L mean^2 (1 + cv^2), read
    off features 3-5, and 16 sum_b c_b^2 for candidates whose leaves are
    narrower than the cutoff a = sigma sqrt(2 ln 10^6) of Sec. 4.1 (feature
    11, log10(leaf / sigma), below log10 sqrt(2 ln 10^6)): the scan of the
    ring of leaves the cutoff reaches."""
    p, L = float(feat[0]), int(round(float(feat[1])))
    n = 2.0 ** float(feat[3])
    mean, cv = 2.0 ** float(feat[4]), float(feat[5])
    boxes = (4.0 ** (L + 1) - 1.0) / 3.0
    P = 16.0 if p <= 16 else 32.0
    sum_c2 = 4.0 ** L * mean * mean * (1.0 + cv * cv)
    ring = 16.0 * sum_c2 if float(feat[11]) < math.log10(math.sqrt(2.0 * math.log(1e6))) else 0.0
    return np.array([1.0, n, n * p, boxes * P * P, 9.0 * sum_c2, ring])


def propose(pred_max_log10, cost, cand_p, cand_L, tol, margin, fallback):
    """Index, p and L of the cheapest candidate with predicted log10 max error
    <= log10(tol) - margin (the first such on equal cost); (-1, *fallback)
    when none qualifies."""
    want = math.log10(tol) - margin
    best = -1
    for c in range(len(cost)):
        if pred_max_log10[c] <= want and (best < 0 or cost[c] < cost[best]):
            best = c
    if best < 0:
        return -1, fallback[0], fallback[1]
    return best, int(cand_p[best]), int(cand_L[best])
