"""FP64 CPU reference of the learned frequency-sampling proposal (test
infrastructure only; never imported by the product package).

Written from the definitions stated in include/qrs_proposal.h:
* features of a geometry (r0, L0, D, Bx, By);
* the per-cell prior of the logits (a quadrature of each cell's contribution
  to the differential-piston structure function);
* the 6 -> 128 -> 128 -> C ReLU network, softmax cross entropy, its analytic
  backward pass (pinned by central finite differences in the tests) and the
  bias-corrected Adam step;
* the training targets: per-cell contributions of plain log-polar R2 draws
  (the oracle's own draw) to the differential-piston structure function of
  the geometry (Sec. 4.4 with the Eq. 7 filter), normalised;
* the integer sampling CDF built from a row of logits.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import analytic as an
from . import draw as _draw
from . import lib as _lib

H = 128
STREAM_INIT = 3


def param_count(n_cells: int) -> int:
    return 6 * H + H + H * H + H + H * n_cells + n_cells


def unpack(P, n_cells):
    P = np.asarray(P, np.float64)
    o = 0
    out = []
    for shape in ((6, H), (H,), (H, H), (H,), (H, n_cells), (n_cells,)):
        size = int(np.prod(shape))
        out.append(P[o:o + size].reshape(shape))
        o += size
    return out


def pack(parts):
    return np.concatenate([np.asarray(p, np.float64).ravel() for p in parts])


def features(geom):
    g = np.asarray(geom, np.float64).reshape(-1, 5)
    r0, L0, D, Bx, By = g.T
    B = np.hypot(Bx, By)
    return np.stack([(np.log(r0) - np.log(0.12)) / 0.6, (np.log(L0) - np.log(30.0)) / 0.8,
                     (np.log(D) - np.log(3.0)) / 0.6, (np.log(B) - np.log(15.0)) / 1.5, Bx / B, By / B], -1)


def init(n_cells, seed, out_scale=1.0):
    """He-normal weights from Philox normals (counter = parameter index, stream 3), zero biases;
    the output layer's weights times out_scale."""
    n = param_count(n_cells)
    z = np.zeros(n, np.float64)
    _lib().oracle_normals.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_void_p]
    _lib().oracle_normals(int(seed) & (2**64 - 1), STREAM_INIT, n, z.ctypes.data_as(C.c_void_p))
    fan = np.zeros(n)
    o = 0
    for (size, fan_in) in ((6 * H, 6), (H, 0), (H * H, H), (H, 0), (H * n_cells, H), (n_cells, 0)):
        fan[o:o + size] = fan_in
        o += size
    w = np.where(fan > 0, z * np.sqrt(2.0 / np.maximum(fan, 1)), 0.0)
    o3 = 6 * H + H + H * H + H
    w[o3:o3 + H * n_cells] *= out_scale
    return w


def forward(P, geom, n_cells, keep=False, prior=None):
    """Logits z = MLP(features) (+ prior [n][C] when given)."""
    W1, b1, W2, b2, W3, b3 = unpack(P, n_cells)
    X = features(geom)
    A1 = X @ W1 + b1
    H1 = np.maximum(A1, 0.0)
    A2 = H1 @ W2 + b2
    H2 = np.maximum(A2, 0.0)
    Z = H2 @ W3 + b3
    if prior is not None:
        Z = Z + np.asarray(prior, np.float64)
    if keep:
        return Z, (X, A1, H1, A2, H2)
    return Z


PRIOR_NODES = 64
PRIOR_FLOOR = -60.0


def prior_nodes(m=PRIOR_NODES):
    """The first m points of the R2 sequence of Eq. 6 from s0 = (1/2, 1/2), exact in
    0.64 fixed point, as FP64 fractions (S >> 11) 2^-53."""
    a1, a2 = np.uint64(0xC13FA9A902A6328F), np.uint64(0x91E10DA5C79E7B1D)
    k = np.arange(m, dtype=np.uint64)
    with np.errstate(over="ignore"):
        Sx = np.uint64(1 << 63) + k * a1
        Sy = np.uint64(1 << 63) + k * a2
    return (Sx >> np.uint64(11)).astype(np.float64) * 2.0 ** -53, (Sy >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def prior(psd_kind, dom, n_rho, n_theta, fold, geom, raw=False):
    """The prior of the proposal's logits: per importance cell c the mean, over
    the PRIOR_NODES points (s_x, s_y) of prior_nodes placed in the cell
    (u = (i_rho + s_x) / n_rho, t = (i_theta + s_y) / n_theta), of
        g = W(rho) A(pi D rho)^2 (1 - cos(2 pi rho |B| cos phi)) rho^2,
    rho = fmin (fmax / fmin)^u, phi the angle from the baseline: 2 pi t / fold
    for fold >= 1 (the cell's sector; its mirror images hold the same values),
    2 pi t - atan2(By, Bx) for fold 0.  That is the cell's mean contribution to
    the differential-piston structure function at B (Sec. 4.4 with Eq. 7) up to
    the constant 4 pi ln(fmax / fmin).  raw: v_c; else log(v_c / max v),
    floored at PRIOR_FLOOR.  Returns [n][n_rho n_theta]."""
    fmin, fmax = dom
    sx, sy = prior_nodes()
    u = (np.arange(n_rho)[:, None] + sx[None, :]) / n_rho          # [n_rho][M]
    t = (np.arange(n_theta)[:, None] + sy[None, :]) / n_theta      # [n_theta][M]
    rho = fmin * (fmax / fmin) ** u
    g = np.asarray(geom, np.float64).reshape(-1, 5)
    out = np.zeros((g.shape[0], n_rho * n_theta))
    for i, (r0, L0, D, Bx, By) in enumerate(g):
        B = np.hypot(Bx, By)
        phi = 2.0 * np.pi * t / fold if fold else 2.0 * np.pi * t - np.arctan2(By, Bx)
        env = an.psd(rho, r0, L0, psd_kind) * an.airy(rho.ravel(), D).reshape(rho.shape) ** 2 * rho ** 2
        # 1 - cos x as 2 sin^2 (x / 2): no cancellation where the phase is small
        osc = 2.0 * np.sin(np.pi * B * rho[:, None, :] * np.cos(phi)[None, :, :]) ** 2  # [n_rho][n_theta][M]
        v = np.mean(env[:, None, :] * osc, axis=2).ravel()
        if raw:
            out[i] = v
        else:
            with np.errstate(divide="ignore"):
                out[i] = np.maximum(np.log(v / v.max()), PRIOR_FLOOR)
    return out


def log_softmax(Z):
    m = Z.max(axis=1, keepdims=True)
    return Z - m - np.log(np.exp(Z - m).sum(axis=1, keepdims=True))


def loss(P, geom, T, n_cells, prior=None):
    Z = forward(P, geom, n_cells, prior=prior)
    return float(-np.mean(np.sum(np.asarray(T, np.float64) * log_softmax(Z), axis=1)))


def loss_grad(P, geom, T, n_cells, prior=None):
    """Mean cross entropy of softmax(z (+ prior)) and its gradient by the chain
    rule, layer by layer (the prior is a constant input of the softmax)."""
    W1, b1, W2, b2, W3, b3 = unpack(P, n_cells)
    T = np.asarray(T, np.float64)
    n = T.shape[0]
    Z, (X, A1, H1, A2, H2) = forward(P, geom, n_cells, keep=True, prior=prior)
    ls = log_softmax(Z)
    L = float(-np.mean(np.sum(T * ls, axis=1)))
    dZ = (np.exp(ls) - T) / n            # d L / d z (rows of T sum to 1)
    dW3 = H2.T @ dZ
    db3 = dZ.sum(axis=0)
    dA2 = (dZ @ W3.T) * (A2 > 0)
    dW2 = H1.T @ dA2
    db2 = dA2.sum(axis=0)
    dA1 = (dA2 @ W2.T) * (A1 > 0)
    dW1 = X.T @ dA1
    db1 = dA1.sum(axis=0)
    return L, pack([dW1, db1, dW2, db2, dW3, db3])


def adam(P, m, v, g, lr, step, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return P - lr * mh / (np.sqrt(vh) + eps), m, v


def plain_draws(dom, n_rho, n_theta, seed, n_f, n_draws):
    """The plain log-polar R2 draws the targets are built from (the oracle's own draw)."""
    p = dict(psd="von_karman", r0=1.0, L0=1.0, domain="logpolar", fmin=dom[0], fmax=dom[1], sampler="r2",
             seed=seed, s0=None, coef="gauss", n_rho=n_rho, n_theta=n_theta, cdf=None)
    return _draw(p, n_f=n_f, n_real=n_draws, debug=True)


FOLD_SHIFT = {1: 0, 2: 1, 4: 2}


def frame_fixed(Bx, By):
    """The baseline direction atan2(By, Bx) / 2 pi as a 0.64 fixed-point turn:
    the FP64 value x in (-1/2, 1/2] times 2^63, truncated to an integer, doubled
    modulo 2^64."""
    x = np.arctan2(By, Bx) / (2.0 * np.pi)
    return np.uint64(np.int64(x * 2.0 ** 63).astype(np.uint64)) * np.uint64(2)


def folded_cells(Sy, ir, n_theta, fold, Bx, By):
    """Cell of each plain draw in the baseline frame, folded F = fold times.
    The term's angle is 2 pi Sy 2^-64; its turn relative to the baseline
    direction is W = Sy - frame (mod 2^64); sector q = the top log2 F bits of W;
    the rest, W << log2 F (complemented in odd sectors, the mirror images), puts
    the term in angular cell ((W' >> 32) n_theta) >> 32 of the sector."""
    sh = FOLD_SHIFT[fold]
    with np.errstate(over="ignore"):
        W = Sy - frame_fixed(Bx, By)
        if sh:
            q = W >> np.uint64(64 - sh)
            W = W << np.uint64(sh)
            W = np.where((q & np.uint64(1)) == 1, ~W, W)
        it = ((W >> np.uint64(32)) * np.uint64(n_theta)) >> np.uint64(32)
    return ir * n_theta + it.astype(np.int64)


def targets(psd_kind, dom, n_rho, n_theta, seed, n_f, n_draws, geom, raw=False, kind="mean", fold=0):
    """v_k = w_k A(|f_k|)^2 2 (1 - cos 2 pi f_k . B), w_k = W(f_k; r0_i, L0_i) J_k / N_f
    over the plain draws; kind "mean": t_c ~ sum_{k in c} v_k (raw: / n_draws);
    kind "rms": t_c ~ sqrt(sum_{k in c} v_k^2); rows normalised to 1.
    fold 0: the draw's own cells (angle from the x axis); fold 1, 2, 4: cells of
    the geometry's baseline frame over one of `fold` mirrored sectors
    (folded_cells)."""
    d = plain_draws(dom, n_rho, n_theta, seed, n_f, n_draws)
    fx = d["f"][..., 0].astype(np.float64).ravel()
    fy = d["f"][..., 1].astype(np.float64).ravel()
    J = d["J"].ravel()
    cell = d["cell"].ravel()
    Sy = d["r2"][..., 1].ravel()
    ir = cell.astype(np.int64) // n_theta
    nc = n_rho * n_theta
    g = np.asarray(geom, np.float64).reshape(-1, 5)
    out = np.zeros((g.shape[0], nc))
    fr = np.hypot(fx, fy)
    for i, (r0, L0, D, Bx, By) in enumerate(g):
        w = an.psd(fr, r0, L0, psd_kind) * J / n_f
        A = an.airy(fr, D)
        c = w * A ** 2 * 2.0 * (1.0 - np.cos(2.0 * np.pi * (fx * Bx + fy * By)))
        ci = cell if not fold else folded_cells(Sy, ir, n_theta, fold, Bx, By)
        if kind == "rms":
            out[i] = np.sqrt(np.bincount(ci, weights=c * c, minlength=nc))
        else:
            out[i] = np.bincount(ci, weights=c, minlength=nc) / n_draws
    return out if raw else out / out.sum(axis=1, keepdims=True)


def quantise(p, scale_count):
    """Integer widths of a probability vector: floor(p (2^32 - n)) + 1, the
    remainder to the largest (first on ties); returns (starts, widths)."""
    p = np.asarray(p, np.float64)
    n = p.size
    w = np.floor(p * float(2**32 - n)).astype(np.int64) + 1
    w[np.argmax(w)] += 2**32 - int(w.sum())
    return np.concatenate([[0], np.cumsum(w)[:-1]]).astype(np.int64), w


def cdf(logits, eps, n_rho, n_theta, beta=1.0):
    """Two-level sampling CDF: p = (1 - eps) softmax(beta z) + eps / C over the
    n_rho x n_theta cells (beta: the softmax temperature's inverse); the
    marginal over radial bands, then each band's conditional over its angular
    cells, each quantised to widths summing to 2^32.  Returns (uint32
    [n_rho + n_rho n_theta], cell probabilities as quantised
    (p_band p_cell|band))."""
    z = np.asarray(logits, np.float64).ravel()
    C_ = n_rho * n_theta
    q = np.exp(beta * (z - z.max()))
    q /= q.sum()
    p = ((1 - eps) * q + eps / C_).reshape(n_rho, n_theta)
    Pr = p.sum(axis=1)
    rs, rw = quantise(Pr, n_rho)
    out = [rs]
    pq = np.zeros((n_rho, n_theta))
    for i in range(n_rho):
        ts, tw = quantise(p[i] / Pr[i], n_theta)
        out.append(ts)
        pq[i] = (rw[i] / 2.0**32) * (tw / 2.0**32)
    return np.concatenate(out).astype(np.uint32), pq
