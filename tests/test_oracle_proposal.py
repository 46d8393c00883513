"""Pins of the FP64 reference of the learned proposal.

* The analytic backward pass against central finite differences of the loss.
* Adam's first bias-corrected step is lr * g / (|g| + eps): ~lr * sign(g).
* The per-cell targets, before normalisation, add up to the conditional
  differential-piston structure function of the plain draws, whose mean is
  the Hankel integral D(B) (Sec. 4.4, Eq. 7 filter).
* The sampling CDF is a valid integer CDF; uniform logits give equal widths;
  every cell keeps at least the eps / C mixture share.
* He initialisation: weight variances 2 / fan_in, zero biases.
"""
import numpy as np
import pytest

import oracle.proposal as pr
from oracle import analytic as an


def _geom(n, seed):
    rng = np.random.default_rng(seed)
    B = np.exp(rng.uniform(np.log(1), np.log(200), n))
    th = rng.uniform(0, 2 * np.pi, n)
    return np.stack([np.exp(rng.uniform(np.log(0.05), np.log(0.3), n)), np.exp(rng.uniform(np.log(10), np.log(100), n)),
                     rng.uniform(1, 8, n), B * np.cos(th), B * np.sin(th)], -1)


def test_features_values():
    x = pr.features([[0.12, 30.0, 3.0, 15.0, 0.0]])[0]
    assert np.allclose(x, [0, 0, 0, 0, 1, 0], atol=1e-15)
    x = pr.features([[0.12 * np.e ** 0.6, 30.0, 3.0, 0.0, 15.0 * np.e ** 1.5]])[0]
    assert np.allclose(x, [1, 0, 0, 1, 0, 1], atol=1e-12)


def test_backward_matches_finite_differences():
    C = 8
    rng = np.random.default_rng(0)
    P = pr.init(C, 3) + 0.05 * rng.normal(size=pr.param_count(C))
    g = _geom(5, 1)
    T = rng.dirichlet(np.ones(C), size=5)
    L, G = pr.loss_grad(P, g, T, C)
    assert L == pytest.approx(pr.loss(P, g, T, C), rel=1e-14)
    idx = rng.choice(P.size, 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(P)
        e[i] = h
        fd = (pr.loss(P + e, g, T, C) - pr.loss(P - e, g, T, C)) / (2 * h)
        assert G[i] == pytest.approx(fd, rel=1e-5, abs=1e-9)
    # logit gradient rows sum to zero (softmax minus a distribution)
    W1, b1, W2, b2, W3, b3 = pr.unpack(G, C)
    assert abs(b3.sum()) < 1e-12


def test_adam_first_step():
    rng = np.random.default_rng(1)
    P = rng.normal(size=50)
    g = rng.normal(size=50)
    P1, m, v = pr.adam(P, np.zeros(50), np.zeros(50), g, lr=1e-2, step=1)
    assert np.allclose(P - P1, 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_targets_sum_to_hankel_integral():
    dom = (1e-3, 10.0)
    g = np.array([[0.1, 25.0, 1.0, 10.0, 0.0], [0.15, 40.0, 8.0, 0.0, 56.5], [0.08, 20.0, 2.0, 3.0, -4.0]])
    raw = pr.targets("von_karman", dom, 64, 32, 7, 4096, 8, g, raw=True)
    for i, (r0, L0, D, Bx, By) in enumerate(g):
        Dref = an.piston_sf(np.hypot(Bx, By), r0, L0, D, 0.0, dom[0], dom[1])
        assert raw[i].sum() == pytest.approx(Dref, rel=5e-3)
    t = raw / raw.sum(axis=1, keepdims=True)
    assert np.all(t >= 0) and np.allclose(t.sum(axis=1), 1.0)


def test_cdf_valid_uniform_and_floor():
    rng = np.random.default_rng(2)
    for nr, nt in ((4, 4), (64, 32)):
        C = nr * nt
        z = rng.normal(scale=4.0, size=C)
        cdf, pq = pr.cdf(z, 0.1, nr, nt)
        starts = [cdf[:nr]] + [cdf[nr + i * nt: nr + (i + 1) * nt] for i in range(nr)]
        for s in starts:
            s = s.astype(np.int64)
            w = np.diff(np.concatenate([s, [2**32]]))
            assert s[0] == 0 and np.all(w >= 1) and w.sum() == 2**32
        assert pq.sum() == pytest.approx(1.0, abs=1e-9)
        assert np.all(pq >= 0.1 / C * (1 - 1e-6))  # the mixture floor survives quantisation
        _, pu = pr.cdf(np.zeros(C), 0.1, nr, nt)
        assert np.allclose(pu, 1.0 / C, rtol=1e-6)


def test_cdf_temperature_vs_scipy_softmax():
    """p = (1 - eps) softmax(beta z) + eps / C against scipy's softmax of the
    scaled logits, to the quantisation (2^-32 per level); beta -> 0 is uniform."""
    from scipy.special import softmax
    rng = np.random.default_rng(4)
    nr, nt = 8, 16
    z = rng.normal(scale=3.0, size=nr * nt)
    for beta in (0.5, 0.8, 2.0):
        _, pq = pr.cdf(z, 0.05, nr, nt, beta=beta)
        p = 0.95 * softmax(beta * z) + 0.05 / z.size
        assert np.allclose(pq.ravel(), p, rtol=1e-7, atol=1e-9)
    _, pu = pr.cdf(z, 0.05, nr, nt, beta=1e-9)
    assert np.allclose(pu, 1.0 / z.size, rtol=1e-6)


def test_he_init_statistics():
    C = 2048
    P = pr.init(C, 11)
    W1, b1, W2, b2, W3, b3 = pr.unpack(P, C)
    assert np.all(b1 == 0) and np.all(b2 == 0) and np.all(b3 == 0)
    assert np.var(W3) == pytest.approx(2 / 128, rel=0.02)
    assert np.var(W2) == pytest.approx(2 / 128, rel=0.05)
    assert np.var(W1) == pytest.approx(2 / 6, rel=0.15)


# ------------------------------------------------------------- logit prior
@pytest.mark.parametrize("fold", [0, 1, 4])
def test_prior_cells_add_up_to_the_hankel_integral(fold):
    """The raw prior's cells, weighted by their share of the unit square and the
    constant 4 pi ln(fmax / fmin) dropped from g, add up to the structure function
    D(B) = 4 pi int f W A^2 (1 - J0(2 pi f B)) df (Sec. 4.4 with Eq. 7): the
    quadrature of the whole annulus, up to the accuracy of 64 nodes per cell."""
    g = _geom(4, 11)
    v = pr.prior(0, (1e-3, 10.0), 96, 24, fold, g, raw=True)
    for i, (r0, L0, D, Bx, By) in enumerate(g):
        total = 4.0 * np.pi * np.log(1e4) * v[i].sum() / (96 * 24)
        assert total == pytest.approx(an.piston_sf(np.hypot(Bx, By), r0, L0, D, 0.0, 1e-3, 10.0), rel=3e-3)


def test_prior_normalisation_and_floor():
    g = _geom(3, 12)
    P = pr.prior(0, (1e-3, 10.0), 32, 16, 4, g)
    assert np.allclose(P.max(axis=1), 0.0)
    assert P.min() >= pr.PRIOR_FLOOR
    # the nodes: the R2 sequence from (1/2, 1/2), first point the seed itself
    sx, sy = pr.prior_nodes(4)
    assert sx[0] == 0.5 and sy[0] == 0.5
    psi = 1.32471795724474602596
    assert sx[1] == pytest.approx((0.5 + 1 / psi) % 1.0, abs=1e-15)
    assert sy[1] == pytest.approx((0.5 + 1 / psi ** 2) % 1.0, abs=1e-15)


def test_prior_is_the_mean_of_the_plain_targets():
    """The prior estimates by quadrature what the MEAN targets estimate by plain
    draws: the two normalised distributions over the cells agree within the
    Monte-Carlo noise of the draws (total variation distance)."""
    g = _geom(3, 13)
    nr, nt = 24, 8
    v = pr.prior(0, (1e-3, 10.0), nr, nt, 4, g, raw=True)
    p_q = v / v.sum(axis=1, keepdims=True)
    t = pr.targets(0, (1e-3, 10.0), nr, nt, 5, 1024, 64, g, kind="mean", fold=4)
    tv = 0.5 * np.abs(p_q - t).sum(axis=1)
    assert np.all(tv < 0.03), tv


def test_backward_with_prior_matches_finite_differences():
    C = 8
    rng = np.random.default_rng(1)
    P = pr.init(C, 4) + 0.05 * rng.normal(size=pr.param_count(C))
    g = _geom(5, 2)
    T = rng.dirichlet(np.ones(C), size=5)
    prior = rng.normal(size=(5, C)) * 3.0
    L, G = pr.loss_grad(P, g, T, C, prior=prior)
    assert L == pytest.approx(pr.loss(P, g, T, C, prior=prior), rel=1e-14)
    idx = rng.choice(P.size, 40, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros_like(P)
        e[k] = h
        fd = (pr.loss(P + e, g, T, C, prior=prior) - pr.loss(P - e, g, T, C, prior=prior)) / (2 * h)
        assert G[k] == pytest.approx(fd, rel=1e-6, abs=1e-9)
