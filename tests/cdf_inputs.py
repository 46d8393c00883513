"""Input construction shared by the tests: a valid two-level integer sampling
CDF (the format of qrs_sampler.cell_cdf) for given cell probabilities.  None
of the method's arithmetic lives here; any valid CDF serves the tests."""
import numpy as np


def two_level_cdf(p_c, nr, nt):
    """Input construction: a valid two-level integer CDF (radial marginal, then
    each band's angular conditional) for cell probabilities p_c [nr * nt]."""
    p = np.asarray(p_c, np.float64).reshape(nr, nt)

    def q(v):
        w = np.floor(v / v.sum() * (2**32 - v.size)).astype(np.int64) + 1
        w[np.argmax(w)] += 2**32 - w.sum()
        return np.concatenate([[0], np.cumsum(w)[:-1]]), w

    rs, rw = q(p.sum(axis=1))
    parts, pq = [rs], np.zeros((nr, nt))
    for i in range(nr):
        ts, tw = q(p[i])
        parts.append(ts)
        pq[i] = rw[i] / 2.0**32 * tw / 2.0**32
    return np.concatenate(parts).astype(np.uint32), pq.ravel()
