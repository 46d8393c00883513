"""Batched differential pistons: many interferometers of uneven aperture count,
N_f and realisation count in one persistent launch (cost-sorted atomic work
queue), optionally replayed from a CUDA graph, kernel shape from the
autotuner.  Checked against per-job launches and the FP64 oracle (1e-5 sigma
per value, sigma^2 = sum_k F_k^2 A^2 of the value's realisation)."""
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2404_02978_gb300 as qrs
from oracle import analytic as an
from paper_2404_02978_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _jobs(n, seed, scale=1):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        n_ap = int(rng.integers(2, 13))
        rad = 100 * np.sqrt(rng.uniform(size=n_ap))
        th = rng.uniform(0, 2 * np.pi, n_ap)
        out.append(dict(p=oracle.params(seed=int(1000 * seed + i), r0=float(rng.uniform(0.08, 0.2)),
                                        L0=float(rng.uniform(15, 40)), fmax=10.0),
                        n_f=int(rng.integers(64, 700)) * scale, n_real=int(rng.integers(3, 10)),
                        ap_xy=np.stack([rad * np.cos(th), rad * np.sin(th)], -1).astype(np.float32),
                        ap_D=rng.uniform(1.8, 8, n_ap).astype(np.float32),
                        ap_d=np.where(rng.uniform(size=n_ap) < 0.3, 1.1, 0.0).astype(np.float32),
                        pairs=wl.all_pairs(n_ap), off=int(rng.integers(0, 50))))
    return out


def _submit(h, jobs, flags):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    outs, cj = [], []
    for j in jobs:
        pis = torch.full((j["n_real"], j["ap_xy"].shape[0]), float("nan"), device="cuda")
        dlt = torch.full((j["n_real"], j["pairs"].shape[0]), float("nan"), device="cuda")
        cj.append(qrs.piston_job(j["p"], j["n_f"], j["n_real"], dev(j["ap_xy"]), dev(j["ap_D"]), dev(j["ap_d"]),
                                 dev(j["pairs"]), pis, dlt, real_offset=j["off"]))
        outs.append((pis, dlt))
    qrs.qrs_diff_piston(h, cj, flags=flags)
    qrs.qrs_sync(h)
    return cj, outs


def _sigma(j):
    d = oracle.draw(j["p"], n_f=j["n_f"], n_real=j["n_real"], real_offset=j["off"])
    f = np.hypot(d["f"][..., 0].astype(np.float64), d["f"][..., 1].astype(np.float64))
    A = np.stack([an.airy(f.ravel(), D, dd).reshape(f.shape) for D, dd in zip(j["ap_D"], j["ap_d"])], -1)
    return np.sqrt(np.einsum("rk,rka->ra", d["F"] ** 2, A ** 2))  # [n_real][n_ap]


@pytest.fixture(scope="module")
def h():
    from paper_2404_02978_gb300 import build as B
    B.build()
    return qrs.Handle(0)


def test_batch_modes_agree_and_match_oracle(h):
    jobs = _jobs(24, seed=1)
    _, ref = _submit(h, jobs, 0)
    _, per = _submit(h, jobs, qrs.PISTON_PERSISTENT)
    _, gr1 = _submit(h, jobs, qrs.PISTON_PERSISTENT | qrs.PISTON_GRAPH)   # capture
    cj, gr2 = _submit(h, jobs, qrs.PISTON_PERSISTENT | qrs.PISTON_GRAPH)  # replay (new buffers: new graph)
    for idx, j in enumerate(jobs):
        sig = _sigma(j)
        s_pair = np.sqrt(sig[:, j["pairs"][:, 0]] ** 2 + sig[:, j["pairs"][:, 1]] ** 2)
        for outs in (per, gr1, gr2):
            assert np.all(np.abs(outs[idx][0].cpu().numpy() - ref[idx][0].cpu().numpy()) <= 1e-5 * sig)
            assert np.all(np.abs(outs[idx][1].cpu().numpy() - ref[idx][1].cpu().numpy()) <= 1e-5 * s_pair)
        if idx % 6 == 0:
            pis_o, dlt_o = oracle.diff_piston(j["p"], j["n_f"], j["n_real"], j["ap_xy"], j["ap_D"], j["ap_d"],
                                              j["pairs"], real_offset=j["off"])
            assert np.all(np.abs(per[idx][0].cpu().numpy() - pis_o) <= 1e-5 * sig)
            assert np.all(np.abs(per[idx][1].cpu().numpy() - dlt_o) <= 1e-5 * s_pair)


def test_graph_replay_rewrites_outputs(h):
    jobs = _jobs(6, seed=2)
    cj, outs = _submit(h, jobs, qrs.PISTON_PERSISTENT | qrs.PISTON_GRAPH)
    first = [(p.clone(), d.clone()) for p, d in outs]
    for p, d in outs:
        p.fill_(float("nan"))
        d.fill_(float("nan"))
    before = h.launch_count()
    qrs.qrs_diff_piston(h, cj, flags=qrs.PISTON_PERSISTENT | qrs.PISTON_GRAPH)  # same job set: replay
    qrs.qrs_sync(h)
    assert h.launch_count() == before + 1
    for (p, d), (p0, d0) in zip(outs, first):
        assert torch.equal(p, p0) and torch.equal(d, d0)


def test_autotune_cache_file(tmp_path):
    path = tmp_path / "tune.txt"
    os.environ["QRS_AUTOTUNE_CACHE"] = str(path)
    try:
        hh = qrs.Handle(0)
        _submit(hh, _jobs(5, seed=3), qrs.PISTON_PERSISTENT)
        lines = path.read_text().split("\n")
        assert lines[0].startswith("piston:") and int(lines[0].split()[1]) in range(5)  # one of the five shapes
        hh.close()
    finally:
        del os.environ["QRS_AUTOTUNE_CACHE"]


def test_every_autotuner_shape_matches_the_oracle(tmp_path):
    """Each of the five persistent kernel shapes, forced through the autotuner's
    cache file (the bucket key from a first run, the shape number replaced),
    against per-job launches and the FP64 oracle; jobs with 8 or more
    apertures take the sorted-chunk path, the others the unsorted one."""
    path = tmp_path / "tune.txt"
    jobs = _jobs(10, seed=4) + [dict(j, ap_xy=np.concatenate([j["ap_xy"]] * 3), ap_D=np.concatenate([j["ap_D"]] * 3),
                                     ap_d=np.concatenate([j["ap_d"]] * 3), pairs=wl.all_pairs(3 * len(j["ap_D"])))
                                for j in _jobs(4, seed=5)]
    os.environ["QRS_AUTOTUNE_CACHE"] = str(path)
    try:
        h0 = qrs.Handle(0)
        _, ref = _submit(h0, jobs, 0)
        _submit(h0, jobs, qrs.PISTON_PERSISTENT)
        key = path.read_text().split()[0]
        h0.close()
        for shape in range(5):
            path.write_text("%s %d\n" % (key, shape))
            hs = qrs.Handle(0)
            _, got = _submit(hs, jobs, qrs.PISTON_PERSISTENT)
            for idx, j in enumerate(jobs):
                sig = _sigma(j)
                assert np.all(np.abs(got[idx][0].cpu().numpy() - ref[idx][0].cpu().numpy()) <= 1e-5 * sig), (shape,
                                                                                                           idx)
            pis_o, _ = oracle.diff_piston(jobs[-1]["p"], jobs[-1]["n_f"], jobs[-1]["n_real"], jobs[-1]["ap_xy"],
                                          jobs[-1]["ap_D"], jobs[-1]["ap_d"], jobs[-1]["pairs"],
                                          real_offset=jobs[-1]["off"])
            assert np.all(np.abs(got[-1][0].cpu().numpy() - pis_o) <= 1e-5 * _sigma(jobs[-1])), shape
            hs.close()
    finally:
        del os.environ["QRS_AUTOTUNE_CACHE"]


def test_batched_interferometers_full_size(h):
    """1000 interferometers: n_ap ~ U{4..64}, D ~ U(1.8, 8) m, centres in a
    200 m disc, N_f ~ U{256..8192}, 256 realisations each, all pairs, one
    persistent graph-captured launch; 12 sampled (job, realisation) items
    against the oracle."""
    cfg = wl.BATCHED
    inst = wl.batched_instances(cfg["n_inst"], seed=cfg["seed"])
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    cj, outs = [], []
    for i in inst:
        p = wl.method_params(dict(cfg, seed=i["seed"]))
        dlt = torch.empty(i["n_real"], i["pairs"].shape[0], device="cuda")
        cj.append(qrs.piston_job(p, i["n_f"], i["n_real"], dev(i["ap_xy"]), dev(i["ap_D"]), dev(i["ap_d"]),
                                 dev(i["pairs"]), None, dlt))
        outs.append(dlt)
    qrs.qrs_diff_piston(h, cj, flags=qrs.PISTON_PERSISTENT | qrs.PISTON_GRAPH)
    qrs.qrs_sync(h)
    rng = np.random.default_rng(0)
    for q in range(12):
        k = int(rng.integers(len(inst)))
        r = int(rng.integers(inst[k]["n_real"]))
        i = inst[k]
        p = wl.method_params(dict(cfg, seed=i["seed"]))
        _, d_o = oracle.diff_piston(p, i["n_f"], 1, i["ap_xy"], i["ap_D"], i["ap_d"], i["pairs"], real_offset=r)
        j = dict(p=p, n_f=i["n_f"], n_real=1, off=r, ap_D=i["ap_D"], ap_d=i["ap_d"])
        sig = _sigma(j)
        s_pair = np.sqrt(sig[:, i["pairs"][:, 0]] ** 2 + sig[:, i["pairs"][:, 1]] ** 2)
        got = outs[k][r:r + 1].cpu().numpy()
        assert np.all(np.abs(got - d_o) <= 1e-5 * s_pair), (k, r, np.max(np.abs(got - d_o) / s_pair))
