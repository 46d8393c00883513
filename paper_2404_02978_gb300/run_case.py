"""Run one named workload once through the C ABI (for profilers: no CPU reference,
no timing).  python -m paper_2404_02978_gb300.run_case --case phase_screen --n-real 16"""
import argparse

import torch

import paper_2404_02978_gb300 as qrs
from paper_2404_02978_gb300 import build as B
from paper_2404_02978_gb300 import workloads as wl


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="phase_screen",
                    choices=["phase_screen", "piston_plain", "gemm_screen", "batched", "grid_screen", "fft_screen"])
    ap.add_argument("--mode", default="gemm_3xtf32", choices=["gemm_3xtf32", "gemm_bf16x3", "gemm_tf32"])
    ap.add_argument("--points", type=int, default=0, help="gemm_screen: first N points only (0 = all)")
    ap.add_argument("--n-real", type=int, default=16)
    ap.add_argument("--n-inst", type=int, default=1000, help="batched: number of interferometers")
    ap.add_argument("--repeat", type=int, default=2)
    a = ap.parse_args()
    B.build()
    h = qrs.Handle(0)
    if a.case == "phase_screen":
        cfg = wl.PHASE_SCREEN
        xy = torch.from_numpy(wl.pupil_grid(cfg["grid"], cfg["pupil"])).cuda()
        for i in range(a.repeat):
            qrs.qrs_synthesize_points(h, wl.method_params(cfg), cfg["n_f"], a.n_real, xy, real_offset=i * a.n_real)
    elif a.case == "gemm_screen":
        cfg = wl.GEMM_SCREEN
        xy_np = wl.pupil_grid(cfg["grid"], cfg["pupil"])
        if a.points:
            xy_np = xy_np[: a.points]
        xy = torch.from_numpy(xy_np).cuda()
        for i in range(a.repeat):
            qrs.qrs_synthesize_points(h, wl.method_params(cfg), cfg["n_f"], cfg["n_real"], xy, mode=a.mode,
                                      real_offset=i * cfg["n_real"])
    elif a.case == "grid_screen":
        import numpy as np
        cfg = wl.PHASE_SCREEN
        n, L = cfg["grid"], cfg["pupil"]
        c = (np.arange(n, dtype=np.float64) + 0.5 - n / 2) * (L / n)
        X, Y = np.meshgrid(c, c, indexing="xy")
        inside = (X ** 2 + Y ** 2 <= (L / 2) ** 2).ravel()
        index = np.full(n * n, -1, np.int32)
        index[inside] = np.arange(int(inside.sum()), dtype=np.int32)
        cd = torch.from_numpy(c.astype(np.float32)).cuda()
        idx = torch.from_numpy(index).cuda()
        for i in range(a.repeat):
            qrs.qrs_synthesize_grid(h, wl.method_params(cfg), cfg["n_f"], a.n_real, cd, cd, index=idx,
                                    n_points=int(inside.sum()), mode=a.mode, real_offset=i * a.n_real)
    elif a.case == "fft_screen":
        p = qrs.params(seed=21, r0=0.15, L0=30.0)
        for i in range(a.repeat):
            qrs.fft_screens(h, p, 256, 8.0 / 256, a.n_real, real_offset=i * a.n_real)
    elif a.case == "batched":
        cfg = wl.BATCHED
        dev = lambda v: torch.from_numpy(v).cuda()
        jobs = []
        for i in wl.batched_instances(a.n_inst, seed=cfg["seed"]):
            dlt = torch.empty(i["n_real"], i["pairs"].shape[0], device="cuda")
            jobs.append(qrs.piston_job(wl.method_params(dict(cfg, seed=i["seed"])), i["n_f"], i["n_real"],
                                       dev(i["ap_xy"]), dev(i["ap_D"]), dev(i["ap_d"]), dev(i["pairs"]), None, dlt))
        for i in range(a.repeat):
            qrs.qrs_diff_piston(h, jobs, flags=qrs.PISTON_PERSISTENT | qrs.PISTON_GRAPH)
    else:
        cfg = wl.PISTON_PLAIN
        B_, ap_xy, ap_D, ap_d, pairs = wl.piston_plain_apertures()
        dev = lambda v: torch.from_numpy(v).cuda()
        delta = torch.empty(a.n_real, pairs.shape[0], device="cuda")
        for i in range(a.repeat):
            job = qrs.piston_job(wl.method_params(cfg), cfg["n_f"], a.n_real, dev(ap_xy), dev(ap_D), dev(ap_d),
                                 dev(pairs), None, delta, real_offset=i * a.n_real)
            qrs.qrs_diff_piston(h, [job])
    qrs.qrs_sync(h)
    print("ok", a.case, a.n_real, "launches", h.launch_count())


if __name__ == "__main__":
    main()
