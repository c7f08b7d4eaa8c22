"""Accuracy and timing report for the workloads of the parity tests: the CUDA
path against the FP64 oracle (relative L2, norm and energy drift), the GPU
paths' speed, and the oracle's own speed on this host's cores.

Test infrastructure (it imports the oracle); run on a machine with a GPU:

    python tests/accuracy_report.py > report.json

Prints one JSON object per workload, then a summary object.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import oracle  # noqa: E402
from paper_1208_2407_gb300 import trotter  # noqa: E402
from paper_1208_2407_gb300 import workloads as wl  # noqa: E402

NCPU = max(1, os.cpu_count() or 1)


def rel_l2(are, aim, bre, bim):
    num = np.sqrt(np.sum((are - bre) ** 2 + (aim - bim) ** 2))
    return float(num / np.sqrt(np.sum(bre ** 2 + bim ** 2)))


def timed(fn):
    t0 = time.perf_counter()
    out = fn()
    return out, time.perf_counter() - t0


def gpu_ms(fn):
    import torch
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def emit(obj):
    print(json.dumps(obj), flush=True)
    return obj


def plain_fp64_256():
    c = wl.plain_fp64_256()
    n = c["nx"] * c["ny"] * c["steps"]
    args = (c["re"], c["im"], c["V"], c["dt"], c["theta"], c["steps"])
    (ore, oim), t1 = timed(lambda: oracle.evolve(*args, nthreads=1))
    _, tn = timed(lambda: oracle.evolve(*args, nthreads=NCPU))
    g = trotter.Grid(c["nx"], c["ny"], "f64")
    g.set_state(c["re"], c["im"])
    g.set_potential(c["V"], c["dt"], c["theta"])
    ms = gpu_ms(lambda: g.evolve_plain(c["steps"]))
    gre, gim = g.get_state(np.float64)
    obs = g.observe()
    g.close()
    m = oracle.moments(ore, oim)
    return emit({"workload": "256^2 FP64 plain, V=0, 100 steps",
                 "rel_l2": rel_l2(gre, gim, ore, oim),
                 "norm_minus_1": obs["norm"] - 1.0,
                 "dx": obs["x"] - m[1] / m[0], "dy": obs["y"] - m[2] / m[0],
                 "gpu_fp64_plain_site_steps_per_s": n / (ms / 1e3),
                 "oracle_site_steps_per_s_1thr": n / t1,
                 "oracle_site_steps_per_s_nthr": n / tn, "host_cores": NCPU})


def harmonic_2048(seed, fp64_too):
    c = wl.harmonic_2048(seed=seed)
    n = c["nx"] * c["ny"] * c["steps"]
    (ore, oim), tn = timed(lambda: oracle.evolve(c["re"], c["im"], c["V"], c["dt"], c["theta"],
                                                 c["steps"], nthreads=NCPU))
    e0 = sum(oracle.energy(c["re"], c["im"], c["V"]))
    eT = sum(oracle.energy(ore, oim, c["V"]))
    g = trotter.Grid(c["nx"], c["ny"], "f32")
    g.set_state(c["re"], c["im"])
    g.set_potential(c["V"], c["dt"], c["theta"])
    o0 = g.observe()
    ms = gpu_ms(lambda: g.evolve(c["steps"]))
    oT = g.observe()
    gre, gim = g.get_state(np.float64)
    g.close()
    E0, ET = o0["e_kin"] + o0["e_pot"], oT["e_kin"] + oT["e_pot"]
    out = {"workload": "2048^2 harmonic, 1000 steps", "seed": seed,
           "fp32_fused_rel_l2": rel_l2(gre, gim, ore, oim),
           "fp32_norm_drift": abs(oT["norm"] - o0["norm"]),
           "fp32_energy_drift_rel": abs(ET - E0) / max(abs(E0), 1e-12),
           "fp32_energy_drift_abs": abs(ET - E0),
           "oracle_energy_drift_rel": abs(eT - e0) / max(abs(e0), 1e-12),
           "gpu_fp32_fused_site_steps_per_s": n / (ms / 1e3),
           "oracle_site_steps_per_s_nthr": n / tn, "host_cores": NCPU}
    if fp64_too:
        g = trotter.Grid(c["nx"], c["ny"], "f64")
        g.set_state(c["re"], c["im"])
        g.set_potential(c["V"], c["dt"], c["theta"])
        ms = gpu_ms(lambda: g.evolve_plain(c["steps"]))
        dre, dim = g.get_state(np.float64)
        g.close()
        out["fp64_plain_rel_l2"] = rel_l2(dre, dim, ore, oim)
        out["gpu_fp64_plain_site_steps_per_s"] = n / (ms / 1e3)
    return emit(out)


def order4_2048():
    c = wl.harmonic_2048(seed=0, steps=200)
    n = c["nx"] * c["ny"] * c["steps"]
    (ore, oim), tn = timed(lambda: oracle.evolve(c["re"], c["im"], c["V"], c["dt"], c["theta"],
                                                 c["steps"], order=4, nthreads=NCPU))
    g = trotter.Grid(c["nx"], c["ny"], "f32")
    g.set_state(c["re"], c["im"])
    g.set_potential(c["V"], c["dt"], c["theta"], order=4)
    o0 = g.observe()
    ms = gpu_ms(lambda: g.evolve(c["steps"]))
    oT = g.observe()
    gre, gim = g.get_state(np.float64)
    g.close()
    return emit({"workload": "2048^2 harmonic, 200 fourth-order steps", "seed": 0,
                 "fp32_rel_l2": rel_l2(gre, gim, ore, oim),
                 "fp32_norm_drift": abs(oT["norm"] - o0["norm"]),
                 "gpu_fp32_site_steps_per_s": n / (ms / 1e3),
                 "oracle_site_steps_per_s_nthr": n / tn, "host_cores": NCPU})


def driven_2048():
    c = wl.harmonic_2048(seed=2)
    n, dt, steps = c["nx"], c["dt"], c["steps"]
    V1 = (np.arange(n) - n / 2.0)[None, :] * np.ones((n, 1))
    a = 2e-3 * np.cos(0.05 * (np.arange(steps) + 0.5) * dt)
    (ore, oim), tn = timed(lambda: oracle.evolve_driven(c["re"], c["im"], c["V"], V1, a, dt,
                                                        c["theta"], nthreads=NCPU))
    g = trotter.Grid(n, n, "f32")
    g.set_state(c["re"], c["im"])
    g.set_potential(c["V"], dt, c["theta"])
    g.set_drive(V1, a)
    o0 = g.observe()
    ms = gpu_ms(lambda: g.evolve(steps))
    oT = g.observe()
    gre, gim = g.get_state(np.float64)
    g.close()
    return emit({"workload": "2048^2 harmonic + field along x, a = 2e-3 cos(0.05 t), 1000 steps",
                 "seed": 2, "fp32_rel_l2": rel_l2(gre, gim, ore, oim),
                 "fp32_norm_drift": abs(oT["norm"] - o0["norm"]),
                 "gpu_fp32_site_steps_per_s": n * n * steps / (ms / 1e3),
                 "oracle_site_steps_per_s_nthr": n * n * steps / tn, "host_cores": NCPU})


def roofline_sizes():
    import torch
    rows = []
    for side in (8192, 16384):
        c = wl.roofline_grid(n=side, seed=0, steps=200)
        steps_o = 10
        _, tn = timed(lambda: oracle.evolve(c["re"], c["im"], c["V"], c["dt"], c["theta"],
                                            steps_o, nthreads=NCPU))
        row = {"workload": "%d^2 random Gaussians" % side,
               "oracle_site_steps_per_s_nthr": side * side * steps_o / tn,
               "oracle_steps": steps_o, "host_cores": NCPU}
        if side == 8192:
            _, t1 = timed(lambda: oracle.evolve(c["re"], c["im"], c["V"], c["dt"], c["theta"], 2,
                                                nthreads=1))
            row["oracle_site_steps_per_s_1thr"] = side * side * 2 / t1
        re = torch.from_numpy(c["re"].astype(np.float32)).cuda()
        im = torch.from_numpy(c["im"].astype(np.float32)).cuda()
        V = torch.from_numpy(c["V"]).cuda()
        g = trotter.Grid(side, side, "f32")
        g.set_potential(V, c["dt"], c["theta"])
        fused = {}
        for K in range(1, 9):
            g.set_state(re, im)
            g.evolve(2 * K, K)
            ms = gpu_ms(lambda: g.evolve(200, K))
            fused[K] = side * side * 200 / (ms / 1e3)
        row["gpu_fp32_fused_site_steps_per_s"] = fused
        g.set_state(re, im)
        ms = gpu_ms(lambda: g.evolve_plain(10))
        row["gpu_fp32_plain_site_steps_per_s"] = side * side * 10 / (ms / 1e3)
        g.close()
        g = trotter.Grid(side, side, "f64")
        g.set_state(c["re"], c["im"])
        g.set_potential(V, c["dt"], c["theta"])
        g.evolve_plain(1)
        ms = gpu_ms(lambda: g.evolve_plain(10))
        row["gpu_fp64_plain_site_steps_per_s"] = side * side * 10 / (ms / 1e3)
        g.close()
        del re, im, V
        torch.cuda.empty_cache()
        rows.append(emit(row))
    return rows


def adjoint_1024():
    c = wl.adjoint_pair(n=1024, steps=500, seed=0)
    steps = c["steps"]
    g = trotter.Grid(c["nx"], c["ny"], "f32")
    g.set_state(c["re"], c["im"])
    g.set_potential(c["V"], c["dt"], c["theta"])
    res = {}

    def run():
        res["F"], res["grad"] = trotter.adjoint_fidelity_grad(g, c["target_re"], c["target_im"],
                                                              steps, 50)
    run()
    g.set_state(c["re"], c["im"])
    ms = gpu_ms(run)
    g.close()
    grad = res["grad"].double().cpu().numpy()
    (og, oF, _), tn = timed(lambda: oracle.adjoint_grad(
        c["re"], c["im"], c["target_re"], c["target_im"], c["V"], c["dt"], c["theta"], steps,
        nthreads=NCPU))
    rng = np.random.default_rng(123)
    weight = c["re"] ** 2 + c["im"] ** 2 + c["target_re"] ** 2 + c["target_im"] ** 2
    cand = np.flatnonzero(weight.ravel() > 1e-3 * weight.max())
    sites = rng.choice(cand, 64, replace=False)
    h = 1e-3
    g64 = trotter.Grid(c["nx"], c["ny"], "f64")

    def fid(V):
        g64.set_state(c["re"], c["im"])
        g64.set_potential(V, c["dt"], c["theta"])
        g64.evolve_plain(steps)
        re, im = g64.get_state(np.float64)
        return abs(np.vdot(c["target_re"] + 1j * c["target_im"], re + 1j * im)) ** 2
    fd = np.zeros(len(sites))
    for i, j in enumerate(sites):
        Vp, Vm = c["V"].copy(), c["V"].copy()
        Vp.flat[j] += h
        Vm.flat[j] -= h
        fd[i] = (fid(Vp) - fid(Vm)) / (2 * h)
    g64.close()
    gs = grad.ravel()[sites]
    return emit({"workload": "1024^2 adjoint, 500 steps, checkpoints every 50",
                 "F_gpu": res["F"], "F_oracle": oF,
                 "grad_vs_fd_rel_l2_64_sites": float(np.linalg.norm(gs - fd) / np.linalg.norm(fd)),
                 "grad_vs_oracle_rel_l2": float(np.linalg.norm(grad - og) / np.linalg.norm(og)),
                 "gpu_forward_backward_ms": ms, "oracle_adjoint_s_nthr": tn,
                 "host_cores": NCPU})


def main():
    trotter.load()
    out = {"c1": plain_fp64_256(),
           "c2": [harmonic_2048(s, s == 0) for s in range(5)],
           "order4": order4_2048(),
           "drive": driven_2048(),
           "c3": roofline_sizes(),
           "c5": adjoint_1024()}
    c2 = out["c2"]
    emit({"summary": True,
          "c2_max_rel_l2": max(r["fp32_fused_rel_l2"] for r in c2),
          "c2_max_norm_drift": max(r["fp32_norm_drift"] for r in c2),
          "c2_max_energy_drift_rel": max(r["fp32_energy_drift_rel"] for r in c2)})
    return 0


if __name__ == "__main__":
    sys.exit(main())
