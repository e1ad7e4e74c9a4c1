"""Error table of FP32 / BF16 / FP16 population storage (needs a GPU).

Part 1: against the FP64 oracle on lattices it finishes quickly (the D2Q9
channel at its full 128x64 size, scaled mixer and exchanger lattices).
Part 2: at the full 512x256x256 heat exchanger, where the oracle cannot run,
BF16 and FP16 against the FP32 GPU path, with the device time of one solve.

    python tests/precision_report.py [--skip-full]
"""
import argparse
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle.solver import Oracle  # noqa: E402
from paper_1501_04741_gb300 import inputs  # noqa: E402
from paper_1501_04741_gb300.albm import Solver  # noqa: E402


def gpu_run(P, theta):
    with Solver(P, torch.from_numpy(theta.reshape(-1)).cuda()) as s:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.primal_step(P.nsteps)
        f = s.populations(0).double().cpu().numpy()
        J = s.objective()
        s.adjoint_step(P.nsteps)
        g = s.gradient().cpu().numpy()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    return f, J, g, dt


def part1():
    cases = {
        "channel2d 128x64 BGK, 2000+2000": inputs.channel2d(),
        "mixer3d 40x20x20 MRT+2 scalars, 1000+1000": inputs.scaled(inputs.mixer3d(), (40, 20, 20),
                                                                   nsteps=1000, obj_window=100),
        "exchanger3d 56x28x28 BGK+T, 1200+1200": inputs.scaled(inputs.exchanger3d(), (56, 28, 28),
                                                               nsteps=1200),
    }
    print("| workload | storage | populations err / max|f| | J rel err | dJ/dtheta rel err (inf) |")
    print("|---|---|---|---|---|")
    for name, P in cases.items():
        th = inputs.theta_grf(P, 0) if "exchanger" in name else inputs.theta_uniform(P, 0)
        o = Oracle(P, th)
        J, g, _ = o.gradient()
        _, traj = o.primal(keep=False)
        fN = traj[-1].reshape(o.model.M, -1).numpy()
        g = g.reshape(-1).numpy()
        for prec in ("fp32", "bf16", "fp16"):
            f_gpu, J_gpu, grad, _ = gpu_run(P.replace(precision=prec), th)
            print(f"| {name} | {prec} | {np.abs(f_gpu - fN).max() / np.abs(fN).max():.2e} | "
                  f"{abs(J_gpu - J) / abs(J):.2e} | {np.abs(grad - g).max() / np.abs(g).max():.2e} |",
                  flush=True)


def part2():
    P = inputs.exchanger3d()
    th = inputs.theta_grf(P, 0)
    res = {}
    for prec in ("fp32", "bf16", "fp16"):
        f, J, g, dt = gpu_run(P.replace(precision=prec), th)
        res[prec] = (f, J, g, dt)
    f0, J0, g0, _ = res["fp32"]
    print("\n| exchanger3d 512x256x256, 1000+1000 | storage | J | J rel diff vs FP32 | "
          "dJ/dtheta rel diff vs FP32 (inf) | populations diff / max|f| | solve s |")
    print("|---|---|---|---|---|---|---|")
    for prec, (f, J, g, dt) in res.items():
        print(f"| | {prec} | {J:.6e} | {abs(J - J0) / abs(J0):.2e} | "
              f"{np.abs(g - g0).max() / np.abs(g0).max():.2e} | "
              f"{np.abs(f - f0).max() / np.abs(f0).max():.2e} | {dt:.2f} |", flush=True)


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--skip-full", action="store_true")
    a = ap.parse_args()
    part1()
    if not a.skip_full:
        part2()
