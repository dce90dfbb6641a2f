"""Writes tests/golden/oracle_solve_heat2d_128_N512.json: the FP64 oracle's
Algorithm 1 (PiTSBiCG) run on the 2D heat workload (128 x 128 interior
points, nu = 1e-2, T = 1, N = 512 slices, 50 RK4 fine steps per slice, one IE
coarse step, seed of the heat2d recipe, relative tolerance 1e-6).

Calls only oracle/ and the seeded input generator.  Stored: iteration and
matvec counts, the residual history, the error against the serial fine
trajectory, and sampled solution values (every 64th slice at 16 fixed
points) so that full-size GPU results can be checked point by point.

Also writes tests/golden/oracle_serial_heat2d_128_N512_every32.npy: the
oracle's serial fine trajectory (the exact solution of eq. (4)) on every
32nd slice boundary, lambda_0, lambda_32, ..., lambda_512 = y(T), in full
(17 x 16384 float64 values), for element-by-element checks of full-size
GPU solves.

Run:  python tests/golden/make_oracle_solve_heat2d.py   (several minutes)
      python tests/golden/make_oracle_solve_heat2d.py --serial-only   (the .npy alone)
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import OracleProblem, pitsbicg  # noqa: E402
from paper_2203_10148_gb300 import inputs  # noqa: E402

SAMPLE_POINTS = [0, 1, 127, 128, 1000, 4095, 5000, 8191, 8256, 9999, 12000, 16000, 16255,
                 16256, 16382, 16383]
SAMPLE_SLICES = list(range(0, 513, 64))
EVERY = 32
SERIAL_NPY = os.path.join(HERE, "oracle_serial_heat2d_128_N512_every32.npy")


def write_serial_slices(lam):
    np.save(SERIAL_NPY, np.ascontiguousarray(lam[::EVERY], dtype=np.float64))


def main():
    w = inputs.heat2d()
    o = OracleProblem.from_workload(w)
    t0 = time.time()
    lam = o.serial_fine()
    t_serial = time.time() - t0
    write_serial_slices(lam)
    if "--serial-only" in sys.argv:
        print(f"wrote {SERIAL_NPY} ({t_serial:.1f} s)")
        return
    t0 = time.time()
    X, info = pitsbicg(o, tol=1e-6)
    t_solve = time.time() - t0
    err = float(np.linalg.norm(X - lam) / np.linalg.norm(lam))
    out = {
        "citation": "Algorithm 1 (PiTSBiCG) on eq. (8); exact solution = serial fine trajectory, eq. (7) left",
        "workload": w.describe(),
        "tol_rel": 1e-6,
        "iterations": info.iterations,
        "matvecs": info.matvecs,
        "restarts": info.restarts,
        "status": info.status,
        "r0": info.r0,
        "history": info.history,
        "rel_err_vs_serial": err,
        "oracle_seconds_solve": t_solve,
        "oracle_seconds_serial": t_serial,
        "sample_slices": SAMPLE_SLICES,
        "sample_points": SAMPLE_POINTS,
        "X_samples": [[float(X[n, i]) for i in SAMPLE_POINTS] for n in SAMPLE_SLICES],
        "serial_samples": [[float(lam[n, i]) for i in SAMPLE_POINTS] for n in SAMPLE_SLICES],
    }
    with open(os.path.join(HERE, "oracle_solve_heat2d_128_N512.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in ("iterations", "matvecs", "rel_err_vs_serial",
                                          "oracle_seconds_solve")}))


if __name__ == "__main__":
    main()
