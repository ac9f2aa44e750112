"""Write mlmc_2d_5levels_oracle_y.txt: the oracle's per-sample level
differences Y_l = Q_l - Q_{l-1} (eq. StandardML, Q_{-1} = 0) of the
five-level 2D MLMC workload, every sample of every level pair over the
whole horizon.

Workload: nested unit-square meshes of 17^2, 33^2, 65^2, 129^2 and 257^2
nodes, dt_l = 0.1 2^-l over T = 10 (100 .. 1600 time blocks), 4096 / 1024 /
256 / 64 / 16 samples, K = 16 KL modes of 0.09 exp(-|x - y|^2 / 0.04) built
on the 257^2 mesh and moved to every level by the midpoint rule (Sec. 4),
xi from the counter-based sample points (seed 0, stream = level).  The
coarse member of pair l solves level l - 1 with the xi of pair l.

Only the oracle and the seeded sample points are used.  On 8 host cores the
run takes about 40 minutes:

    python tests/golden/make_mlmc_2d_5levels_oracle.py
"""
from __future__ import annotations

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_2105_02007_gb300 import inputs  # noqa: E402

LEVEL_M = [17, 33, 65, 129, 257]
LEVEL_N = [4096, 1024, 256, 64, 16]
K = 16
OUT = os.path.join(HERE, "mlmc_2d_5levels_oracle_y.txt")


def main():
    fine = O.mesh2d(LEVEL_M[-1])
    modes, _ = O.kl_build(fine, 0.09, 0.04, K)
    meshes = [O.mesh2d(m) for m in LEVEL_M]
    phis = [O.centroid_table(fine, modes, mm) for mm in meshes]
    dts = [0.1 * 0.5 ** l for l in range(len(LEVEL_M))]
    steps = [int(round(10.0 / dt)) for dt in dts]
    ys = []
    for l, N in enumerate(LEVEL_N):
        xi = inputs.gaussian_xi(0, l, 0, N, K)
        qf, _, sf = O.solve_batch(meshes[l], phis[l], xi, dts[l], steps[l])
        assert np.all(sf == 0)
        y = qf
        if l > 0:
            qc, _, sc = O.solve_batch(meshes[l - 1], phis[l - 1], xi, dts[l - 1], steps[l - 1])
            assert np.all(sc == 0)
            y = qf - qc
        ys.append(y)
        sys.stderr.write(f"level {l} done\n")
        sys.stderr.flush()
    est, var, rmse = O.mlmc_estimate(ys)
    with open(OUT, "w") as f:
        f.write("# Y_l = Q_l - Q_{l-1} per sample (eq. StandardML), five-level 2D MLMC workload, written by\n")
        f.write("# make_mlmc_2d_5levels_oracle.py from the FP64 oracle (every sample, whole horizon)\n")
        f.write(f"estimate {est:.17e}\n")
        f.write("var " + " ".join(f"{v:.17e}" for v in var) + "\n")
        f.write(f"rmse {rmse:.17e}\n")
        for l, y in enumerate(ys):
            f.write(f"level {l} {y.size}\n")
            for v in y:
                f.write(f"{v:.17e}\n")


if __name__ == "__main__":
    main()
