"""Writes br_shell_128_activation.npz: the FP64 oracle's activation map of the
quarter-scale Beeler-Reuter shell (the ellipsoidal shell of workloads.br_shell
at n = 128: outer semi-axes 50/50/60 nodes, wall 10, helical fibres, apex
stimulus), run for the full 500 ms (25 000 steps of 0.02 ms) from the
float32-rounded initial state the GPU test starts from.  Calls only the
oracle (and the seeded input generators); the GPU parity test compares the
library's activation map with it.

    python tests/golden/make_br_shell_activation.py [n_threads]

Takes about ten minutes on eight cores (threads do not change the result).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1605_06015_gb300 import workloads as wl  # noqa: E402

OUT = os.path.join(HERE, "br_shell_128_activation.npz")


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    oracle.set_threads(threads)
    w = wl.br_shell(128)
    rest = oracle.rest_state(w.model, w.params)
    st0 = w.initial_state(rest).astype(np.float32).astype(np.float64)
    g = oracle.Grid(w.nx, w.ny, w.nz, w.h, w.mask, w.fibres, w.D_par, w.D_perp)
    sim = oracle.Sim(g, w.model, par=w.params, theta=w.theta, state=st0)
    sim.step(w.dt, w.n_steps)
    tis = w.mask.reshape(-1) != 0
    np.savez_compressed(OUT, act=sim.act.reshape(-1)[tis].astype(np.int32), n_steps=np.int64(w.n_steps),
                        dt=np.float64(w.dt), n=np.int64(128), n_tissue=np.int64(tis.sum()))
    a = sim.act.reshape(-1)[tis]
    print("wrote", OUT, "tissue", int(tis.sum()), "activated", int((a < oracle.INT32_MAX).sum()),
          "latest", int(a[a < oracle.INT32_MAX].max()))


if __name__ == "__main__":
    main()
