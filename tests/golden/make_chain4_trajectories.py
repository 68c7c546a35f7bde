"""Writes the FP64 oracle's reference trajectories of the 4-bead chain and the
3D dumbbell in shear (Sec. 3.3, simple shear; Appendix A, explicit scheme)
that the GPU tests compare final-time stresses against.

Calls only ``oracle`` and the seeded input generator; nothing here touches the
CUDA library.  The runs are too long for a test (tens of minutes of FP64
O(N^2) steps on the host cores), so their results are stored as small JSON
fixtures beside this script:

  chain4_n16384_hookean_T5.json   N = 16384, Hookean, t in [0, 5] (1000 steps)
  chain4_n65536_hookean_s100.json N = 65536, Hookean, 100 steps
  chain4_n65536_fene50_s100.json  N = 65536, FENE b = 50, 100 steps
  dumbbell3d_n16384_rate{0.1,1,10}_T5.json  one bond in 3D (D = 3), N = 16384,
                                  Silverman bandwidth, t in [0, 5]

The chain runs: nb = 3 bonds in s = 3 dimensions (D = 9), H_k = 1, kBT = 1,
zeta = 4, shear rate 1 (kappa_12 = 1), dt = 0.005, the equilibrium Gaussian
cloud of seed 0 (FENE: redrawn into the domain), bandwidth by the median rule
of the initial cloud (Eq. model_bandwidth; order statistic found by pair
counting).  The dumbbell runs: one bond, the same constants, shear rates 0.1,
1 and 10, the Silverman bandwidth of the initial cloud.  Stored per checkpoint: the paper's polymer stress tau (s x s) and
the second moments <q q^T> (D x D); at the end also every 256th particle's
connector vector.

Usage: python tests/golden/make_chain4_trajectories.py [case ...]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2603_12550_gb300 import inputs  # noqa: E402

CASES = {
    "chain4_n16384_hookean_T5": dict(N=16384, spring=0, b=0.0, steps=1000, every=100),
    "chain4_n65536_hookean_s100": dict(N=65536, spring=0, b=0.0, steps=100, every=25),
    "chain4_n65536_fene50_s100": dict(N=65536, spring=1, b=50.0, steps=100, every=25),
    # the 3D Hookean dumbbell (one bond, D = 3) at the three shear rates of
    # its workload, Silverman bandwidth, t in [0, 5]
    "dumbbell3d_n16384_rate0.1_T5": dict(N=16384, nb=1, rate=0.1, bw="silverman", spring=0, b=0.0,
                                         steps=1000, every=200),
    "dumbbell3d_n16384_rate1_T5": dict(N=16384, nb=1, rate=1.0, bw="silverman", spring=0, b=0.0,
                                       steps=1000, every=200),
    "dumbbell3d_n16384_rate10_T5": dict(N=16384, nb=1, rate=10.0, bw="silverman", spring=0, b=0.0,
                                        steps=1000, every=200),
}
NB, S, DT, RATE, SEED, ROW_STRIDE = 3, 3, 0.005, 1.0, 0, 256


def run(name):
    c = CASES[name]
    N, nb, rate = c["N"], c.get("nb", NB), c.get("rate", RATE)
    q32 = inputs.equilibrium_cloud(N, nb, S, seed=SEED, fene_b=c["b"] if c["spring"] else None)
    q = q32.astype(np.float64)
    t0 = time.time()
    h = oracle.silverman_bandwidth(q) if c.get("bw") == "silverman" else oracle.median_bandwidth_count(q)
    kap = inputs.shear_kappa(S, rate)
    p = oracle.params(nb, S, H=1.0, kBT=1.0, zeta=4.0, h=h, dt=DT, kappa=kap,
                      spring=c["spring"], b=c["b"])
    ckpt = []
    done = 0
    while done < c["steps"]:
        n = min(c["every"], c["steps"] - done)
        q = oracle.explicit_steps(q, p, n)
        done += n
        tau, qq = oracle.stress(q, p)
        ckpt.append(dict(step=done, tau=tau.tolist(), qq=qq.tolist()))
        print(f"{name}: step {done} tau_11 {tau[0, 0]:.9f} ({time.time() - t0:.0f} s)", flush=True)
    rows = list(range(0, N, ROW_STRIDE))
    out = dict(
        _source="FP64 oracle (oracle/vds_oracle.c explicit steps), written by "
                "tests/golden/make_chain4_trajectories.py; Appendix A explicit scheme, "
                "Sec. 3.3 shear set-up, stress of Sec. 2.1",
        N=N, nb=nb, s=S, H=[1.0] * nb, kBT=1.0, zeta=4.0, dt=DT, rate=rate, bandwidth=c.get("bw", "median"),
        spring=c["spring"], b=c["b"], seed=SEED, h=h, steps=c["steps"],
        checkpoints=ckpt, rows=rows, q_rows=q[rows].tolist(),
        oracle_seconds=round(time.time() - t0, 1))
    path = os.path.join(HERE, name + ".json")
    with open(path + ".tmp", "w") as f:
        json.dump(out, f)
    os.replace(path + ".tmp", path)


if __name__ == "__main__":
    for name in (sys.argv[1:] or list(CASES)):
        run(name)
