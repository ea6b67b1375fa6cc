"""Writes tests/golden/n11_reconstruction_fidelity.txt from the FP64 oracle only.

Workload (the Fig. 2-4 setting of Sec. 4: noise-free probabilities): N = 11, the Haar pure
state of seed 20, f = its exact Born probabilities of the tetrahedral POVM (Sec. 3.3 eq. PS,
clipped at 0, renormalised and rounded to float32: the input the library receives), the network
initialised from seed 23 (float32 values).  The oracle runs the Fig. 1 loop (Sec. 3.1 network,
Sec. 3.2 Chol_H, likelihood, Rprop of Sec. 4.1) and records the state fidelity
<psi| rho^ |psi> (Sec. 2.3, pure target) after each listed number of iterations.  Only oracle/
and the seeded input generators are called.  Takes a few minutes on a multi-core host.

    python tests/golden/make_n11_fidelity.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2207_05341_gb300 import synth  # noqa: E402

N = 11
STATE_SEED = 20
THETA_SEED = 23
CHECKPOINTS = (20, 50)
OUT = os.path.join(HERE, "n11_reconstruction_fidelity.txt")


def inputs():
    """psi, f (float32) and theta0 (float32) of the workload."""
    psi = synth.haar_pure(N, STATE_SEED)
    P = O.born_probabilities(synth.pure_density(psi), O.tetrahedral_povm()).real
    P = np.clip(P, 0.0, None)
    f = (P / P.sum()).astype(np.float32)
    theta = synth.init_theta(N, THETA_SEED).astype(np.float32)
    return psi, f, theta


def read(path=OUT):
    """{iterations: fidelity} from the stored file."""
    out = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            k, F = line.split()
            out[int(k)] = float(F)
    return out


def main():
    psi, f, theta = inputs()
    M = O.tetrahedral_povm()
    th = theta.astype(np.float64)
    f64 = f.astype(np.float64)
    st = O.RpropState(th.size)
    out = {}
    for it in range(1, max(CHECKPOINTS) + 1):
        _, g, _ = O.loss_and_grad(th, f64, M, N)
        th = O.rprop_update(th, g, st)
        if it in CHECKPOINTS:
            out[it] = O.fidelity_pure(O.state_from_theta(th, f64, N), psi)
            print(it, out[it], flush=True)
    with open(OUT, "w") as fh:
        fh.write("# N = 11 Chol_H reconstruction from exact probabilities (Sec. 4, Figs. 2-4 setting):\n")
        fh.write("# <psi|rho^|psi> after k Rprop iterations of the FP64 oracle, written by make_n11_fidelity.py\n")
        for k, F in out.items():
            fh.write(f"{k} {F:.12f}\n")


if __name__ == "__main__":
    main()
