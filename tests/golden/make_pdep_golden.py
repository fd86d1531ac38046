"""Writes tests/golden/pdep_L16_48.txt: the 64 leading PDEP eigenvalues of the 48^3 model.

Calls only the oracle (block Davidson of oracle/pdep.py on the static sum over
states of oracle/chi0.py) and the seeded generator.  Takes tens of minutes on a
few CPU cores.  Start block: synth.perturbations(miller_rho, L, 64, seed=11).
Run from the repository root:  python tests/golden/make_pdep_golden.py
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import chi0, pdep  # noqa: E402
from oracle.model import Model  # noqa: E402


def main():
    s = synth.make_system("pdep_L16_48")
    m = Model(s.L, s.ecut, s.grid, s.vloc_G, s.psi_v, s.e_v)
    t0 = time.time()
    states = chi0._states(m)
    print(f"eigh done {time.time() - t0:.0f} s", flush=True)
    x0 = synth.perturbations(s.miller_rho, s.L, 64, 11)
    calls = [0]

    def apply(V):
        calls[0] += V.shape[1]
        out = m.vsqrt[:, None] * chi0.sos_static_block(m, m.vsqrt[:, None] * V, states)
        print(f"  applied {V.shape[1]} vectors ({calls[0]} total) at {time.time() - t0:.0f} s", flush=True)
        return out

    theta, X, it = pdep.davidson(apply, m.mr.shape[0], 64, x0, tol=1e-11, max_iter=200)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pdep_L16_48.txt")
    with open(path, "w") as f:
        f.write("# 64 leading eigenvalues of chi0bar(w=0) for synth config pdep_L16_48 (well seed 9),\n")
        f.write(f"# oracle block Davidson (tol 1e-11, {it} iterations, {calls[0]} applications), "
                "start block synth.perturbations(miller_rho, L, 64, seed=11)\n")
        for t in theta:
            f.write(f"{t:.17e}\n")
    print("wrote", path, theta[:4], flush=True)


if __name__ == "__main__":
    main()
