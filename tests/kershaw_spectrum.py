"""Spectrum of the Jacobi-scaled Hessian of the Kershaw benchmark mesh at its
start (paper Sec. 4.1: 9^3 Gauss points, mu_303, eps_y = eps_z = 0.3,
sliding boundaries) and the MINRES iterations the FP64 oracle needs per
relative tolerance, on small meshes (dense Hessian: ndof actions).  Explains
why a 50-iteration MINRES cap always binds on the 24^3 mesh.

    python tests/kershaw_spectrum.py [--big]     # --big adds the 6x6x6 and 12x4x4 meshes (~30 min)
"""
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_2205_12721_b300 import meshgen as mg  # noqa: E402


def main(big=False):
    O.build()
    cases = [(1, (6, 2, 2)), (1, (6, 4, 4)), (2, (6, 2, 2))]
    if big:
        cases += [(1, (6, 6, 6)), (1, (12, 4, 4))]
    for p, n in cases:
        m = mg.kershaw(p, n, 0.3, 0.3)
        om = O.Mesh(3, p, 9, m.map, m.num_nodes, 303, m.fixed)
        x = m.x.copy()
        t0 = time.time()
        H = O.dense_hessian(om, x)
        dg = O.hessian_diag(om, x)
        free = np.flatnonzero(m.fixed == 0)
        d = np.abs(dg[free])
        ev = np.linalg.eigvalsh(H[np.ix_(free, free)] / np.sqrt(np.outer(d, d)))
        g = O.gradient(om, x)
        its = {}
        for rtol in (1e-2, 1e-4, 1e-6, 1e-8, 1e-12):
            its[f"{rtol:g}"] = O.minres(om, x, dg, g, rtol=rtol, max_it=2000)[2]
        print(json.dumps({"p": p, "n": list(n), "free_dofs": int(len(free)),
                          "negative_eigenvalues": int((ev < 0).sum()),
                          "kappa_abs": float(np.abs(ev).max() / np.abs(ev).min()),
                          "minres_iterations": its, "seconds": round(time.time() - t0, 1)}), flush=True)


if __name__ == "__main__":
    main("--big" in sys.argv)
