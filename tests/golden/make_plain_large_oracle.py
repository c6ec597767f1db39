"""Write tests/golden/plain_large_oracle.txt: the oracle's full solve of the
n = 1e6 convection-diffusion workload (2-D, N = 1000, beta = 100, d = 50,
Arnoldi(50, 25), nev = 20, rtol = 1e-8, smallest real part).

Calls only the oracle and the seeded input generator.  Takes about an hour on
8 host cores; run from the repository root:
    python tests/golden/make_plain_large_oracle.py
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from oracle.ppa import make_operator  # noqa: E402
from paper_1806_08020_gb300 import inputs  # noqa: E402


def main(out=os.path.join(ROOT, "tests", "golden", "plain_large_oracle.txt"), max_cycles=400):
    cfg = inputs.plain_large()
    A = O.to_scipy(cfg["A"])
    n = A.shape[0]
    c = O.Counters()
    sigma = O.gershgorin_shift(A)
    op = O.Operator(A, sigma, c)
    b = inputs.start_vector(n, cfg["seed"], 0)
    v0 = inputs.start_vector(n, cfg["seed"], 1)
    t0 = time.time()
    P = O.build_poly(op, b, cfg["d"], c)
    t_build = time.time() - t0

    def log(cycle, r):
        print(f"cycle {cycle} max_resid {r:.3e} t {time.time() - t0:.0f}s", flush=True)

    R = O.eigs(A, make_operator(op, P, c), cfg["nev"], cfg["m"], cfg["k"], cfg["rtol"], v0, c,
               target="SR", sigma=sigma, max_cycles=max_cycles, log=log)
    t = time.time() - t0
    with open(out, "w") as f:
        f.write("# Oracle full solve (written by tests/golden/make_plain_large_oracle.py; oracle only).\n")
        f.write(f"# workload {cfg['name']}: 2-D CD N=1000 beta=100, d=50, Arnoldi(50,25), nev=20, rtol=1e-8, SR\n")
        f.write(f"converged {int(R.converged)}\ncycles {R.cycles}\nmvps {c.mvps}\ndots {c.dots}\nvops {c.vops}\n")
        f.write(f"degree {P.degree}\nadded {P.added}\nseconds {t:.1f}\nbuild_seconds {t_build:.2f}\n")
        for j, (lam, res) in enumerate(zip(R.lam, R.resid)):
            f.write(f"lam{j} {lam.real:.17g} {lam.imag:.17g} {res:.6e}\n")
    print("wrote", out, R.converged, R.cycles, t)


if __name__ == "__main__":
    main()
