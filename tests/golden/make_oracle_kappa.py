"""Write tests/golden/oracle_kappa_diffusion3d_128.txt: the oracle's 200-step Lanczos (full
reorthogonalisation by classical Gram-Schmidt applied twice) estimates of kappa (Sec. 3.1,
kappa = lambda_max / lambda_min of the SPD operator) for the 3D diffusion workload at the size
the bench times (128^3 grid, sigma 2, b ~ N(0,1) seed 0): A itself, and the block-Jacobi
preconditioned operator L^-1 A L^-T at block size 16 (Sec. 3.2-3.3 with full diagonal blocks).

Only the oracle (oracle/) and the seeded input generators run here; nothing comes from the
CUDA path.  The oracle's loops may use several threads; its results do not depend on how many.

Usage: python tests/golden/make_oracle_kappa.py [threads]
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2410_02408_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "oracle_kappa_diffusion3d_128.txt")


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    oracle.set_threads(threads)
    A = W.diffusion3d(128, 2.0)
    b = W.rhs(A.n, 0)
    rows = []
    for name, bs in (("before", 0), ("after_bs16", 16)):
        t0 = time.time()
        k = oracle.kappa(A, b, 200, bs)
        rows.append((name, k, time.time() - t0))
        print(name, repr(k["kappa"]), f"{time.time() - t0:.1f} s", flush=True)
    with open(OUT, "w") as f:
        f.write("# Oracle kappa estimates, 3D 7-point diffusion 128^3 (sigma 2, face coefficients seed 1),\n")
        f.write("# start vector b = default_rng(0).standard_normal(N) (L^-1 b / ||L^-1 b|| after), 200 Lanczos\n")
        f.write("# steps with CGS2 reorthogonalisation, extreme Ritz values by Sturm bisection (Sec. 3.1:\n")
        f.write("# kappa = lambda_max / lambda_min).  Written by tests/golden/make_oracle_kappa.py (oracle only).\n")
        f.write("#\n# name          steps  kappa                   lambda_min              lambda_max\n")
        for name, k, _ in rows:
            f.write(f"{name:<14} {k['steps']:<6} {k['kappa']!r:<23} {k['lambda_min']!r:<23} {k['lambda_max']!r}\n")
    print("wrote", OUT)


if __name__ == "__main__":
    main()
