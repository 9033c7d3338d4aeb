"""Write tests/golden/oracle_iterations.txt: SQMR iteration counts of the CPU oracle (Alg. 4 with the
Alg. 1/3 V-cycle, FP64) on the Gaussian-bump workloads, to the stated relative residual.

Calls only oracle/ and synthetic/ (no CUDA code).  Usage:
    python tests/golden/make_oracle_iterations.py 256:0:1e-8 128:0:1e-8
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synthetic  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_iterations.txt")


def main(specs):
    rows = []
    if os.path.exists(OUT):
        rows = [l.rstrip("\n") for l in open(OUT) if l.strip() and not l.startswith("#")]
    for spec in specs:
        n, seed, tol = spec.split(":")
        n, seed, tol = int(n), int(seed), float(tol)
        prob = synthetic.bumps(n, seed=seed)
        t0 = time.time()
        o = oracle.Oracle(n, coarsest_max=8)
        b = o.rhs(prob["f"].numpy(), None)
        t1 = time.time()
        x, rc, it, rr, hist = o.sqmr(b, tol=tol, maxit=200)
        t2 = time.time()
        rows = [r for r in rows if not r.startswith(f"{n}, {seed}, {tol:g},")]
        rows.append(f"{n}, {seed}, {tol:g}, {it}, {rr:.3e}, {t2 - t1:.1f}")
        print(rows[-1], f"setup {t1 - t0:.1f}s", flush=True)
    with open(OUT, "w") as f:
        f.write("# oracle MG-SQMR on Gaussian bumps (16 bumps, eta = 1, gamma = 1e-3, k_b = 1), x0 = 0\n")
        f.write("# columns: n (n^3 cells), seed, tol, iterations, final true rel. residual, solve seconds (1 x86 core)\n")
        for r in sorted(rows, key=lambda s: [float(v) for v in s.split(",")[:3]]):
            f.write(r + "\n")


if __name__ == "__main__":
    main(sys.argv[1:])
