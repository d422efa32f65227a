"""Writes tests/golden/stencil_8x8x8x8_inertia.json with the oracle only: the number of eigenvalues of
the seeded 8^4 stencil below a shift between the golden's lambda_nev and the next eigenvalue.

    python tests/golden/make_inertia.py

1. lambda_{nev+1}: the oracle's Algorithm 1 for nev + 1 eigenvalues (residual 1e-10).
2. sigma = (lambda_nev + lambda_{nev+1}) / 2, with lambda_nev from tests/golden/stencil_8x8x8x8.json.
3. The dense A assembled entry by entry from the stencil's definition (oracle.jsym, eq. (4)), and the
   count of its eigenvalues below sigma by Sylvester's law of inertia (oracle.inertia; LAPACK's
   Bunch-Kaufman LDL^H of A - sigma I).  n = 24,576: about 30 GB of memory and a quarter of an hour.
Nothing here touches the CUDA library.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import inertia, jsym  # noqa: E402
from oracle import trlan_jsym as tj  # noqa: E402
from paper_2001_07428_gb300 import inputs  # noqa: E402


def main(name="stencil_8x8x8x8"):
    gold = json.load(open(os.path.join(HERE, f"{name}.json")))
    w = inputs.WORKLOADS[name]
    dims = w["dims"]
    nev = len(gold["evals"])
    U, W = inputs.stencil_links(dims, w["seed"])
    n = 6 * inputs.lattice_volume(dims)
    mv = lambda x: jsym.stencil_matvec(U, W, dims, w["m0"], w["kappa"], x)
    t0 = time.time()
    out = tj.trlan_jsym(mv, n, nev + 1, w["m"], w["mwin"], 1e-10)
    lam_nev, lam_next = max(gold["evals"]), float(out["evals"][nev])
    sigma = 0.5 * (lam_nev + lam_next)
    t1 = time.time()
    A11, A12 = jsym.stencil_blocks_dense(U, W, dims, w["m0"], w["kappa"])
    A = jsym.assemble_block_form(A11, A12)
    del A11, A12
    count = inertia.count_below(A, sigma, overwrite=True)
    rec = dict(workload=name, nev=nev, n=n, lambda_nev=lam_nev, lambda_next=lam_next, sigma=sigma,
               count_below=count, oracle_seconds=round(t1 - t0, 1), inertia_seconds=round(time.time() - t1, 1),
               note="count of eigenvalues of the dense stencil below sigma, by LDL^H inertia; 2 nev means the "
                    "golden's nev eigenvalues (each doubly degenerate) are the nev smallest")
    with open(os.path.join(HERE, f"{name}_inertia.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
