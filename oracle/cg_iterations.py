"""Run the oracle's CG to convergence on the benchmark system (3D Poisson 128^3,
b = A x*, x* ~ U[-1, 1] seed 2002, x0 = 0, tol 1e-10) and store its iteration
count and single-core time in cg_iterations_poisson3d_128.json, against which
the full-size GPU test checks the library's iteration count.  Calls only the
oracle and the input generators."""
import json
import sys
import time
from pathlib import Path

sys.path.insert(0, str(Path(__file__).resolve().parents[1]))

import oracle  # noqa: E402
from paper_2411_10143_b300 import workloads as W  # noqa: E402

if __name__ == "__main__":
    A = W.poisson3d(128)
    b = oracle.spmv(A, W.vector(A.nrows, 2002))
    t0 = time.perf_counter()
    r = oracle.cg(A, b, tol=1e-10)
    dt = time.perf_counter() - t0
    out = {"grid": 128, "tol": 1e-10, "iters": r.iters, "relres_true": r.relres_true,
           "status": r.status, "seconds_one_core": dt}
    (Path(__file__).parent / "cg_iterations_poisson3d_128.json").write_text(json.dumps(out))
    print(out)
