"""Solves through the checked-index library (test helper, run as a child
process with HZ_LIB set to libhz_checked.so by test_gpu_checked.py).

Each case solves with the CUDA path and with the oracle at the same tolerance
and prints one line; the last line is the library's checked-index status.
Exit code 0 only if every case agreed and no access left its array."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import workloads  # noqa: E402
from pairs import AGREE, l2_rel, make_pair, medium  # noqa: E402

CASES = [
    dict(dim=2, n=65, levels=3, patch="plus", scheme="leveldep", precision="mixed"),
    dict(dim=2, n=129, levels=4, patch="rb", scheme="leveldep", precision="mixed", layer=8),
    dict(dim=2, n=65, levels=3, patch="element", scheme="cubic", precision="fp64"),
    dict(dim=3, n=17, levels=3, patch="element", scheme="linear", precision="mixed", alpha=0.5),
    dict(dim=3, n=17, levels=3, patch="jacobi", scheme="linear", precision="mixed", alpha=0.5,
         patch_coarse="element"),
    dict(dim=2, n=65, levels=3, patch="rb", scheme="leveldep", precision="mixed", stencil="compact"),
    dict(dim=2, n=65, levels=3, patch="plus", scheme="leveldep", precision="mixed", cycle="W"),
]


def run_case(c):
    kw = {k: v for k, v in c.items() if k not in ("dim", "n", "levels", "patch", "scheme")}
    orc, gpu = make_pair(c["dim"], c["n"], c["levels"], c["patch"], c["scheme"], **kw)
    n, dim = c["n"], c["dim"]
    q = workloads.point_source((n,) * dim, tuple([(n - 1) // 2] * dim), 1.0 / (n - 1)).ravel()
    p, info = gpu.solve(torch.tensor(q, device="cuda"))
    p_o, info_o = orc.solve(q.copy(), tol=1e-7)
    err = l2_rel(p.cpu().numpy(), p_o)
    gpu.close()
    ok = info.converged == 1 and abs(info.iters - info_o.iters) <= 1 and err <= AGREE[c["precision"]]
    return ok, {"case": c, "iters": info.iters, "oracle_iters": info_o.iters, "err": err}


def run_batched():
    from oracle import solver as osolver
    from paper_2511_16808_gb300.solver import HelmholtzSolver
    n, R = 65, 16
    h, omega, kappa, gamma = medium(2, n, 0, 8)
    orc = osolver.Problem((n, n), h, kappa, omega, gamma, 0.25, 3, "rb", "leveldep")
    gpu = HelmholtzSolver(2, [n, n], kappa, omega, gamma, 0.25, 3, patch="rb", intergrid="leveldep",
                          precision="mixed", tol=1e-7, nrhs_max=R)
    rng = np.random.default_rng(3)
    nodes = [tuple(int(v) for v in rng.integers(2, n - 2, size=2)) for _ in range(R)]
    Q = np.stack([workloads.point_source((n, n), nd, h).ravel() for nd in nodes], axis=1)
    P, infos = gpu.solve_batch(torch.tensor(Q, device="cuda"))
    P = P.cpu().numpy()
    ok = True
    out = []
    for r in (0, R - 1):
        p_o, info_o = orc.solve(Q[:, r].copy(), tol=1e-7)
        err = l2_rel(P[:, r], p_o)
        ok = ok and infos[r].converged == 1 and abs(infos[r].iters - info_o.iters) <= 1 and err <= AGREE["mixed"]
        out.append({"rhs": r, "iters": infos[r].iters, "oracle_iters": info_o.iters, "err": err})
    gpu.close()
    return ok, {"case": "batched 65^2 x 16 (tensor-core coarsest product)", "rhs": out}


def main():
    from paper_2511_16808_gb300 import hz
    torch.cuda.set_device(0)
    st0 = hz.hz_check_status(clear=True)
    all_ok = st0["enabled"]
    for c in CASES:
        ok, rec = run_case(c)
        all_ok = all_ok and ok
        print(json.dumps(dict(rec, ok=ok)), flush=True)
    ok, rec = run_batched()
    all_ok = all_ok and ok
    print(json.dumps(dict(rec, ok=ok)), flush=True)
    torch.cuda.synchronize()
    st = hz.hz_check_status()
    print(json.dumps({"check_status": st, "library": hz.LIB_PATH}), flush=True)
    return 0 if all_ok and st["failures"] == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
