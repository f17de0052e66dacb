"""Small-case driver for Nsight Compute captures of the library's kernels (measurement
support beside bench.py, not part of the package).

Runs ``--steps`` HEVI 1D-IMEX ARK2 steps (and optionally RK35 steps) of the benchmark's
workload shape on a smaller box: ``--nex`` x ``--nex`` x 12 elements of order 4 over
(2.083 km * nex)^2 x 15 km, the same element size as the benchmark.  The default nex = 72
gives a 164 MB state (larger than the 129 MB L2) and about 1.7 GB of device memory.
Every step reads the same input and writes a separate output.

  python profile_case.py [--nex 72] [--steps 3] [--rk 0] [--adj 0] [--precision mixed]
                         [--scheme ark5] [--solve 0] [--imex3d 0]

--adj K also runs K adjoint steps (numa_step_imex1d_adjoint) and K tangent-linear steps from
the same input, for captures of the differentiation form's kernels.  --scheme selects the
ARK scheme of the steps (ark2 .. ark5; FP64).  --solve K runs K standalone column solves
(numa_solve_columns) of a seeded right-hand side.  --imex3d K runs K 3D-IMEX steps of a
separate 3D context (polynomial preconditioner) from the same input.
"""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nex", type=int, default=72)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--rk", type=int, default=0)
    ap.add_argument("--adj", type=int, default=0)
    ap.add_argument("--C", type=float, default=15.0)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "rhs32", "df"])
    ap.add_argument("--scheme", default="ark2", choices=["ark2", "ark3", "ark4", "ark5"])
    ap.add_argument("--solve", type=int, default=0)
    ap.add_argument("--imex3d", type=int, default=0)
    a = ap.parse_args()
    import torch
    import paper_1702_04316_gb300 as pkg
    import synthetic

    nex, nez, N = a.nex, 12, 4
    L, Lz = 200e3 / 96 * nex, 15e3
    xi = np.array([-1.0, -np.sqrt(3.0 / 7.0), 0.0, np.sqrt(3.0 / 7.0), 1.0])
    c_s = (1004.67 / (1004.67 - 287.17) * 287.17 * 300.0) ** 0.5
    dt = a.C * (xi[1] + 1.0) / 2.0 * (Lz / nez) / c_s
    g = pkg.Numa(nex, nex, nez, L, L, Lz, N, dt, precision=a.precision, scheme=a.scheme)
    lev = g.reference_levels()
    h = L / nex
    ax = np.concatenate([e * h + (1.0 + xi[:-1]) * h / 2.0 for e in range(nex)] + [[L]])
    q0 = torch.from_numpy(synthetic.balanced_state(ax, ax, lev["z"], L, L, Lz, lev["rho0"],
                                                   lev["theta0"], 7)).cuda()
    q1 = torch.empty_like(q0)
    for _ in range(a.steps):
        g.step_imex1d(q0, q1, 1)
    for _ in range(a.rk):
        g.step_explicit_rk(q0, dt / a.C, q1, 1)
    if a.adj:
        lam = torch.empty_like(q0).copy_(q0)
        for _ in range(a.adj):
            g.step_imex1d_adjoint(q0, lam, q1)
        g.step_imex1d_tlm(q0, lam, a.adj, q1, torch.empty_like(q0))
    if a.solve:
        gen = torch.Generator(device="cuda").manual_seed(11)
        b = torch.randn(g.ncol * g.M, dtype=torch.float64, device="cuda", generator=gen)
        x = torch.empty_like(b)
        for _ in range(a.solve):
            g.solve_columns(b, x)
        assert bool(torch.isfinite(x).all())
    if a.imex3d:
        g3 = pkg.Numa(nex, nex, nez, L, L, Lz, N, dt, imex="3d")
        q3 = torch.empty_like(q0)
        g3.step_imex3d(q0, q3, a.imex3d)
        torch.cuda.synchronize()
        assert g3.count_nonfinite(q3) == 0 and g3.status() == pkg.NUMA_OK
        g3.close()
    torch.cuda.synchronize()
    assert g.count_nonfinite(q1) == 0
    assert g.status() == pkg.NUMA_OK
    g.close()
    print("profile_case ok: nex=%d steps=%d rk=%d adj=%d scheme=%s" % (nex, a.steps, a.rk, a.adj,
                                                                       a.scheme))


if __name__ == "__main__":
    main()
