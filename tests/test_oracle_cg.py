"""Pins for the oracle's conjugate-gradient solver on -L x = f (the Krylov use, Sec. 4)."""
import numpy as np

import oracle
from paper_1905_08375_gb300 import synth


def test_cg_matches_dense_solve_scalar():
    n = 20
    f = synth.heterogeneous_2d(n=n, seed=2)
    rhs = synth.cg_rhs(n, seed=3)[0]
    kw = dict(alpha=1.5, coef=oracle.COEF_XY, a=f["a"])
    x, it, rr = oracle.cg(rhs, 2, n, f["delta"], rtol=1e-10, **kw)
    assert rr <= 1e-10 and it > 5
    N = n * n
    A = np.zeros((N, N))
    E = np.eye(N)
    for j in range(N):
        A[:, j] = -oracle.direct_scalar(E[j], 2, n, f["delta"], symmetric=True, **kw)
    xd = np.linalg.solve(A, rhs)                     # LAPACK, independent of CG
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-8


def test_jacobi_cuts_iterations_and_pd_cg_converges():
    n = 24
    f = synth.heterogeneous_2d(n=n, seed=5)
    rhs = synth.cg_rhs(n, seed=6)[0]
    kw = dict(alpha=1.5, coef=oracle.COEF_XY, a=f["a"], rtol=1e-8)
    _, it_j, rr_j = oracle.cg(rhs, 2, n, f["delta"], jacobi=True, **kw)
    _, it_p, rr_p = oracle.cg(rhs, 2, n, f["delta"], jacobi=False, **kw)
    assert rr_j <= 1e-8 and rr_p <= 1e-8 and it_j <= it_p
    p = synth.pd_2d(n=16, seed=1, radius_cells=3)
    rhs2 = np.random.default_rng(0).standard_normal(2 * 16 * 16)
    x, it, rr = oracle.cg(rhs2, 2, 16, p["delta"], kind="pd", c=p["c"], rtol=1e-9)
    assert rr <= 1e-9
    Lx = oracle.pd_direct(x.reshape(2, -1), 2, 16, p["delta"], p["c"]).reshape(-1)
    assert np.linalg.norm(-Lx - rhs2) / np.linalg.norm(rhs2) < 1e-8
