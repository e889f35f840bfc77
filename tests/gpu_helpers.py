"""Shared helpers of the GPU parity tests: seeded cases, oracle twins, tolerances."""
from __future__ import annotations

import numpy as np

from oracle import physics as ph
from oracle import residual as rs
from oracle import scale as sc
from oracle import solver as sv
from paper_1903_06304_gb300 import inputs as inp


def case(nx, ny, p, mach, re, kappa, deforming, seed=3, rel=0.1, t=0.13):
    ref = inp.box_mesh(nx, ny, 0, 10, 0, 10)
    c, v = inp.deform(ref, t, inp.Motion()) if deforming else (ref, np.zeros_like(ref))
    q = inp.random_perturbation(inp.uniform_state(nx * ny, p, mach, 0.8, 0.3), seed, rel, mach)
    return c, v, q


def oracle_problem(c, v, nx, ny, p, mach, re, kappa):
    gas = ph.Gas(mach=mach, re=re, kappa=kappa)
    return sv.Problem(rs.Mesh(nx, ny, c, v), p, gas)


def to_dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda:0")


def to_host(t):
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def solver_for(c, v, nx, ny, p, mach, re, kappa, **kw):
    from paper_1903_06304_gb300 import fr
    S = fr.Solver(fr.Config(p=p, mach=mach, re=re, kappa=kappa, **kw), nx, ny)
    S.update_mesh(to_dev(c), to_dev(v))
    return S


# Parity tolerances (see the tolerance derivation in the design notes):
#  residual: |R_gpu - R_ora|_k <= RES_TOL * sigma_k, sigma_k = magnitude of the terms summed
#            into equation k (oracle.scale.residual_scale);
#  JVP:      |Av_gpu - Av_ora|_k <= JVP_TOL * max|Av_ora|_k;
#  blocks:   per row group k, <= BLK_TOL * max|B_ora[rows of k]|.
RES_TOL = 1e-12
JVP_TOL = 1e-12
BLK_TOL = 1e-11


def residual_errors(R_gpu, R_ora, q, mesh, p, gas):
    s = sc.residual_scale(q, mesh, p, gas)
    return np.abs(R_gpu - R_ora).max(axis=(1, 2, 3)) / s


def jvp_errors(A_gpu, A_ora):
    return np.abs(A_gpu - A_ora).max(axis=(1, 2, 3)) / np.abs(A_ora).max(axis=(1, 2, 3))


def block_errors(B_gpu, B_ora, np2):
    out = []
    for k in range(4):
        rows = slice(k * np2, (k + 1) * np2)
        out.append(np.abs(B_gpu[:, rows] - B_ora[:, rows]).max() / np.abs(B_ora[:, rows]).max())
    return np.array(out)
