"""The element-block inversion on the tensor cores (blocked Gauss-Jordan with BF16 rank-16
updates, FP32 accumulation): at every degree B_e z_e = r_e in the oracle's FP64 blocks to
the accuracy the BF16 operands allow, the split-operand form to near-FP32 accuracy and
close to the SIMT FP32 inverse, and GMRES with either takes the iterations of the FP32
inverse on the benchmark's linear systems."""
import numpy as np
import pytest

from gpu_helpers import case, oracle_problem, solver_for, to_dev, to_host
from oracle import solver as sv
from paper_1903_06304_gb300 import inputs as inp

pytestmark = pytest.mark.gpu

# Relative residual of B_e z_e = r_e, about twice the measured worst element: BF16 operands
# (8-bit mantissa) in each of the b/16 rank-16 updates of the equilibrated block, with the
# Gauss-Jordan multipliers above the pivot (not bounded by one) and the block's condition
# number amplifying them, grow from 1e-2 (b = 16) to 0.5 (b = 100): a coarse preconditioner,
# like BF16 storage; split operands (about 16 bits) stay near FP32 Gauss-Jordan (2e-5 to
# 1e-3).  Index: degree p.
TOL = {("tc_bf16", "fp32"): {1: 3e-2, 2: 2e-1, 3: 4e-1, 4: 1.0},
       ("tc_bf16", "bf16"): {1: 3e-2, 2: 2e-1, 3: 4e-1, 4: 1.1},
       ("tc_bf16x3", "fp32"): {1: 1e-4, 2: 3e-4, 3: 1e-3, 4: 3e-3},
       ("tc_bf16x3", "fp64"): {1: 1e-4, 2: 3e-4, 3: 1e-3, 4: 3e-3}}


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _block_residual(Bo, got, r):
    ne, bs = Bo.shape[0], Bo.shape[1]
    ge = got.transpose(1, 0, 2, 3).reshape(ne, bs)
    re_ = r.transpose(1, 0, 2, 3).reshape(ne, bs)
    return np.linalg.norm(np.einsum("eab,eb->ea", Bo, ge) - re_, axis=1) / np.linalg.norm(re_, axis=1)


@pytest.mark.parametrize("mode,prec", list(TOL))
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_tensor_core_inverse_every_degree(torch, p, mode, prec):
    nx, ny, mach, re, kappa = 4, 3, 0.05, 10.0, 1.0
    c, v, q = case(nx, ny, p, mach, re, kappa, True)
    prob = oracle_problem(c, v, nx, ny, p, mach, re, kappa)
    Bo = sv.block_jacobian(prob, q, 0.0, 150.0)
    r = inp.random_vector(q.shape, 5 + p)
    S = solver_for(c, v, nx, ny, p, mach, re, kappa, prec=prec, factor=mode)
    S.precond_build(to_dev(q), 0.0, 150.0)
    z = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
    S.precond_apply(to_dev(r), z)
    rel = _block_residual(Bo, to_host(z), r)
    print(f"p={p} {mode} {prec}: max relative block residual {rel.max():.2e}")
    assert rel.max() <= TOL[(mode, prec)][p], rel.max()
    S.close()


@pytest.mark.parametrize("p", [2, 3])
def test_split_operands_close_to_the_simt_inverse(torch, p):
    """The split-operand tensor-core inverse and the SIMT FP32 Gauss-Jordan inverse apply
    to the same vector within 1e-3 (both FP32-stored), and the one-product BF16 form is
    within its own rounding of them."""
    nx, ny, mach, re, kappa = 6, 5, 0.01, 10.0, 1.0
    c, v, q = case(nx, ny, p, mach, re, kappa, True)
    r = to_dev(inp.random_vector(q.shape, 3))
    out = {}
    for mode in ("simt", "tc_bf16x3", "tc_bf16"):
        S = solver_for(c, v, nx, ny, p, mach, re, kappa, prec="fp32", factor=mode)
        S.precond_build(to_dev(q), 0.0, 150.0)
        z = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
        S.precond_apply(r, z)
        out[mode] = to_host(z)
        S.close()
    scale = np.abs(out["simt"]).max()
    assert np.abs(out["tc_bf16x3"] - out["simt"]).max() <= 1e-3 * scale
    assert np.abs(out["tc_bf16"] - out["simt"]).max() <= 5e-2 * scale


def test_gmres_iterations_with_tensor_core_blocks(torch):
    """The benchmark's linear system (64 x 64, p = 3 vortex, GMRES(30), 1e-6): the tensor-core
    inverses give the iteration count of the SIMT FP32 inverse within a few iterations."""
    w = inp.NS_VORTEX_64
    c, v, q = inp.make_case(w, t=0.13)
    qd = to_dev(q)
    b = to_dev(inp.random_vector(q.shape, 23))
    its = {}
    for mode in ("simt", "tc_bf16x3", "tc_bf16"):
        S = solver_for(c, v, w.nx, w.ny, w.p, w.mach, w.re, w.kappa, prec="fp32", factor=mode,
                       maxit_lin=400)
        S.precond_build(qd, 1e-20, 1.5 / w.dt)
        x = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
        its[mode] = S.gmres(qd, b, x, 1e-20, 1.5 / w.dt)
        S.close()
    assert abs(its["tc_bf16x3"] - its["simt"]) <= max(2, 0.05 * its["simt"]), its
    assert its["tc_bf16"] <= 1.3 * its["simt"] + 5, its
