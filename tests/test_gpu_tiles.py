"""Tile shapes of the point-parallel kernels (elements per CTA): either shape, and the
autotuner's pick, give the same residuals, JVPs and linearised products to rounding
(the per-point operations are the same; the separately compiled kernels may contract
multiply-adds differently)."""
import numpy as np
import pytest

from paper_1903_06304_gb300 import inputs as inp

from gpu_helpers import case, solver_for, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("cfg", [(5, 3, 1, 0.1, 10.0, 1.0, True), (7, 5, 2, 0.05, 10.0, 1.0, True),
                                 (9, 4, 3, 0.05, 0.0, 1.0, False), (3, 5, 4, 0.2, 10.0, 1.0, True)],
                         ids=lambda c: f"p{c[2]}")
def test_tile_shapes_agree_to_rounding(torch, cfg):
    nx, ny, p, mach, re, kappa, deforming = cfg
    c, v, q = case(nx, ny, p, mach, re, kappa, deforming)
    vec = to_dev(inp.random_vector(q.shape, 5))
    outs = {}
    for tiles in (1, 2, 0):
        S = solver_for(c, v, nx, ny, p, mach, re, kappa, tiles=tiles)
        if tiles:
            assert set(S.tiles.values()) == {tiles}
        else:
            assert set(S.tiles.values()) <= {1, 2}
        qd = to_dev(q)
        R, J, L = (torch.empty(S.shape, dtype=torch.float64, device="cuda:0") for _ in range(3))
        S.residual(qd, R)
        S.jvp(qd, vec, J, 1e-20, 150.0)
        S.linearize(qd, 1e-20, 150.0)
        S.apply_linear(vec, L)
        outs[tiles] = [to_host(x) for x in (R, J, L)]
    for tiles in (2, 0):
        for a, b in zip(outs[1], outs[tiles]):
            assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()
