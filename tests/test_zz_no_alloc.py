"""GPU check of fr_residual_noalloc, the residual entry point for callers that cannot
allocate device memory (graph capture, foreign allocators, runtimes that own all device
memory): through the C ABI, two calls in a row on different states must match the
context-based fr_residual within the residual parity tolerance, and a mesh larger than
the static scratch must be refused before any GPU work.  This file is collected last so
that a run stopping at the first failure has run every other test first."""
import ctypes

import numpy as np
import pytest

from gpu_helpers import RES_TOL, case, oracle_problem, residual_errors, solver_for, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def _noalloc(lib, cfg, nx, ny, corners, vel, q, out, stream):
    return lib.fr_residual_noalloc(ctypes.byref(cfg), nx, ny, ctypes.c_void_p(corners.data_ptr()),
                                   ctypes.c_void_p(vel.data_ptr()), ctypes.c_void_p(q.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


@pytest.mark.parametrize("cfg", [(9, 7, 3, 0.05, 10.0, 1.0, True), (6, 5, 2, 0.01, 0.0, 1.0, False)])
def test_noalloc_matches_context_residual_twice(torch, cfg):
    from paper_1903_06304_gb300 import fr
    nx, ny, p, mach, re, kappa, deforming = cfg
    lib = fr.load()
    c, v, q1 = case(nx, ny, p, mach, re, kappa, deforming, seed=3)
    _, _, q2 = case(nx, ny, p, mach, re, kappa, deforming, seed=4)
    S = solver_for(c, v, nx, ny, p, mach, re, kappa)
    prob = oracle_problem(c, v, nx, ny, p, mach, re, kappa)
    cc = S.cfg.to_c()
    dc, dv = to_dev(c), to_dev(v)
    stream = torch.cuda.current_stream().cuda_stream
    for q in (q1, q2):
        qd = to_dev(q)
        want = torch.empty(S.shape, dtype=torch.float64, device="cuda:0")
        S.residual(qd, want)
        got = torch.full(S.shape, float("nan"), dtype=torch.float64, device="cuda:0")
        assert _noalloc(lib, cc, nx, ny, dc, dv, qd, got, stream) == 0
        err = residual_errors(to_host(got), to_host(want), q, prob.mesh, p, prob.gas)
        assert np.all(err <= RES_TOL), err
    S.close()


def test_noalloc_rejects_meshes_beyond_the_scratch(torch):
    from paper_1903_06304_gb300 import fr
    lib = fr.load()
    cc = fr.Config(p=3).to_c()
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    # 81 x 81 = 6561 elements > 6528 at p = 3: refused before the pointers are touched
    assert _noalloc(lib, cc, 81, 81, dummy, dummy, dummy, dummy, stream) == -1
