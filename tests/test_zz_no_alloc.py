"""The allocation-free diagnostics entry point, checked against lbm_diag.

lbm_diag_fields_noalloc is for callers that cannot allocate device memory
(their device memory belongs to another allocator, or cudaMalloc's implicit
synchronisation is not acceptable on their path).  It reduces field arrays the
caller already owns, with its partial sums in a static device array.  This
file runs last in the suite so that a failure here leaves every other test
already run; it passes alone in a fresh process as well.
"""
import ctypes

import numpy as np
import pytest

from paper_1701_00702_gb300 import inputs

pytestmark = pytest.mark.gpu

KEYS = ("melt_frac", "nu_hot", "enthalpy", "mass")


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1701_00702_gb300 import build, lbm as mod
    build.build()
    return mod


def _noalloc_diag(lbm, solver, out):
    fields = solver.fields(names=("T_f", "T_s", "f_l", "rho", "H_f"), device=True)
    lbm.diag_fields_noalloc(solver.params, fields, out, stream=solver.stream)
    solver.stream.synchronize()
    return out.cpu().numpy().copy()


# FP64: FP64 rounding; the FP32-field modes: the melt fraction and Nusselt
# number to FP64 rounding of the same FP32 values, enthalpy and mass to the
# ~1e-7 the FP32 fields carry (no float-float low part, rho rounded to FP32)
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-6), (2, 1e-6), (3, 1e-6)])
def test_noalloc_diag_matches_lbm_diag_on_two_calls_in_a_row(lbm, prec, tol):
    """Two consecutive calls (a large grid, then a smaller one that reuses the
    same static scratch) agree with lbm_diag on the same states."""
    import torch
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")   # caller-owned output
    runs = [(inputs.cavity(320, ny=288, precision=prec), 300), (inputs.cavity(64, ny=48, precision=prec), 120)]
    for p, steps in runs:
        s = lbm.Solver(p)
        s.step(steps)
        got = _noalloc_diag(lbm, s, out)
        ref = s.diag()
        for i, k in enumerate(KEYS):
            assert abs(got[i] / ref[k] - 1.0) < tol, (k, got[i], ref[k])
        s.close()


def test_noalloc_diag_rejects_grids_beyond_its_scratch(lbm):
    import torch
    small = torch.zeros(4, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    p = inputs.cavity(8192, ny=8193, precision=1)
    ptr = ctypes.c_void_p(small.data_ptr())
    rc = lbm.lib().lbm_diag_fields_noalloc(ctypes.byref(lbm.to_struct(p)), ptr, ptr, ptr, ptr, ptr,
                                           ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -8
    assert "static scratch" in lbm.strerror(rc)
    assert np.all(out.cpu().numpy() == 0.0)      # nothing was launched
