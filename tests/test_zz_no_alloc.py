"""rm_precondition_noalloc: the allocation-free preconditioner entry point.

It is meant for callers that must not allocate device memory while they run
(a device-memory budget owned by another allocator, or code that cannot pay
for the synchronisation cudaMalloc/cudaFree imply).  Its scratch is a static
device array of the library rather than buffers of the handle, so this file
checks that it reproduces rm_precondition on two calls in a row (the array
keeps the previous call's contents), and that it refuses handles it cannot
serve.  The file is collected last so that a run stopping at the first
failure has run every other test; it also passes alone in a fresh process.
"""

import numpy as np
import pytest

from paper_2211_14284_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _solver(**opts):
    from paper_2211_14284_gb300.rm import Solver
    n, p = 3, 3
    X = inputs.vertices(n, perturb=0.1, seed=31)
    al = inputs.loguniform_coefficient(n, 0.1, 10, seed=32)
    be = inputs.loguniform_coefficient(n, 0.1, 10, seed=33)
    return Solver(0, n, p, vertices=X, alpha=al, beta=be, **opts)


def test_noalloc_matches_precondition_twice():
    s = _solver()
    dev = "cuda"
    for call in range(2):
        r = torch.tensor(inputs.normal_rhs(s.size, 40 + call), dtype=torch.float64, device=dev)
        z_ref = torch.empty_like(r)
        z_new = torch.full_like(r, np.nan)
        s.precondition(r, z_ref)
        s.precondition_noalloc(r, z_new)
        torch.cuda.synchronize()
        a, b = z_ref.cpu().numpy(), z_new.cpu().numpy()
        assert np.all(np.isfinite(b))
        # same kernels, same operands; only the order of the atomic
        # scatter-adds may differ, so the preconditioner tolerance applies
        assert np.abs(a - b).max() <= 1e-11 * np.abs(a).max()


def test_noalloc_rejects_condensed_handles():
    from paper_2211_14284_gb300.rm import RmError
    s = _solver(static_condensation=1, factor=1)
    r = torch.zeros(s.size, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    with pytest.raises(RmError, match="lattice-sized scratch"):
        s.precondition_noalloc(r, z)


def _free_bytes():
    free, _ = torch.cuda.mem_get_info()
    return free


def test_noalloc_allocates_nothing():
    """The property the entry point exists for: after a warm-up call, many
    calls leave the device's free memory unchanged (no cudaMalloc, no
    caching-allocator growth)."""
    s = _solver()
    r = torch.tensor(inputs.normal_rhs(s.size, 50), dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    s.precondition_noalloc(r, z)
    torch.cuda.synchronize()
    before = _free_bytes()
    for _ in range(20):
        s.precondition_noalloc(r, z)
    torch.cuda.synchronize()
    assert _free_bytes() == before


def test_noalloc_fp32_and_off_modes():
    """An FP32-preconditioner handle matches rm_precondition, and a handle
    whose coarse term is switched off (RM_CORRECTOR_OFF) is served too."""
    from paper_2211_14284_gb300.rm import RM_CORRECTOR_OFF
    for opts, mode in ((dict(precision=1), None), ({}, RM_CORRECTOR_OFF)):
        s = _solver(**opts)
        if mode is not None:
            s.corrector_use(mode)
        r = torch.tensor(inputs.normal_rhs(s.size, 51), dtype=torch.float64, device="cuda")
        z_ref = torch.empty_like(r)
        z_new = torch.full_like(r, np.nan)
        s.precondition(r, z_ref)
        s.precondition_noalloc(r, z_new)
        torch.cuda.synchronize()
        a, b = z_ref.cpu().numpy(), z_new.cpu().numpy()
        assert np.all(np.isfinite(b))
        assert np.abs(a - b).max() <= 1e-6 * np.abs(a).max()


def test_noalloc_rejects_multigrid_coarse():
    from paper_2211_14284_gb300.rm import RmError
    s = _solver(coarse=2)
    r = torch.zeros(s.size, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    with pytest.raises(RmError, match="multigrid"):
        s.precondition_noalloc(r, z)


def test_noalloc_rejects_deterministic_relaxation():
    """A deterministic handle gathers its patch values from per-patch scratch,
    which this entry point does not use."""
    from paper_2211_14284_gb300.rm import RmError
    s = _solver(deterministic=1)
    r = torch.zeros(s.size, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    with pytest.raises(RmError, match="deterministic"):
        s.precondition_noalloc(r, z)
