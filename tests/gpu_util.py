"""Helpers shared by the GPU parity tests (comparison only, no method arithmetic)."""
import numpy as np

F64_TOL = 1e-12      # maps and stencils, float64
F32_TOL = 1e-5       # maps and stencils, float32
F64_RED_TOL = 1e-10  # reductions, float64
F32_RED_TOL = 1e-4   # reductions, float32


def tol_for(dtype):
    return F32_TOL if dtype == "f32" else F64_TOL


def red_tol_for(dtype):
    return F32_RED_TOL if dtype == "f32" else F64_RED_TOL


def to_dev(a):
    import torch
    a = np.asarray(a)
    if not a.flags.c_contiguous:
        a = a.copy()
    return torch.from_numpy(a).cuda()


def to_host(t):
    return t.detach().cpu().numpy()


def assert_close(got, ref, tol, scale, what=""):
    """Elementwise mixed bound |got - ref| <= tol * max(|ref|, scale)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    err = np.abs(got - ref)
    bound = tol * np.maximum(np.abs(ref), scale)
    bad = ~(err <= bound)
    if bad.any():
        idx = np.unravel_index(int(np.argmax(np.where(bad, err / np.maximum(bound, 1e-300), 0))),
                               got.shape)
        raise AssertionError("%s: %d of %d elements outside tol %g; worst at %s: got %r ref %r"
                             % (what, int(bad.sum()), bad.size, tol, idx, got[idx], ref[idx]))
