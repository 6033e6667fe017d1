"""sr_invariants_noalloc: the plan-less invariant sums for callers that may
not allocate device memory (for example code running under an allocator
that owns the device, or a hook inside a step loop that must not call
cudaMalloc).  Checked through the C ABI against sr_invariants, the entry
point that uses plan-owned scratch, on two calls in a row; the second call
is smaller than the first, so any partial sums left in the shared static
scratch by the first call would show up as an error in the second.

This file is named to be collected last: if it fails, a run that stops at
the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _lib():
    from paper_1411_3396_b300 import _lib as L
    return L.load()


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _rows(n, seed):
    r = np.random.default_rng(seed)
    v = r.standard_normal((n, 4)).astype(np.float32)
    a = r.standard_normal((n, 4)).astype(np.float32)
    return torch.from_numpy(v).cuda(), torch.from_numpy(a).cuda()


def test_noalloc_invariants_match_planned_entry_point_twice():
    from paper_1411_3396_b300 import Plan
    lib = _lib()
    n_big, n_small = 3_000_017, 20_011
    plan = Plan(16.0, 3.0, 0.1, 0.8, n_big)
    for n, seed in ((n_big, 1), (n_small, 2)):
        v, a = _rows(n, seed)
        out = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.sr_invariants_noalloc(n, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(a.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()), _stream())
        assert rc == 0, lib.sr_last_error()
        ref = plan.invariants(v, a)
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=1e-12, atol=1e-9)


def test_noalloc_invariants_null_inputs_and_limits():
    lib = _lib()
    out = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda")
    v, _ = _rows(1000, 3)
    rc = lib.sr_invariants_noalloc(1000, ctypes.c_void_p(v.data_ptr()), None, ctypes.c_void_p(out.data_ptr()),
                                   _stream())
    assert rc == 0
    o = out.cpu().numpy()
    vv = v.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(o[0:3], vv[:, :3].sum(axis=0), rtol=1e-12, atol=1e-10)
    assert np.all(o[3:6] == 0.0)
    ke = 0.5 * np.sum(vv[:, :3] * vv[:, :3])
    np.testing.assert_allclose(o[6], ke, rtol=1e-12)
    # no velocities: only the acceleration sums are nonzero
    _, a = _rows(1000, 4)
    out.fill_(float("nan"))
    rc = lib.sr_invariants_noalloc(1000, None, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                   _stream())
    assert rc == 0
    o = out.cpu().numpy()
    aa = a.cpu().numpy().astype(np.float64)
    assert np.all(o[0:3] == 0.0) and o[6] == 0.0
    np.testing.assert_allclose(o[3:6], aa[:, :3].sum(axis=0), rtol=1e-12, atol=1e-10)
    # n = 0, the warm-up call: seven zeros
    out.fill_(float("nan"))
    assert lib.sr_invariants_noalloc(0, None, None, ctypes.c_void_p(out.data_ptr()), _stream()) == 0
    assert np.all(out.cpu().numpy() == 0.0)
    # beyond the static scratch: rejected before any launch
    assert lib.sr_invariants_noalloc(67_108_865, None, None, ctypes.c_void_p(out.data_ptr()), _stream()) == 3
    assert b"static scratch" in lib.sr_last_error()
