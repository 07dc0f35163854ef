"""The Poisson entry point that allocates nothing (ek_poisson_solve_static).

Some callers cannot call cudaMalloc: code whose device memory is all reserved
by another runtime's pool, loops that must not let the allocator synchronise
the device, code that may not allocate after start-up.  This entry point keeps
its scratch in fixed device arrays instead.  Its output must equal the
allocating entry point's (ek_poisson_solve) within the Poisson tolerance of the
other GPU tests, on two calls in a row (the second call finds the first
call's data in the shared scratch).  This file is collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _reference(ek, q, shape):
    import torch
    nx, ny, nz = shape
    phi = torch.empty_like(q)
    spec = torch.empty(ek.poisson_scratch_bytes(nx, ny, nz) // 8, dtype=torch.float64,
                       device="cuda")
    ek.poisson_solve(q, phi, shape, 0.7, spec)
    return phi


def test_static_poisson_two_calls_match_allocating_entry_point(gpu_lib):
    import torch
    ek = gpu_lib
    rng = np.random.default_rng(1607)
    for shape in [(48, 32, 64), (48, 32, 64), (24, 16, 18)]:
        nx, ny, nz = shape
        q = torch.from_numpy(rng.standard_normal(nx * ny * nz)).cuda()
        ref = _reference(ek, q, shape)
        out = torch.empty_like(q)
        ek.poisson_solve_static(q, out, shape, 0.7)
        torch.cuda.synchronize()
        scale = float(ref.abs().max())
        assert float((out - ref).abs().max()) <= 1e-12 * scale


def test_static_poisson_shape_changes_in_order_on_one_stream(gpu_lib):
    """Calls queued back to back on a non-default stream, changing the box
    shape between them with no synchronisation: each table reload is ordered
    after the solves already queued, so every result equals the allocating
    solve of its own shape."""
    import torch
    ek = gpu_lib
    rng = np.random.default_rng(1608)
    shapes = [(48, 32, 64), (24, 16, 18), (48, 32, 64), (32, 36, 24), (24, 16, 18)]
    qs = [torch.from_numpy(rng.standard_normal(s[0] * s[1] * s[2])).cuda() for s in shapes]
    refs = [_reference(ek, q, s) for q, s in zip(qs, shapes)]
    torch.cuda.synchronize()
    outs = [torch.full_like(q, float("nan")) for q in qs]
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        for q, out, s in zip(qs, outs, shapes):
            ek.poisson_solve_static(q, out, s, 0.7, stream=st)
    st.synchronize()
    for out, ref in zip(outs, refs):
        scale = float(ref.abs().max())
        assert float((out - ref).abs().max()) <= 1e-12 * scale


def test_static_poisson_rejects_too_large_box(gpu_lib):
    import torch
    ek = gpu_lib
    q = torch.zeros(128 * 128 * 128, dtype=torch.float64, device="cuda")
    with pytest.raises(ek.EKError):
        ek.poisson_solve_static(q, q, (128, 128, 128), 0.7)
