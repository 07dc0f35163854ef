"""Multigrid Poisson solve through the C ABI (ek_poisson_solve_mg): the same
periodic problem of Eq. 3 the FFT solves, reached by V-cycles; checked
against the oracle's FFT solve element by element, with the V-cycle count and
the residual it reports, on boxes with several levels, with an odd coarsest
edge, and one that cannot be coarsened (solved by the FFT in one cycle)."""
import numpy as np
import pytest

from oracle import ek_oracle as O

pytestmark = pytest.mark.gpu

LB = 0.7
SHAPES = [(32, 32, 32), (48, 32, 64), (64, 32, 128), (128, 128, 128), (24, 18, 32), (36, 32, 32),
          (12, 96, 27)]


def _solve(ek, q, shape, tol=1e-12, max_cycles=40, inplace=False):
    import torch
    nx, ny, nz = shape
    qd = torch.tensor(q.ravel(), device="cuda", dtype=torch.float64)
    phi = qd if inplace else torch.full_like(qd, 7.0)  # the solver overwrites phi
    scratch = torch.empty(ek.poisson_mg_scratch_bytes(shape), dtype=torch.uint8, device="cuda")
    cycles, res = ek.poisson_solve_mg(qd, phi, shape, LB, scratch, tol=tol, max_cycles=max_cycles)
    return phi.cpu().numpy().reshape(nz, ny, nx), cycles, res


@pytest.mark.parametrize("shape", SHAPES)
def test_multigrid_matches_the_fft_oracle(gpu_lib, shape):
    ek = gpu_lib
    nx, ny, nz = shape
    rng = np.random.default_rng(5)
    q = rng.random((nz, ny, nx)) - 0.3  # nonzero mean: the k = 0 mode is dropped
    ref = O.poisson(q, LB)
    got, cycles, res = _solve(ek, q, shape)
    assert res <= 1e-12
    assert 1 <= cycles <= 20, cycles  # about a tenth of the residual per V-cycle
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) <= 1e-10 * scale
    assert abs(got.mean()) <= 1e-13 * scale


def test_multigrid_in_place_tolerance_and_arguments(gpu_lib):
    import torch
    ek = gpu_lib
    shape = (32, 32, 32)
    rng = np.random.default_rng(6)
    q = rng.random(shape[::-1]) - 0.5
    ref = O.poisson(q, LB)
    got, cycles, _ = _solve(ek, q, shape, inplace=True)
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
    # a looser tolerance stops earlier, with the residual it reports
    _, c2, r2 = _solve(ek, q, shape, tol=1e-4)
    assert c2 < cycles and r2 <= 1e-4
    # the cycle limit is honoured
    _, c3, r3 = _solve(ek, q, shape, max_cycles=2)
    assert c3 == 2 and r3 > 1e-12
    # a uniform charge has the zero solution, without any cycle
    got, c4, r4 = _solve(ek, np.full(shape[::-1], 0.25), shape)
    assert c4 == 0 and r4 == 0.0 and np.all(got == 0.0)
    # invalid arguments are status codes
    qd = torch.zeros(32 ** 3, device="cuda", dtype=torch.float64)
    scratch = torch.empty(ek.poisson_mg_scratch_bytes(shape), dtype=torch.uint8, device="cuda")
    for kw in (dict(tol=0.0), dict(max_cycles=0)):
        with pytest.raises(ek.EKError) as e:
            ek.poisson_solve_mg(qd, qd, shape, LB, scratch, **kw)
        assert e.value.code == -1
    with pytest.raises(ek.EKError):
        ek.poisson_solve_mg(qd, qd, (10, 32, 32), LB, scratch)  # 10 is not 2^a 3^b
    assert ek.poisson_mg_scratch_bytes((10, 32, 32)) == 0
