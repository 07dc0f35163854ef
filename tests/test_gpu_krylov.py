"""The conjugate-gradient Poisson solve with an inhomogeneous permittivity and
fixed-potential nodes (ek_poisson_solve_cg; Sec. III.C, the paragraph after
Eq. 16) against the oracle's sparse direct solve of the same discrete
problem, against the FFT solve where the two problems coincide, and against
the closed form of two dielectrics between fixed planes."""
import numpy as np
import pytest

from oracle import ek_oracle as O

pytestmark = pytest.mark.gpu

LB = 0.7


def solve(ek, q, eps=None, fixed=None, phi_fixed=None, tol=1e-13, max_iter=50000, stream=None):
    import torch
    shape_zyx = q.shape
    shape = (shape_zyx[2], shape_zyx[1], shape_zyx[0])
    dev = torch.device("cuda")
    t = lambda a, dt=torch.float64: None if a is None else torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    qd = t(q)
    phi = torch.empty_like(qd)
    scratch = torch.empty(ek.poisson_cg_scratch_bytes(shape), dtype=torch.uint8, device=dev)
    it, res = ek.poisson_solve_cg(qd, phi, shape, LB, scratch, eps=t(eps),
                                  fixed=t(fixed, torch.uint8) if fixed is not None else None,
                                  phi_fixed=t(phi_fixed), tol=tol, max_iter=max_iter, stream=stream)
    torch.cuda.synchronize()
    return phi.cpu().numpy(), it, res


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("shape", [(16, 24, 32), (12, 12, 12), (9, 10, 11)])
def test_homogeneous_periodic_equals_the_fft_solve(gpu_lib, shape):
    rng = np.random.default_rng(1)
    q = rng.normal(size=shape)
    phi, it, res = solve(gpu_lib, q)
    assert res <= 1e-13
    assert rel(phi, O.poisson(q, LB)) <= 1e-10


def test_dielectric_and_fixed_planes_against_the_oracle(gpu_lib):
    """A smooth random permittivity, fixed potentials on the planes z = 0 and
    z = nz - 1 and inside a sphere (an electrode), random charge."""
    rng = np.random.default_rng(2)
    shape = (20, 24, 16)
    eps = np.exp(0.5 * rng.normal(size=shape))
    z, y, x = np.meshgrid(*(np.arange(n) for n in shape), indexing="ij")
    fixed = (z == 0) | (z == shape[0] - 1) | ((x - 8) ** 2 + (y - 12) ** 2 + (z - 10) ** 2 <= 9)
    pf = np.where(z == 0, 1.3, np.where(z == shape[0] - 1, -0.4, 0.25))
    q = 0.05 * rng.normal(size=shape)
    phi, it, res = solve(gpu_lib, q, eps=eps, fixed=fixed, phi_fixed=pf)
    ref = O.poisson_dielectric(q, LB, eps=eps, fixed=fixed, phi_fixed=pf)
    assert res <= 1e-13
    assert np.array_equal(phi[fixed], pf[fixed])
    assert rel(phi, ref) <= 1e-10


def test_sharp_dielectric_jump_against_the_oracle(gpu_lib):
    """A low-permittivity sphere (eps 2) in water (eps 80) between fixed
    planes, with a charged shell around it: a factor-40 jump."""
    shape = (24, 20, 20)
    z, y, x = np.meshgrid(*(np.arange(n) for n in shape), indexing="ij")
    r = np.sqrt((x - 9.7) ** 2 + (y - 10.2) ** 2 + (z - 11.9) ** 2)
    eps = np.where(r < 5.0, 2.0, 80.0)
    q = np.where((r >= 5.0) & (r < 6.5), -0.01, 0.0)
    fixed = (z == 0) | (z == shape[0] - 1)
    phi, it, res = solve(gpu_lib, q, eps=eps, fixed=fixed)
    ref = O.poisson_dielectric(q, LB, eps=eps, fixed=fixed)
    assert res <= 1e-13
    assert rel(phi, ref) <= 1e-9


def test_two_dielectrics_closed_form(gpu_lib):
    nz, L, zi, V, e1, e2 = 64, 60, 23, 2.0, 3.0, 78.5
    shape = (nz, 8, 8)
    eps = np.where(np.arange(nz)[:, None, None] < zi, e1, e2) * np.ones(shape)
    fixed = np.zeros(shape, dtype=bool)
    fixed[0] = fixed[L] = True
    pf = np.zeros(shape)
    pf[0] = V
    phi, it, res = solve(gpu_lib, np.zeros(shape), eps=eps, fixed=fixed, phi_fixed=pf)
    ez = eps[:, 0, 0]
    ef = 2.0 * ez[:L] * ez[1:L + 1] / (ez[:L] + ez[1:L + 1])
    D = V / np.sum(1.0 / ef)
    exact = np.concatenate([[V], V - D * np.cumsum(1.0 / ef)])
    assert np.max(np.abs(phi[:L + 1] - exact[:, None, None])) <= 1e-11 * V


def test_reproducible_and_errors(gpu_lib):
    ek = gpu_lib
    rng = np.random.default_rng(4)
    shape = (16, 16, 16)
    eps = 1.0 + rng.random(shape)
    q = rng.normal(size=shape)
    import torch
    a, ia, ra = solve(ek, q, eps=eps)
    b, ib, rb = solve(ek, q, eps=eps)
    assert np.array_equal(a, b) and ia == ib and ra == rb
    # on a caller stream the iterations run as captured graphs: the same result
    c, ic, rc = solve(ek, q, eps=eps, stream=torch.cuda.Stream())
    assert np.array_equal(a, c) and ia == ic and ra == rc
    # a cap on the iterations is reported through the residual, not an error
    _, it, res = solve(ek, q, eps=eps, max_iter=10)
    assert it == 10 and res > 1e-13
    bad = eps.copy()
    bad[3, 4, 5] = -1.0
    with pytest.raises(ek.EKError):
        solve(ek, q, eps=bad)


def test_large_homogeneous_box_equals_the_fft_solve(gpu_lib):
    import torch
    ek = gpu_lib
    shape = (64, 64, 64)
    rng = np.random.default_rng(6)
    q = rng.normal(size=shape)
    phi, it, res = solve(ek, q, tol=1e-12)
    qd = torch.as_tensor(q, device="cuda")
    ref = torch.empty_like(qd)
    spec = torch.empty(ek.poisson_scratch_bytes(64, 64, 64), dtype=torch.uint8, device="cuda")
    ek.poisson_solve(qd, ref, (64, 64, 64), LB, spec)
    assert res <= 1e-12
    assert rel(phi, ref.cpu().numpy()) <= 1e-9
