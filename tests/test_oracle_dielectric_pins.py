"""Pins of the oracle's Poisson solve with an inhomogeneous permittivity and
fixed-potential nodes (Sec. III.C, the paragraph after Eq. 16; reading: face
permittivity = harmonic mean of its two nodes).  Each pin is fixed by the
mathematics, not by the oracle: the FFT solve of the homogeneous periodic
problem, closed forms of one-dimensional problems (whose discrete solutions
are exact), and the symmetry of the Green's function."""
import numpy as np
import pytest

from oracle import ek_oracle as O


def test_homogeneous_periodic_equals_the_fft_solve():
    rng = np.random.default_rng(3)
    q = rng.normal(size=(8, 12, 16))
    a = O.poisson_dielectric(q, 0.7)
    b = O.poisson(q, 0.7)
    assert np.max(np.abs(a - b)) <= 1e-10 * np.max(np.abs(b))


def test_uniform_charge_between_fixed_planes_is_a_parabola():
    """eps uniform, Phi = 0 on the planes z = 0 and z = L, charge q0 between:
    the second difference of a quadratic is exact, so the discrete solution is
    Phi(z) = 2 pi l_B q0 z (L - z) / eps."""
    nz, L, q0, eps, lb = 12, 11, 0.03, 2.5, 0.7
    shape = (nz, 4, 4)
    fixed = np.zeros(shape, dtype=bool)
    fixed[0] = fixed[L] = True
    q = np.full(shape, q0)
    phi = O.poisson_dielectric(q, lb, eps=np.full(shape, eps), fixed=fixed)
    z = np.arange(nz, dtype=np.float64)
    exact = 2.0 * np.pi * lb * q0 * z * (L - z) / eps
    assert np.max(np.abs(phi - exact[:, None, None])) <= 1e-12 * exact.max()


def test_two_dielectrics_between_fixed_planes():
    """No charge, Phi = V at z = 0 and 0 at z = L, eps1 below z_i and eps2
    from z_i on: the flux eps_f (Phi_k - Phi_k+1) is the same through every
    face, so Phi_k = V - D sum over the faces below k of 1 / eps_f with
    D = V / sum of all 1 / eps_f (the face at the jump has the harmonic mean)."""
    nz, L, zi, V, e1, e2 = 16, 13, 6, 1.7, 1.0, 40.0
    shape = (nz, 3, 5)
    eps = np.where(np.arange(nz)[:, None, None] < zi, e1, e2) * np.ones(shape)
    fixed = np.zeros(shape, dtype=bool)
    fixed[0] = fixed[L] = True
    pfix = np.zeros(shape)
    pfix[0] = V
    phi = O.poisson_dielectric(np.zeros(shape), 0.7, eps=eps, fixed=fixed, phi_fixed=pfix)
    ez = eps[:, 0, 0]
    ef = 2.0 * ez[:L] * ez[1:L + 1] / (ez[:L] + ez[1:L + 1])
    D = V / np.sum(1.0 / ef)
    exact = np.concatenate([[V], V - D * np.cumsum(1.0 / ef)])
    assert np.max(np.abs(phi[:L + 1, 1, 2] - exact)) <= 1e-12 * V
    # the field jumps by eps2 / eps1 across the interface
    assert np.isclose((phi[zi - 2, 0, 0] - phi[zi - 1, 0, 0]) / (phi[zi + 1, 0, 0] - phi[zi + 2, 0, 0]),
                      e2 / e1, rtol=1e-10)


def test_green_function_is_symmetric():
    """Potential at j of a unit charge at i equals that at i of a unit charge
    at j, for a random permittivity and a random set of fixed nodes (a
    transposed or one-sided face term breaks it)."""
    rng = np.random.default_rng(5)
    shape = (6, 7, 8)
    eps = np.exp(rng.normal(size=shape))
    fixed = rng.random(shape) < 0.1
    i, j = (1, 2, 3), (4, 5, 6)
    fixed[i] = fixed[j] = False
    qi = np.zeros(shape)
    qi[i] = 1.0
    qj = np.zeros(shape)
    qj[j] = 1.0
    a = O.poisson_dielectric(qi, 0.7, eps=eps, fixed=fixed)[j]
    b = O.poisson_dielectric(qj, 0.7, eps=eps, fixed=fixed)[i]
    assert abs(a - b) <= 1e-12 * abs(a)
    assert a > 0.0


def test_fixed_nodes_keep_their_values_and_gauss_law_holds():
    """The fixed nodes hold phi_fixed; around a free region enclosed by fixed
    nodes, the total flux out through the faces into fixed nodes equals 4 pi
    l_B times the enclosed charge."""
    rng = np.random.default_rng(8)
    shape = (10, 10, 10)
    fixed = np.ones(shape, dtype=bool)
    fixed[2:8, 2:8, 2:8] = False
    eps = 1.0 + rng.random(shape)
    pf = rng.normal(size=shape)
    q = rng.normal(size=shape)
    lb = 0.7
    phi = O.poisson_dielectric(q, lb, eps=eps, fixed=fixed, phi_fixed=pf)
    assert np.array_equal(phi[fixed], pf[fixed])
    flux = 0.0
    for axis in range(3):
        for sgn in (1, -1):
            nb = np.roll(phi, -sgn, axis=axis)
            enb = np.roll(eps, -sgn, axis=axis)
            fnb = np.roll(fixed, -sgn, axis=axis)
            ef = 2.0 * eps * enb / (eps + enb)
            flux += np.sum((ef * (phi - nb))[(~fixed) & fnb])
    assert np.isclose(flux, 4.0 * np.pi * lb * q[~fixed].sum(), rtol=1e-10)
