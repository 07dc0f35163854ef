"""Pins of the FP64 oracle against closed forms, invariants and brute force.

None of these compare the oracle with itself: each checks a consequence that
the paper or the mathematics fixes (a decay rate, a moment, a conservation law,
an analytic flow profile, a dense linear solve, a naive restatement).
"""
import math

import numpy as np
import pytest

from oracle import ek_oracle as O
from oracle.ek_oracle import EKOracle


def quiet_box(n, **kw):
    kw.setdefault("bulk", (0.0, 0.0))
    kw.setdefault("flags", O.PV | O.NEUTRALIZE)
    return EKOracle(*n, **kw)


# --------------------------------------------------------------------------
# lattice constants: D3Q19 isotropy (Sec. III.A)
# --------------------------------------------------------------------------
def test_d3q19_moments():
    c = O.CV.astype(float)
    w = O.WT
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose((w[:, None] * c).sum(0), 0.0)
    second = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(second, np.eye(3) / 3.0, atol=1e-15)
    for i in range(19):
        assert (c[O.OPP[i]] == -c[i]).all()
    # 18 links: 6 faces of length 1, 12 edges of length sqrt 2
    assert sorted(np.round(O.CLEN[1:] ** 2).astype(int).tolist()) == [1] * 6 + [2] * 12


# --------------------------------------------------------------------------
# Pin 1: a Fourier mode of the diffusive flux decays by the exact lattice factor
#        and reduces to D k^2 in the continuum limit (Eq. 15, A_0 = 1 + 2 sqrt 2)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kvec", [(1, 0, 0), (1, 2, 0), (2, 1, 3)])
def test_diffusion_fourier_mode(kvec):
    n = (12, 10, 8)
    o = quiet_box(n, valence=(1, -1), D=(0.3, 0.17), bulk=(0.0, 0.0))
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    k = [2 * np.pi * kvec[0] / n[0], 2 * np.pi * kvec[1] / n[1], 2 * np.pi * kvec[2] / n[2]]
    phase = k[0] * x + k[1] * y + k[2] * z
    eps = 1e-3
    for s in range(2):
        o.set_species(s, 0.01 + eps * np.cos(phase))
    o.phi[:] = 0.0
    J = o.link_fluxes()
    drho = -J[:, 1:].sum(axis=1)
    for s, D in enumerate((0.3, 0.17)):
        # closed form: sum over the 18 links of (1 - cos k.c)/|c|, times D/A0
        lam = 0.0
        for cx in (-1, 0, 1):
            for cy in (-1, 0, 1):
                for cz in (-1, 0, 1):
                    L2 = cx * cx + cy * cy + cz * cz
                    if L2 in (1, 2):
                        lam += (1 - math.cos(k[0] * cx + k[1] * cy + k[2] * cz)) / math.sqrt(L2)
        expect = -D / (1 + 2 * math.sqrt(2)) * lam * eps * np.cos(phase)
        assert np.max(np.abs(drho[s] - expect)) < 1e-17 + 1e-12 * eps


def test_diffusion_continuum_limit():
    """For small k the lattice decay rate tends to D |k|^2: the paper's A_0
    recovers the bulk diffusion coefficient."""
    D = 0.3
    for kk in (1e-2, 3e-3):
        lam = 0.0
        for cx in (-1, 0, 1):
            for cy in (-1, 0, 1):
                for cz in (-1, 0, 1):
                    L2 = cx * cx + cy * cy + cz * cz
                    if L2 in (1, 2):
                        lam += (1 - math.cos(kk * cx)) / math.sqrt(L2)
        rate = D / O.A0 * lam
        assert abs(rate / (D * kk * kk) - 1.0) < kk * kk


# --------------------------------------------------------------------------
# Pin 2: the second moment of a point source grows by exactly 2 D per step
#        per axis and the mass is constant (mean-square displacement 6 D t)
# --------------------------------------------------------------------------
def test_point_source_second_moment():
    n = (16, 16, 16)
    o = quiet_box(n, valence=(1, -1), D=(0.3, 0.3))
    rho = np.zeros(o.shape)
    rho[8, 8, 8] = 1.0
    o.set_species(0, rho)
    o.set_species(1, np.zeros(o.shape))
    o.phi[:] = 0.0
    z, y, x = np.meshgrid(np.arange(16), np.arange(16), np.arange(16), indexing="ij")
    for step in range(1, 4):
        J = o.link_fluxes()
        o.rho = o.rho - J[:, 1:].sum(axis=1)
        m = o.rho[0].sum()
        assert abs(m - 1.0) < 1e-14
        for coord in (x, y, z):
            var = ((coord - 8.0) ** 2 * o.rho[0]).sum() / m
            assert abs(var - 2 * 0.3 * step) < 1e-13


# --------------------------------------------------------------------------
# Pin 3: uniform species in a uniform field carry no divergence, and the fluid
#        feels exactly q E (Eqs. 13, 16; the 1/2 and the migration sign)
# --------------------------------------------------------------------------
def test_uniform_drift_force():
    n = (8, 8, 8)
    o = quiet_box(n, valence=(1, -1), D=(0.3, 0.2))
    o.set_species(0, np.full(o.shape, 0.02))
    o.set_species(1, np.full(o.shape, 0.005))
    o.phi[:] = 0.0
    o.E = np.array([0.01, -0.003, 0.002])
    J = o.link_fluxes()
    assert np.max(np.abs(J[:, 1:].sum(axis=1))) < 1e-18
    f = o.coupling_force(J)
    q = 0.02 - 0.005
    for a in range(3):
        assert np.allclose(f[a], q * o.E[a], rtol=1e-13, atol=1e-19)
    # a positive ion moves down the potential: flux along +E is positive
    assert J[0, 1].mean() > 0 and J[1, 1].mean() < 0


def test_migration_sign_equilibrium():
    """A Boltzmann-distributed species in its own potential has (nearly) no
    net flux: (rho - rho') and z rho_bar (Phi - Phi') cancel to second order."""
    n = (32, 4, 4)
    o = quiet_box(n, valence=(1, -1), D=(0.3, 0.3))
    x = np.arange(32)
    phi = 0.05 * np.sin(2 * np.pi * x / 32)
    o.phi = np.broadcast_to(phi[None, None, :], o.shape).copy()
    o.set_species(0, np.broadcast_to(np.exp(-phi)[None, None, :], o.shape))
    o.set_species(1, np.broadcast_to(np.exp(+phi)[None, None, :], o.shape))
    J = o.link_fluxes()
    flux_scale = 0.3 / O.A0 * 0.05 * 2 * np.pi / 32
    assert np.max(np.abs(J[:, 1])) < 1e-2 * flux_scale
    # the opposite sign would double the flux instead
    o.set_species(0, np.broadcast_to(np.exp(+phi)[None, None, :], o.shape))
    J2 = o.link_fluxes()
    assert np.max(np.abs(J2[0, 1])) > 1.5 * flux_scale


# --------------------------------------------------------------------------
# Pin 4: volume-of-fluid advection moves the centre of mass by exactly u
# --------------------------------------------------------------------------
def test_vof_translation():
    n = (16, 16, 16)
    o = quiet_box(n)
    rho = np.zeros(o.shape)
    rho[6:9, 7:10, 5:8] = np.arange(27).reshape(3, 3, 3) + 1.0
    o.set_species(0, rho)
    o.set_species(1, np.zeros(o.shape))
    u = np.array([0.3, -0.45, 0.2])
    uf = np.broadcast_to(u.reshape(3, 1, 1, 1), (3,) + o.shape).copy()
    z, y, x = np.meshgrid(np.arange(16), np.arange(16), np.arange(16), indexing="ij")
    m0 = rho.sum()
    com0 = np.array([(x * rho).sum(), (y * rho).sum(), (z * rho).sum()]) / m0
    for step in range(1, 4):
        o.rho = o.rho + o.advection(uf)
        m = o.rho[0].sum()
        assert abs(m - m0) < 1e-12 * m0
        com = np.array([(x * o.rho[0]).sum(), (y * o.rho[0]).sum(), (z * o.rho[0]).sum()]) / m
        assert np.allclose(com, com0 + step * u, atol=1e-12)
        assert o.rho[0].min() >= 0.0


def test_vof_blocked_by_boundary():
    n = (8, 8, 8)
    o = quiet_box(n)
    mask = np.zeros(o.shape, dtype=bool)
    mask[:, :, 5] = True
    o.set_walls(mask)
    rho = np.zeros(o.shape)
    rho[:, :, 4] = 1.0
    o.set_species(0, rho)
    o.set_species(1, np.zeros(o.shape))
    uf = np.zeros((3,) + o.shape)
    uf[0] = 0.4
    o.rho = o.rho + o.advection(uf)
    assert np.allclose(o.rho[0][:, :, 4], 1.0) and np.all(o.rho[0][:, :, 5] == 0.0)


# --------------------------------------------------------------------------
# Pin 5: Poisson (Eq. 3) -- 7-point residual and a dense pseudo-inverse solve
# --------------------------------------------------------------------------
def _lap7(phi):
    out = -6.0 * phi
    for ax in range(3):
        out = out + np.roll(phi, 1, axis=ax) + np.roll(phi, -1, axis=ax)
    return out


def test_poisson_residual():
    rng = np.random.default_rng(5)
    q = rng.standard_normal((10, 12, 14))
    phi = O.poisson(q, 0.7)
    assert np.max(np.abs(_lap7(phi) + 4 * np.pi * 0.7 * (q - q.mean()))) < 1e-12
    assert abs(phi.mean()) < 1e-14


def test_poisson_dense_solve():
    rng = np.random.default_rng(6)
    shape = (4, 5, 6)
    N = 120
    q = rng.standard_normal(shape)
    # brute force: assemble the periodic 7-point Laplacian as a dense matrix
    A = np.zeros((N, N))
    idx = np.arange(N).reshape(shape)
    for zz in range(4):
        for yy in range(5):
            for xx in range(6):
                r = idx[zz, yy, xx]
                A[r, r] -= 6.0
                for dz, dy, dx in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    A[r, idx[(zz + dz) % 4, (yy + dy) % 5, (xx + dx) % 6]] += 1.0
    rhs = -4 * np.pi * 0.7 * (q - q.mean()).ravel()
    sol = np.linalg.pinv(A, rcond=1e-10) @ rhs
    phi = O.poisson(q, 0.7)
    assert np.max(np.abs(phi.ravel() - sol)) < 1e-11


def test_poisson_plane_wave():
    shape = (8, 8, 16)
    z, y, x = np.meshgrid(np.arange(8), np.arange(8), np.arange(16), indexing="ij")
    k = 2 * np.pi * 3 / 16
    q = np.cos(k * x)
    phi = O.poisson(q, 1.0)
    expect = 4 * np.pi * np.cos(k * x) / (2 - 2 * np.cos(k))
    assert np.max(np.abs(phi - expect)) < 1e-12


# --------------------------------------------------------------------------
# Pin 6: body-force Poiseuille flow between bounce-back walls (Sec. III.A)
# --------------------------------------------------------------------------
def _poiseuille(magic, H=8, steps=1500):
    n = (H + 2, 1, 1)
    o = quiet_box(n, magic=magic)
    mask = np.zeros(o.shape, dtype=bool)
    mask[:, :, 0] = True
    mask[:, :, H + 1] = True
    o.set_walls(mask)
    g = 1e-6
    o.g = np.array([0.0, g, 0.0])
    nu = 1.0 / 6.0
    xs = np.arange(1, H + 1, dtype=float)
    exact = g / (2 * nu) * (xs - 0.5) * (H + 0.5 - xs)
    u0 = np.zeros((3,) + o.shape)
    u0[1, 0, 0, 1:H + 1] = exact
    o.set_velocity(u0)
    o.step(steps)
    return o.u[1, 0, 0, 1:H + 1], exact


def test_poiseuille_trt_magic_exact():
    """TRT with Lambda = 3/16 puts the bounce-back wall exactly half-way."""
    u, exact = _poiseuille(3.0 / 16.0)
    assert np.max(np.abs(u - exact)) < 1e-10 * exact.max()


def test_poiseuille_bgk_slip():
    """BGK at tau = 1 (Lambda = 1/4) has a small, known-sign slip."""
    u, exact = _poiseuille(None)
    err = np.max(np.abs(u - exact)) / exact.max()
    assert 1e-6 < err < 0.05


# --------------------------------------------------------------------------
# momentum: a uniform force adds exactly f per node per step, mass unchanged
# --------------------------------------------------------------------------
def test_uniform_force_momentum():
    o = quiet_box((6, 5, 4))
    o.g = np.array([1e-4, -2e-4, 3e-5])
    m0 = o.density().sum()
    for step in range(1, 4):
        o.step()
        p = o.fluid_momentum()
        assert np.allclose(p, step * o.g * 120, rtol=1e-12, atol=1e-18)
        assert abs(o.density().sum() - m0) < 1e-12


# --------------------------------------------------------------------------
# Pin 8/9: conservation through covering and uncovering; drag sign
# --------------------------------------------------------------------------
def test_species_conserved_through_transitions():
    n = (16, 16, 16)
    o = EKOracle(*n, bulk=(1e-3, 1e-3))
    o.E = np.array([0.01, 0.0, 0.0])
    o.add_particle((7.3, 8.1, 7.7), vel=(0.06, 0.025, 0.0), radius=3.0, charge=-10.0, rho_p=1e9)
    N0 = o.total_species().copy()
    Q0 = o.total_charge()
    x0 = o.particles[0].pos.copy()
    nflip = 0
    for _ in range(60):
        old = o.owner.copy()
        o.step()
        nflip += int((old != o.owner).sum())
        assert np.allclose(o.total_species(), N0, rtol=1e-12, atol=0)
        assert abs(o.total_charge() - Q0) < 1e-12 * np.abs(o.valence * N0).sum()
    assert np.linalg.norm(o.particles[0].pos - x0) > 3.0
    assert nflip > 50
    assert o.rho.min() > -1e-6


def test_vacate_zero_conserves():
    n = (16, 16, 16)
    o = EKOracle(*n, bulk=(1e-3, 1e-3), flags=O.PV | O.NEUTRALIZE | O.VACATE_ZERO)
    o.add_particle((7.3, 8.1, 7.7), vel=(0.07, 0.0, 0.0), radius=3.0, charge=-10.0, rho_p=1e9)
    N0 = o.total_species().copy()
    for _ in range(30):
        o.step()
        assert np.allclose(o.total_species(), N0, rtol=1e-12, atol=0)


def test_momentum_conserved_with_moving_sphere():
    n = (16, 16, 16)
    o = quiet_box(n)
    o.add_particle((7.6, 8.2, 8.4), vel=(0.03, -0.01, 0.005), radius=3.0, charge=0.0, rho_p=2.0)
    p = o.particles[0]

    def total():
        return o.fluid_momentum() + p.mass * p.vel + p.f_trans

    P0 = total()
    nflip = 0
    for _ in range(40):
        old = o.owner.copy()
        o.step()
        nflip += int((old != o.owner).sum())
        assert np.allclose(total(), P0, rtol=0, atol=1e-12 * p.mass * 0.03)
    assert nflip > 0


def test_drag_opposes_motion():
    o = quiet_box((16, 16, 16))
    o.add_particle((8.0, 8.0, 8.0), vel=(0.02, 0.0, 0.0), radius=3.0, charge=0.0,
                   rho_p=1e9)
    for _ in range(15):
        o.step()
    p = o.particles[0]
    assert p.force[0] < 0.0 and abs(p.force[0]) > 10 * abs(p.force[1])


def test_electrophoresis_direction():
    """A negatively charged sphere in +E moves along -x."""
    o = EKOracle(16, 16, 16, bulk=(1e-3, 1e-3))
    o.E = np.array([0.01, 0.0, 0.0])
    o.add_particle((8.3, 7.9, 8.1), radius=3.0, charge=-10.0)
    o.step(10)
    assert o.particles[0].vel[0] < 0.0


# --------------------------------------------------------------------------
# Pin 11: Psi geometry (Sec. III.D.2)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("R,c", [(3.0, (0.0, 0.0, 0.0)), (4.0, (0.31, -0.27, 0.44)), (5.5, (0.5, 0.5, 0.5))])
def test_psi_volume_and_range(R, c):
    lo, hi = O.particle_box(c, R)
    X, Y, Z = np.meshgrid(np.arange(lo[0], hi[0]), np.arange(lo[1], hi[1]),
                          np.arange(lo[2], hi[2]), indexing="ij")
    ps = O.psi_cells(X.astype(float), Y.astype(float), Z.astype(float), np.array(c), R)
    assert ps.min() >= 0.0 and ps.max() <= 1.0
    # depth-4 error bound: the undecided level-4 cubes straddle the surface;
    # their count is at most the surface area over (1/16)^2 times a small factor
    vol = 4.0 / 3.0 * math.pi * R ** 3
    area = 4 * math.pi * R * R
    bound = 0.5 * (1 / 16) ** 3 * 3 * area * 16 ** 2
    assert abs(ps.sum() - vol) < bound
    assert abs(ps.sum() - vol) < 0.01 * vol


def test_psi_cubic_symmetry():
    R = 3.7
    lo, hi = O.particle_box((0.0, 0.0, 0.0), R)
    X, Y, Z = np.meshgrid(np.arange(lo[0], hi[0]), np.arange(lo[1], hi[1]),
                          np.arange(lo[2], hi[2]), indexing="ij")
    ps = O.psi_cells(X.astype(float), Y.astype(float), Z.astype(float), np.zeros(3), R)
    assert np.array_equal(ps, ps.transpose(1, 0, 2))
    assert np.array_equal(ps, ps.transpose(2, 1, 0))
    # the box runs -5..4; the part -4..4 maps onto itself under r -> -r
    assert lo[0] == -5 and hi[0] == 5 and ps[0].max() == 0.0
    sym = ps[1:, 1:, 1:]
    assert np.array_equal(sym, sym[::-1][:, ::-1][:, :, ::-1])


def test_psi_against_fine_sampling():
    """Brute force: Psi of a few surface cells against a 64^3 point sampling of
    the cell, within the depth-4 resolution."""
    R = 4.0
    c = np.array([0.2, 0.1, -0.3])
    cells = [(4, 0, 0), (3, 2, 1), (2, 2, 2), (0, 3, -2), (-3, -2, 1)]
    s = (np.arange(64) + 0.5) / 64 - 0.5
    for cell in cells:
        ps = O.psi_cells(np.array([float(cell[0])]), np.array([float(cell[1])]),
                         np.array([float(cell[2])]), c, R)[0]
        gx, gy, gz = np.meshgrid(cell[0] + s, cell[1] + s, cell[2] + s, indexing="ij")
        frac = (((gx - c[0]) ** 2 + (gy - c[1]) ** 2 + (gz - c[2]) ** 2) < R * R).mean()
        assert abs(ps - frac) < 0.02, (cell, ps, frac)


def _psi_level4(cell, c, R):
    """Psi of one cell from its 4096 level-4 cubes alone, each tested on its own
    (all 8 corners strictly inside: 1; closest point at distance >= R: 0; else
    1/2), FP64, corners as the cube's exact corner coordinates minus the centre,
    squares summed x, y, z."""
    e = np.arange(17) / 16.0 - 0.5
    d = [cell[a] + e - c[a] for a in range(3)]            # plane offsets per axis
    lo = [d[a][:-1] for a in range(3)]
    hi = [d[a][1:] for a in range(3)]
    far = [np.maximum(np.abs(lo[a]), np.abs(hi[a])) for a in range(3)]
    near = [np.where((lo[a] <= 0) & (hi[a] >= 0), 0.0, np.minimum(np.abs(lo[a]), np.abs(hi[a])))
            for a in range(3)]
    R2 = R * R

    def d2(v):
        x, y, z = np.meshgrid(v[0], v[1], v[2], indexing="ij")
        return x * x + y * y + z * z

    inside = d2(far) < R2
    out = d2(near) >= R2
    und = ~inside & ~out
    return (inside.sum() + 0.5 * und.sum()) / 4096.0


@pytest.mark.parametrize("c,R", [((0.31, -0.27, 0.44), 4.0), ((0.5, 0.25, 0.125), 2.0),
                                 ((0.0, 0.0, 0.0), 3.0), ((0.0625, 0.5, -0.1875), 2.5),
                                 ((0.123456789, 0.987654321, 0.5), 5.3)])
def test_psi_octree_equals_level4_cubes(c, R):
    """The octree of Sec. III.D.2 (decided cubes take their whole volume,
    undecided ones are split, to depth 4) gives every cell exactly the value of
    its level-4 cubes classified one by one: a cube decided at a coarser level
    has all its sub-cubes decided alike (a sub-cube's farthest corner is no
    farther per axis, its closest point no nearer, and rounding is monotone).
    Dyadic centres put many corners exactly on the sphere."""
    lo, hi = O.particle_box(c, R)
    cells = [(x, y, z) for x in range(lo[0], hi[0]) for y in range(lo[1], hi[1])
             for z in range(lo[2], hi[2])]
    X = np.array([float(q[0]) for q in cells])
    Y = np.array([float(q[1]) for q in cells])
    Z = np.array([float(q[2]) for q in cells])
    ps = O.psi_cells(X, Y, Z, np.array(c), R)
    surface = 0
    for i, cell in enumerate(cells):
        flat = _psi_level4(cell, c, R)
        assert ps[i] == flat, (cell, ps[i], flat)
        surface += 0.0 < flat < 1.0
    assert surface > 20


def test_boundary_nodes_strictly_inside():
    o = quiet_box((16, 16, 16))
    o.add_particle((8.0, 8.0, 8.0), radius=3.0, charge=0.0)
    inside = np.argwhere(o.owner == 0)
    # nodes at distance exactly 3 (e.g. (11, 8, 8)) are fluid
    assert o.owner[8, 8, 11] == O.FLUID and o.owner[8, 8, 10] == 0
    d2 = ((inside[:, ::-1] - 8.0) ** 2).sum(axis=1)
    assert (d2 < 9.0).all() and len(inside) == int(sum(1 for a in range(-3, 4) for b in range(-3, 4)
                                                        for cc in range(-3, 4) if a * a + b * b + cc * cc < 9))


# --------------------------------------------------------------------------
# Pin 12: brute force -- a naive per-node restatement of S2a, S2b and S3
#         (pull streaming, explicit loops) on a tiny box with a moving sphere
# --------------------------------------------------------------------------
def _naive_step_parts(o):
    nx, ny, nz = o.n
    K = o.K
    fluid = o.owner == O.FLUID
    A0 = 1 + 2 * math.sqrt(2)
    dirs = [tuple(c) for c in O.CV]
    w = O.WT
    J = np.zeros((K, 19) + o.shape)
    fext = np.zeros((3,) + o.shape)
    pv = bool(o.flags & O.PV)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if not fluid[z, y, x]:
                    continue
                for i in range(1, 19):
                    cx, cy, cz = dirs[i]
                    X, Y, Z = (x + cx) % nx, (y + cy) % ny, (z + cz) % nz
                    if not fluid[Z, Y, X]:
                        continue
                    pa = o.psi[z, y, x] if pv else 0.0
                    pb = o.psi[Z, Y, X] if pv else 0.0
                    L = math.sqrt(cx * cx + cy * cy + cz * cz)
                    for k in range(K):
                        a = o.rho[k, z, y, x] / (1 - pa)
                        b = o.rho[k, Z, Y, X] / (1 - pb)
                        dphi = o.phi[z, y, x] - o.phi[Z, Y, X] + o.E[0] * cx + o.E[1] * cy + o.E[2] * cz
                        j = o.D[k] / (A0 * L) * ((a - b) + o.valence[k] * (a + b) / 2 * dphi) * (1 - pa) * (1 - pb)
                        J[k, i, z, y, x] = j
                        fext[0, z, y, x] += 0.5 * j * cx / o.D[k]
                        fext[1, z, y, x] += 0.5 * j * cy / o.D[k]
                        fext[2, z, y, x] += 0.5 * j * cz / o.D[k]
    # collision, per node
    tau_e = 3 * o.nu + 0.5
    lam_e, lam_o = o.lam_e, o.lam_o
    fstar = np.zeros_like(o.f)
    uu = np.zeros((3,) + o.shape)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if not fluid[z, y, x]:
                    continue
                fl = o.f[:, z, y, x]
                F = fext[:, z, y, x] + o.g
                rho = fl.sum()
                j = np.array([sum(fl[i] * dirs[i][a] for i in range(19)) for a in range(3)])
                u = (j + F / 2) / rho
                uu[:, z, y, x] = u
                for i in range(19):
                    c = np.array(dirs[i], dtype=float)
                    ib = [m for m in range(19) if dirs[m] == tuple(-c.astype(int))][0]
                    eq_even = w[i] * rho * (1 + 4.5 * (c @ u) ** 2 - 1.5 * (u @ u))
                    eq_odd = w[i] * 3 * (c @ j)
                    fp = (fl[i] + fl[ib]) / 2
                    fm = (fl[i] - fl[ib]) / 2
                    G = (1 + lam_e / 2) * (np.outer(u, F) + np.outer(F, u))
                    delta = 3 * w[i] * (F @ c + 1.5 * (np.trace(G @ np.outer(c, c)) - np.trace(G) / 3))
                    fstar[i, z, y, x] = fl[i] + lam_e * (fp - eq_even) + lam_o * (fm - eq_odd) + delta
    # pull streaming with bounce-back
    fnew = np.zeros_like(o.f)
    vb, _ = o.boundary_velocity_field()
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                if not fluid[z, y, x]:
                    continue
                for i in range(19):
                    cx, cy, cz = dirs[i]
                    sx, sy, sz = (x - cx) % nx, (y - cy) % ny, (z - cz) % nz
                    ib = [m for m in range(19) if dirs[m] == (-cx, -cy, -cz)][0]
                    if fluid[sz, sy, sx]:
                        fnew[i, z, y, x] = fstar[i, sz, sy, sx]
                    else:
                        # the population ibar left x towards the boundary node and came back as i
                        v = vb[:, sz, sy, sx]
                        fnew[i, z, y, x] = fstar[ib, z, y, x] - 6 * w[ib] * o.rho0 * (-cx * v[0] - cy * v[1] - cz * v[2])
    return J, fext, fnew, uu


def test_brute_force_against_naive_loops():
    o = EKOracle(10, 10, 12, bulk=(2e-3, 1e-3), magic=3.0 / 16.0)
    o.E = np.array([0.01, 0.002, -0.004])
    o.g = np.array([1e-5, 0.0, 2e-5])
    o.add_particle((4.2, 3.9, 5.1), vel=(0.01, -0.02, 0.015), omega=(0.001, 0.002, -0.003),
                   radius=1.7, charge=-3.0)
    rng = np.random.default_rng(3)
    o.set_populations(o.f * (1 + 0.01 * rng.standard_normal(o.f.shape)) * (o.owner == -1))
    for k in range(2):
        o.set_species(k, o.rho[k] * (1 + 0.2 * rng.random(o.shape)))
    o.phi = O.poisson(o.charge_density(), o.bjerrum)
    Jn, fn, fnew_n, un = _naive_step_parts(o)
    J = o.link_fluxes()
    f = o.coupling_force(J)
    fnew, u, Fh, Th = o.lb_step(f)
    assert np.max(np.abs(J - Jn)) < 1e-17
    assert np.max(np.abs(f - fn)) < 1e-15
    assert np.max(np.abs(fnew - fnew_n)) < 1e-14
    assert np.max(np.abs(u - un)) < 1e-15
    # the momentum exchange equals the fluid's momentum loss at the boundary links
    mom_before = np.array([(O.CV[:, a][:, None, None, None] * o.f).sum() for a in range(3)]) + \
        (f + o.g.reshape(3, 1, 1, 1) * (o.owner == -1)).sum(axis=(1, 2, 3))
    mom_after = np.array([(O.CV[:, a][:, None, None, None] * fnew).sum() for a in range(3)])
    assert np.allclose(mom_before - mom_after, Fh[0], atol=1e-13)


# --------------------------------------------------------------------------
# momentum balance with charges: the solute is massless, so the particle's
# solute force is the reaction of the solute's force on the fluid, and the
# total momentum of fluid + particles changes only by E times the total charge
# --------------------------------------------------------------------------
def test_total_momentum_conserved_with_charges():
    o = EKOracle(16, 16, 16, bulk=(1e-3, 1e-3))
    o.E = np.array([0.01, 0.003, -0.002])
    o.add_particle((8.3, 7.9, 8.1), vel=(0.01, 0.0, 0.0), radius=3.0, charge=-15.0)
    p = o.particles[0]

    def total():
        return o.fluid_momentum() + p.mass * p.vel + p.f_trans

    P0 = total()
    for _ in range(40):
        o.step()
        assert np.allclose(total(), P0, rtol=0, atol=1e-12)
    assert abs(p.vel[0] - 0.01) > 1e-3  # the particle did respond to the field


def test_momentum_two_particles_and_remainder():
    """Two spheres: the per-particle split (nearest surface in the widened
    boxes plus the evenly shared remainder) keeps the total exact."""
    o = EKOracle(24, 16, 16, bulk=(1e-3, 1e-3))
    o.E = np.array([0.01, 0.0, 0.0])
    o.add_particle((5.3, 7.9, 8.1), radius=2.5, charge=-10.0)
    o.add_particle((16.7, 8.4, 7.2), radius=2.5, charge=-6.0)

    def total():
        s = o.fluid_momentum()
        for p in o.particles:
            s = s + p.mass * p.vel + p.f_trans
        return s

    P0 = total()
    o.step(20)
    assert np.allclose(total(), P0, rtol=0, atol=1e-12)


def test_neutral_box_with_net_charge_gains_QE():
    """Without neutralisation the box carries charge Q and its momentum grows by
    exactly Q E per step (the uniform background of the k = 0 mode feels no field)."""
    o = EKOracle(16, 16, 16, bulk=(1e-3, 1e-3), flags=O.PV)
    o.E = np.array([0.01, 0.0, 0.0])
    o.add_particle((8.3, 7.9, 8.1), radius=3.0, charge=-15.0)
    p = o.particles[0]
    Q = o.total_charge()

    def total():
        return o.fluid_momentum() + p.mass * p.vel + p.f_trans

    P0 = total()
    o.step(10)
    assert np.allclose(total() - P0, 10 * Q * o.E, rtol=0, atol=1e-12)


# --------------------------------------------------------------------------
# Poisson-Boltzmann slit: counter-ions only between two charged walls
# --------------------------------------------------------------------------
def test_poisson_boltzmann_slit_counterions_only():
    """Equilibrium of the full step (fluxes of Eqs. 13/15, Poisson Eq. 3 with
    4 pi l_B, wall charge, zero flux at the walls) against the closed-form
    solution of the Poisson-Boltzmann equation for counter-ions alone between
    two planes of charge density -sigma (k_B T = e = 1, z = +1):
        rho(z) = rho_m / cos^2(alpha (z - z_c)),  alpha^2 = 2 pi l_B rho_m,
        sigma = (rho_m / alpha) tan(alpha d)     (neutrality),
    with the fluid cells filling [z_c - d, z_c + d].  A wrong migration sign
    pushes the ions to the midplane, a wrong 4 pi l_B or z/2 changes alpha or
    the exponent of the Boltzmann factor; the discretisation error is ~0.2%."""
    nx = ny = 4
    nz = 34                     # walls at z = 0 and 33, fluid cells 1..32: d = 16
    lB, d = 0.7, 16.0
    alpha = 1.0 / 16.0
    rho_m = alpha ** 2 / (2.0 * math.pi * lB)
    sigma = rho_m * math.tan(alpha * d) / alpha
    o = EKOracle(nx, ny, nz, bjerrum=lB, valence=(1,), D=(0.3,), bulk=(0.0,), flags=O.NEUTRALIZE)
    walls = np.zeros((nz, ny, nx), bool)
    walls[0] = walls[nz - 1] = True
    q = np.where(walls, -sigma, 0.0)
    o.set_wall_charge(q)
    o.set_walls(walls)          # fills the counter-ions uniformly (neutral box)
    o.step(1200)
    z = np.arange(1, nz - 1) - 0.5 * (nz - 1)
    expect = rho_m / np.cos(alpha * z) ** 2
    prof = o.rho[0][1:nz - 1]
    assert np.allclose(prof, prof[:, :1, :1], rtol=0, atol=1e-15)  # laterally uniform
    assert np.max(np.abs(prof[:, 0, 0] / expect - 1.0)) < 0.01
    # the walls attract the counter-ions: 3.1x the midplane density next to them
    assert prof[0, 0, 0] / prof[16, 0, 0] > 3.0
