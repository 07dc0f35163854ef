"""Plain FP64 CPU oracle of the moving-boundary lattice electrokinetics step.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module.  The product path (the CUDA
library behind ``include/ek.h``) never calls it and shares no code with it.

The method is Kuron et al., "Moving Charged Particles in Lattice Boltzmann-Based
Electrokinetics" (arXiv 1607.04572).  It is an explicit time-stepping scheme, so
this oracle restates its steps one by one, in the paper's notation, with numpy
arrays and ``np.roll`` for the lattice shifts.  No blocking, no fusion: every
stage of a time step is a separate function below.

Lattice units throughout: grid spacing a = 1, time step tau = 1, k_B T = 1,
elementary charge e = 1 (the paper's energy unit is k_B T, Table I).
Arrays are indexed [z, y, x] (x fastest), i.e. node index x + nx*(y + ny*z).

One time step (the paper never writes the order down; this is the reading used
by both the oracle and the CUDA path):

  S1  charge assembly and periodic FFT Poisson solve              (Sec. III.C, Eq. 3)
  S2a diffusive + migrative link fluxes and fluid coupling force  (Eqs. 13/20, 16)
  S2b TRT/BGK collide with the Guo force term, push stream with
      velocity bounce-back and momentum exchange                  (Eqs. 5, 8, 9, 10, 12)
  S3  species update: flux divergence + volume-of-fluid advection (Eq. 15, Sec. III.C)
  S4  particle forces and symplectic Euler integration            (Sec. III.B)
  S5  re-flag, partial volumes Psi, fluid create/destroy and
      solute expel/refill                                         (Sec. III.B, Eqs. 17-18, III.D.2)

Readings of passages where the paper is silent, garbled or ambiguous are noted
inline as "Reading:".

Parity pins: every public function here is pinned by tests under tests/ against
closed forms, invariants or brute force.  Functions without an independent pin
are marked "parity unpinned" in their docstring (there are none at present).
"""
from __future__ import annotations

import math
import numpy as np

# ---------------------------------------------------------------------------
# D3Q19 velocity set (Sec. III.A): rest, 6 faces, 12 edges, c_{ibar} = -c_i.
# ---------------------------------------------------------------------------
CV = np.array(
    [
        (0, 0, 0),
        (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
        (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
        (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
        (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1),
    ],
    dtype=np.int64,
)  # columns are (cx, cy, cz)
WT = np.array([1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12)
Q = 19
OPP = np.array([int(np.where((CV == -CV[i]).all(axis=1))[0][0]) for i in range(Q)])
CLEN = np.sqrt((CV ** 2).sum(axis=1).astype(np.float64))  # |c_i| in {0, 1, sqrt 2}
A0 = 1.0 + 2.0 * math.sqrt(2.0)  # effective area, Sec. III.C

# the 26 neighbour offsets of the volume-of-fluid advection (Sec. III.C)
OFFS26 = [(sx, sy, sz) for sz in (-1, 0, 1) for sy in (-1, 0, 1) for sx in (-1, 0, 1)
          if (sx, sy, sz) != (0, 0, 0)]

# flags (same meaning as in include/ek.h; restated here, not shared)
PV = 1             # partial-volume flux (Eq. 20) and Psi-smeared particle charge (Eq. 21)
VACATE_ZERO = 2    # vacated cells are left empty instead of refilled by Eq. 17
CHARGE_NORM_VP = 4  # smeared charge divided by the continuous V_p (Eq. 21 literally)
NEUTRALIZE = 8     # add counter-ions of one species so the initial box is neutral

FLUID = -1
WALL = -2


class OracleError(RuntimeError):
    """A condition the paper's scheme cannot handle (overlap, nowhere to expel)."""


def shift_from(a, c):
    """Value at x + c for every node x (periodic): the neighbour along c."""
    return np.roll(a, shift=(-int(c[2]), -int(c[1]), -int(c[0])), axis=(-3, -2, -1))


def shift_to(a, c):
    """Array b with b[x + c] = a[x] (periodic): a pushed along c."""
    return np.roll(a, shift=(int(c[2]), int(c[1]), int(c[0])), axis=(-3, -2, -1))


# ---------------------------------------------------------------------------
# LB building blocks (Sec. III.A)
# ---------------------------------------------------------------------------
def feq(rho, u):
    """Second-order D3Q19 equilibrium f_i^eq(rho, u), i = 0..18 (Sec. III.A).

    rho: array; u: (3, ...) array.  Returns (19, ...).
    """
    usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
    out = np.empty((Q,) + np.shape(rho))
    for i in range(Q):
        cu = CV[i, 0] * u[0] + CV[i, 1] * u[1] + CV[i, 2] * u[2]
        out[i] = WT[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq)
    return out


def relaxation_rates(nu, magic):
    """TRT eigenvalues (lambda_e, lambda_o) of Sec. III.A.

    lambda_e follows from the kinematic viscosity: nu = (tau_e - 1/2)/3,
    lambda_e = -1/tau_e.  Reading: the paper's "lambda_o = 3/16" is Ginzburg's
    magic product Lambda = (tau_e - 1/2)(tau_o - 1/2); magic=None gives BGK
    (lambda_o = lambda_e).
    """
    tau_e = 3.0 * nu + 0.5
    if magic is None:
        tau_o = tau_e
    else:
        tau_o = 0.5 + magic / (tau_e - 0.5)
    return -1.0 / tau_e, -1.0 / tau_o


def collide(f, force, lam_e, lam_o):
    """TRT collision with the Guo/Schiller force term, Eqs. (8)-(9).

    f: (19, ...) pre-collision populations; force: (3, ...) force density.
    Reading (Schiller's MRT form of Guo's term, which the paper cites): the
    collision conserves momentum, so the odd equilibrium is built from the
    unshifted momentum j = sum_i f_i c_i, while the even equilibrium, G and the
    fluid velocity use u = (j + f/2)/rho.  The paper's 1/rho prefactor of
    Delta_i is read as 1/rho_0 = 1.
      Delta_i = w_i [3 c_i.f + 9/2 G:c_i c_i - 3/2 Tr G],
      G = (1 + lambda_e/2)(u f + f u).
    Returns (post-collision populations, density, velocity u).
    """
    rho = f.sum(axis=0)
    j = np.stack([np.tensordot(CV[:, a].astype(np.float64), f, axes=(0, 0)) for a in range(3)])
    u = (j + 0.5 * force) / rho
    usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
    g = 1.0 + 0.5 * lam_e
    uf = u[0] * force[0] + u[1] * force[1] + u[2] * force[2]
    fplus = np.empty_like(f)
    fminus = np.empty_like(f)
    eqp = np.empty_like(f)
    eqm = np.empty_like(f)
    for i in range(Q):
        ib = OPP[i]
        fplus[i] = 0.5 * (f[i] + f[ib])
        fminus[i] = 0.5 * (f[i] - f[ib])
        cu = CV[i, 0] * u[0] + CV[i, 1] * u[1] + CV[i, 2] * u[2]
        cj = CV[i, 0] * j[0] + CV[i, 1] * j[1] + CV[i, 2] * j[2]
        eqp[i] = WT[i] * rho * (1.0 + 4.5 * cu * cu - 1.5 * usq)
        eqm[i] = WT[i] * 3.0 * cj
    out = np.empty_like(f)
    for i in range(Q):
        cf = CV[i, 0] * force[0] + CV[i, 1] * force[1] + CV[i, 2] * force[2]
        cu = CV[i, 0] * u[0] + CV[i, 1] * u[1] + CV[i, 2] * u[2]
        # G:c c = 2 g (c.u)(c.f);  Tr G = 2 g (u.f)
        delta = WT[i] * (3.0 * cf + 4.5 * (2.0 * g * cu * cf) - 1.5 * (2.0 * g * uf))
        out[i] = f[i] + lam_e * (fplus[i] - eqp[i]) + lam_o * (fminus[i] - eqm[i]) + delta
    return out, rho, u


# ---------------------------------------------------------------------------
# Electrostatics (Sec. III.C, Eq. 3)
# ---------------------------------------------------------------------------
def laplacian_eigenvalues(shape):
    """lambda(k) = sum_a (2 - 2 cos k_a) of the 7-point Laplacian, periodic box."""
    nz, ny, nx = shape
    kx = 2.0 - 2.0 * np.cos(2.0 * np.pi * np.arange(nx) / nx)
    ky = 2.0 - 2.0 * np.cos(2.0 * np.pi * np.arange(ny) / ny)
    kz = 2.0 - 2.0 * np.cos(2.0 * np.pi * np.arange(nz) / nz)
    return kz[:, None, None] + ky[None, :, None] + kx[None, None, :]


def poisson(q, bjerrum):
    """Solve the 7-point discrete Poisson equation, Eq. (3), in a periodic box.

    lap Phi = -4 pi l_B (q - mean q)  (k_B T = e = 1).  The k = 0 mode is dropped:
    a uniform neutralising background.  numpy's FFT is the library primitive.
    """
    lam = laplacian_eigenvalues(q.shape)
    qh = np.fft.fftn(q)
    lam[0, 0, 0] = 1.0
    ph = 4.0 * np.pi * bjerrum * qh / lam
    ph[0, 0, 0] = 0.0
    return np.fft.ifftn(ph).real


def poisson_dielectric(q, bjerrum, eps=None, fixed=None, phi_fixed=None):
    """Eq. (3) with an inhomogeneous permittivity and fixed-potential nodes,
    the problem the paper leaves to iterative solvers (Sec. III.C, the
    paragraph after Eq. 16): div(eps grad Phi) = -4 pi l_B q, eps the
    permittivity relative to the solvent's (whose Bjerrum length is l_B).

    Reading: the 7-point discretisation of the periodic solve with face
    permittivities, the harmonic mean 2 eps_i eps_j / (eps_i + eps_j) of the
    two nodes of a face (it keeps the flux eps grad Phi continuous across a
    jump).  A free node i satisfies sum_f eps_f (Phi_i - Phi_j) = 4 pi l_B q_i
    over its six faces; a node with fixed[i] holds Phi = phi_fixed[i]
    (Dirichlet).  Without fixed nodes the charge's mean is removed and Phi has
    mean 0, as in ``poisson``.  Arrays [z, y, x]; eps, fixed, phi_fixed may be
    None (eps = 1, no fixed node).  scipy's sparse direct solver is the
    library primitive.
    """
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    shape = q.shape
    n = q.size
    e = np.ones(shape) if eps is None else np.asarray(eps, dtype=np.float64)
    fx = np.zeros(shape, dtype=bool) if fixed is None else np.asarray(fixed, dtype=bool)
    pf = np.zeros(shape) if phi_fixed is None else np.asarray(phi_fixed, dtype=np.float64)
    idx = np.arange(n).reshape(shape)
    rows, cols, vals = [], [], []
    diag = np.zeros(n)
    for axis in range(3):
        j = np.roll(idx, -1, axis=axis)            # the node across the face on the + side
        ej = np.roll(e, -1, axis=axis)
        ef = (2.0 * e * ej / (e + ej)).ravel()     # face permittivity
        i_, j_ = idx.ravel(), j.ravel()
        diag[i_] += ef
        diag[j_] += ef
        rows += [i_, j_]
        cols += [j_, i_]
        vals += [-ef, -ef]
    A = sp.csr_matrix((np.concatenate(vals + [diag]),
                       (np.concatenate(rows + [np.arange(n)]), np.concatenate(cols + [np.arange(n)]))),
                      shape=(n, n))
    b = 4.0 * np.pi * bjerrum * q.ravel().astype(np.float64)
    free = ~fx.ravel()
    phi = np.where(fx.ravel(), pf.ravel(), 0.0)
    if not fx.any():
        # singular (constants): remove the mean charge, hold node 0 at 0,
        # then shift to mean 0
        b = b - b.mean()
        keep = np.arange(1, n)
        sol = spl.spsolve(A[keep][:, keep].tocsc(), b[keep])
        phi = np.concatenate([[0.0], sol])
        return (phi - phi.mean()).reshape(shape)
    Aff = A[free][:, free].tocsc()
    rhs = b[free] - A[free][:, ~free] @ phi[~free]
    phi[free] = spl.spsolve(Aff, rhs)
    return phi.reshape(shape)


# ---------------------------------------------------------------------------
# Partial volumes Psi by octree subdivision (Sec. III.D.2)
# ---------------------------------------------------------------------------
def _cube_inside(cx, cy, cz, h, r, R2):
    """All 8 corners strictly inside the sphere."""
    ok = np.ones(cx.shape, dtype=bool)
    for sx in (-1.0, 1.0):
        for sy in (-1.0, 1.0):
            for sz in (-1.0, 1.0):
                dx = (cx + sx * h) - r[0]
                dy = (cy + sy * h) - r[1]
                dz = (cz + sz * h) - r[2]
                ok &= (dx * dx + dy * dy + dz * dz) < R2
    return ok


def _cube_outside(cx, cy, cz, h, r, R2):
    """The cube's closest point to the centre is at distance >= R."""
    dx = np.clip(r[0], cx - h, cx + h) - r[0]
    dy = np.clip(r[1], cy - h, cy + h) - r[1]
    dz = np.clip(r[2], cz - h, cz + h) - r[2]
    return (dx * dx + dy * dy + dz * dz) >= R2


PSI_DEPTH = 4
FORCE_MARGIN = 4  # cells added to ceil(R) around a particle's box for its solute force


def psi_cells(X, Y, Z, r, R):
    """Volume fraction of each unit cell (centres X, Y, Z) inside a sphere.

    Sec. III.D.2: split the cell into 8 sub-cells, classify each as completely
    inside or completely outside; split the undecided ones again, to depth 4.
    Reading: level 0 is the cell itself, level 4 cubes have edge 1/16; a cube
    still undecided at level 4 counts half its volume.  "Completely inside":
    all 8 corners strictly inside; "completely outside": closest point of the
    cube at distance >= R.  All contributions are dyadic fractions, so the sum
    is exact in any order.
    """
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    Z = np.asarray(Z, dtype=np.float64)
    R2 = R * R
    out = np.zeros(X.shape)
    parent = np.arange(X.size)
    cx, cy, cz = X.ravel().copy(), Y.ravel().copy(), Z.ravel().copy()
    h = 0.5
    vol = 1.0
    flat = out.ravel()
    for depth in range(PSI_DEPTH + 1):
        ins = _cube_inside(cx, cy, cz, h, r, R2)
        outs = _cube_outside(cx, cy, cz, h, r, R2) & ~ins
        np.add.at(flat, parent[ins], vol)
        und = ~ins & ~outs
        if depth == PSI_DEPTH:
            np.add.at(flat, parent[und], 0.5 * vol)
            break
        cx, cy, cz, parent = cx[und], cy[und], cz[und], parent[und]
        h2 = 0.5 * h
        kids = [(sx, sy, sz) for sz in (-1.0, 1.0) for sy in (-1.0, 1.0) for sx in (-1.0, 1.0)]
        cx = np.concatenate([cx + k[0] * h2 for k in kids])
        cy = np.concatenate([cy + k[1] * h2 for k in kids])
        cz = np.concatenate([cz + k[2] * h2 for k in kids])
        parent = np.concatenate([parent for _ in kids])
        h = h2
        vol = vol / 8.0
    return flat.reshape(X.shape)


def particle_box(pos, radius):
    """Unwrapped lattice coordinates of the cells that can touch a sphere.

    Per axis: floor(r - R) - 1 .. floor(r + R) + 1.  Both the boundary-node
    test and Psi use coordinates X in this range, so x - r is never wrapped.
    """
    lo = [int(math.floor(pos[a] - radius)) - 1 for a in range(3)]
    hi = [int(math.floor(pos[a] + radius)) + 2 for a in range(3)]
    return lo, hi


# ---------------------------------------------------------------------------
# The oracle system
# ---------------------------------------------------------------------------
class Particle:
    def __init__(self, pos, vel, omega, radius, charge, rho_p, fixed):
        self.pos = np.array(pos, dtype=np.float64)
        self.vel = np.array(vel, dtype=np.float64)
        self.omega = np.array(omega, dtype=np.float64)
        self.radius = float(radius)
        self.charge = float(charge)
        self.rho_p = float(rho_p)
        self.fixed = bool(fixed)
        self.mass = self.rho_p * 4.0 / 3.0 * math.pi * self.radius ** 3
        self.inertia = 0.4 * self.mass * self.radius ** 2
        self.force = np.zeros(3)
        self.torque = np.zeros(3)
        self.f_trans = np.zeros(3)  # create/destroy momentum, applied at the next S4


class EKOracle:
    """FP64 oracle of the full time step (S1-S5) on a periodic nx*ny*nz box."""

    def __init__(self, nx, ny, nz, nu=1.0 / 6.0, rho0=1.0, bjerrum=0.7,
                 valence=(1, -1), D=(0.3, 0.3), bulk=(1e-3, 1e-3),
                 flags=PV | NEUTRALIZE, magic=None):
        self.shape = (nz, ny, nx)
        self.n = np.array([nx, ny, nz])
        self.nu, self.rho0, self.bjerrum = float(nu), float(rho0), float(bjerrum)
        self.valence = np.array(valence, dtype=np.float64)
        self.D = np.array(D, dtype=np.float64)
        self.bulk = np.array(bulk, dtype=np.float64)
        self.K = len(valence)
        self.flags = int(flags)
        self.magic = magic
        self.lam_e, self.lam_o = relaxation_rates(self.nu, magic)
        self.E = np.zeros(3)
        self.g = np.zeros(3)
        self.particles: list[Particle] = []
        self.wall = np.zeros(self.shape, dtype=bool)
        self.qwall = np.zeros(self.shape)
        self.owner = np.full(self.shape, FLUID, dtype=np.int64)
        self.psi = np.zeros(self.shape)
        self.psi_p: list[tuple] = []  # per particle: (lo, hi, psi box array)
        self.phi = np.zeros(self.shape)
        self.u = np.zeros((3,) + self.shape)
        self.f = feq(np.full(self.shape, self.rho0), np.zeros((3,) + self.shape))
        self.rho = np.empty((self.K,) + self.shape)
        self.steps_done = 0
        self._reflag_setup()
        self._fill()

    # ----- set-up ---------------------------------------------------------
    def add_particle(self, pos, vel=(0, 0, 0), radius=4.0, charge=0.0, rho_p=2.0,
                     fixed=False, omega=(0, 0, 0)):
        """Add a sphere.  Re-flags and refills: species back to the initial fill
        (bulk on fluid nodes, plus neutralising counter-ions), populations to
        rest equilibrium on fluid nodes, Poisson re-solved on the next step."""
        n = self.n
        if 2.0 * radius + 6.0 > n.min():
            # the union of a particle's old and new boxes must not wrap onto itself
            raise OracleError("particle does not fit the box (2R + 6 > box edge)")
        p = Particle(np.mod(pos, n), vel, omega, radius, charge, rho_p, fixed)
        self.particles.append(p)
        self._reflag_setup()
        self._fill()
        return len(self.particles) - 1

    def set_walls(self, mask):
        """Static no-slip, zero-flux boundary cells (Sec. III.C, last paragraph)."""
        self.wall = np.asarray(mask, dtype=bool).reshape(self.shape).copy()
        self._reflag_setup()
        self._fill()

    def set_wall_charge(self, q):
        self.qwall = np.asarray(q, dtype=np.float64).reshape(self.shape).copy()

    def set_species(self, k, values):
        self.rho[k] = np.asarray(values, dtype=np.float64).reshape(self.shape)

    def set_populations(self, f):
        self.f = np.asarray(f, dtype=np.float64).reshape((Q,) + self.shape).copy()

    def set_velocity(self, u):
        """Populations set to equilibrium at the current density and velocity u."""
        rho = self.f.sum(axis=0)
        self.f = feq(rho, np.asarray(u, dtype=np.float64).reshape((3,) + self.shape))

    def _classify(self):
        """Owner of every node and Psi from the current particle positions.

        A node is a boundary node of particle p when its centre is strictly
        inside the sphere (Fig. 2 caption).  Psi(r) = min(1, sum_p Psi_p(r)).
        """
        owner = np.where(self.wall, WALL, FLUID).astype(np.int64)
        psi = np.zeros(self.shape)
        boxes = []
        nx, ny, nz = self.n
        for pid, p in enumerate(self.particles):
            lo, hi = particle_box(p.pos, p.radius)
            X, Y, Z = np.meshgrid(np.arange(lo[0], hi[0]), np.arange(lo[1], hi[1]),
                                  np.arange(lo[2], hi[2]), indexing="ij")
            X = X.transpose(2, 1, 0).astype(np.float64)
            Y = Y.transpose(2, 1, 0).astype(np.float64)
            Z = Z.transpose(2, 1, 0).astype(np.float64)
            dx, dy, dz = X - p.pos[0], Y - p.pos[1], Z - p.pos[2]
            inside = (dx * dx + dy * dy + dz * dz) < p.radius * p.radius
            ps = psi_cells(X, Y, Z, p.pos, p.radius)
            iz = np.mod(np.arange(lo[2], hi[2]), nz)
            iy = np.mod(np.arange(lo[1], hi[1]), ny)
            ix = np.mod(np.arange(lo[0], hi[0]), nx)
            sub = np.ix_(iz, iy, ix)
            o = owner[sub]
            if np.any(inside & (o != FLUID)):
                raise OracleError("overlap: node claimed twice")
            o = np.where(inside, pid, o)
            owner[sub] = o
            psi[sub] += ps
            boxes.append((lo, hi, ps, inside))
        psi = np.minimum(psi, 1.0)
        return owner, psi, boxes

    def _reflag_setup(self):
        self.owner, self.psi, self.psi_p = self._classify()

    def _fill(self):
        """Initial fill (reading of 'bulk density'): bulk on fluid nodes, zero in
        boundary nodes; with NEUTRALIZE the first species whose valence has the
        opposite sign of the box's net charge gets a uniform addition that
        makes the box neutral.  Populations: rest equilibrium at rho_0."""
        fluid = self.owner == FLUID
        nf = int(fluid.sum())
        for k in range(self.K):
            self.rho[k] = np.where(fluid, self.bulk[k], 0.0)
        if self.flags & NEUTRALIZE and nf > 0:
            net = sum(p.charge for p in self.particles) + float(self.qwall.sum()) \
                + float(np.dot(self.valence, self.bulk)) * nf
            if net != 0.0:
                cand = [k for k in range(self.K) if self.valence[k] * net < 0]
                if not cand:
                    raise OracleError("no species can neutralise the box")
                s = cand[0]
                self.rho[s] = np.where(fluid, self.rho[s] - net / (self.valence[s] * nf), 0.0)
        self.f = np.where(fluid[None], feq(np.full(self.shape, self.rho0),
                                           np.zeros((3,) + self.shape)), 0.0)

    # ----- S1: charge and Poisson ------------------------------------------
    def particle_charge(self, pid):
        """Charge of particle pid on each node of its box (Eq. 21 with PV; else
        spread evenly over its boundary nodes).  Reading (PV): divided by
        sum Psi_p so the total is exactly Z; CHARGE_NORM_VP divides by V_p."""
        p = self.particles[pid]
        lo, hi, ps, inside = self.psi_p[pid]
        if self.flags & PV:
            if self.flags & CHARGE_NORM_VP:
                return p.charge * ps / (4.0 / 3.0 * math.pi * p.radius ** 3)
            return p.charge * ps / ps.sum()
        nb = int(inside.sum())
        return np.where(inside, p.charge / max(nb, 1), 0.0)

    def _scatter_box(self, pid, vals, out):
        lo, hi, _, _ = self.psi_p[pid]
        nx, ny, nz = self.n
        sub = np.ix_(np.mod(np.arange(lo[2], hi[2]), nz), np.mod(np.arange(lo[1], hi[1]), ny),
                     np.mod(np.arange(lo[0], hi[0]), nx))
        out[sub] += vals

    def charge_density(self):
        """q(r) = sum_k z_k rho_k + particle charge + static boundary charge."""
        q = np.tensordot(self.valence, self.rho, axes=(0, 0)) + self.qwall
        for pid in range(len(self.particles)):
            self._scatter_box(pid, self.particle_charge(pid), q)
        return q

    # ----- S2a: link fluxes and coupling force -------------------------------
    def link_fluxes(self):
        """Diffusive + migrative flux J_ki(r -> r + c_i) on the 18 D3Q19 links.

        Eqs. (13)/(20).  Readings: (i) every link is divided by its length |c_i|
        and by A_0, and the continuity update is rho' = rho - sum_i J_i; then the
        diffusion coefficient is exactly D (the garbled A_0 placement of Eq. 15);
        (ii) the migration term has the sign of the continuum flux -D z rho grad
        Phi and the same 1/(A_0 |c_i|) normalisation as the diffusion term, so
        the Boltzmann distribution carries no flux; (iii) the external field
        enters as +E.c_i in the potential difference.  With PV the densities are
        rho/(1 - Psi) and the flux is scaled by (1 - Psi)(1 - Psi').  Links with a
        boundary node at either end carry no flux.
        Returns J with shape (K, 19, ...) (index 0 unused).
        """
        fluid = self.owner == FLUID
        pv = bool(self.flags & PV)
        one_m = (1.0 - self.psi) if pv else np.ones(self.shape)
        J = np.zeros((self.K, Q) + self.shape)
        # boundary nodes may have Psi = 1; their links are masked out below
        one_m = np.where(fluid, one_m, 1.0)
        for i in range(1, Q):
            c = CV[i]
            link = fluid & shift_from(fluid, c)
            scale = one_m * shift_from(one_m, c)
            dphi = (self.phi - shift_from(self.phi, c)) + float(np.dot(self.E, c))
            for k in range(self.K):
                a = self.rho[k] / one_m
                b = shift_from(self.rho[k], c) / shift_from(one_m, c)
                br = (a - b) + self.valence[k] * (0.5 * (a + b)) * dphi
                J[k, i] = np.where(link, self.D[k] / (A0 * CLEN[i]) * br * scale, 0.0)
        return J

    def coupling_force(self, J):
        """f_ext = k_B T sum_k sum_i J_ki c_i / D_k (Eq. 16).  Reading: each
        link is seen from both its ends, so the sum carries 1/2 (this makes a
        uniform charge density q in a field E feel exactly q E)."""
        fx = np.zeros((3,) + self.shape)
        for k in range(self.K):
            for i in range(1, Q):
                for a in range(3):
                    if CV[i, a] != 0:
                        fx[a] += 0.5 * CV[i, a] * J[k, i] / self.D[k]
        return fx

    # ----- S2b: LB with moving bounce-back ------------------------------------
    def boundary_velocity_field(self):
        """v_b = v + omega x (r_b - r) on every particle boundary node (Eq. 10),
        zero on walls; also the arm r_b - r used for torques."""
        vb = np.zeros((3,) + self.shape)
        arm = np.zeros((3,) + self.shape)
        nx, ny, nz = self.n
        for pid, p in enumerate(self.particles):
            lo, hi, ps, inside = self.psi_p[pid]
            X, Y, Z = np.meshgrid(np.arange(lo[0], hi[0]), np.arange(lo[1], hi[1]),
                                  np.arange(lo[2], hi[2]), indexing="ij")
            d = [X.transpose(2, 1, 0) - p.pos[0], Y.transpose(2, 1, 0) - p.pos[1],
                 Z.transpose(2, 1, 0) - p.pos[2]]
            w = p.omega
            v = [p.vel[0] + (w[1] * d[2] - w[2] * d[1]),
                 p.vel[1] + (w[2] * d[0] - w[0] * d[2]),
                 p.vel[2] + (w[0] * d[1] - w[1] * d[0])]
            sub = np.ix_(np.mod(np.arange(lo[2], hi[2]), nz), np.mod(np.arange(lo[1], hi[1]), ny),
                         np.mod(np.arange(lo[0], hi[0]), nx))
            for a in range(3):
                blk = vb[a][sub]
                vb[a][sub] = np.where(inside, v[a], blk)
                blk = arm[a][sub]
                arm[a][sub] = np.where(inside, d[a], blk)
        return vb, arm

    def lb_step(self, fext):
        """Collide (Eq. 8, 9) and push-stream with velocity bounce-back (Eq. 12).

        Fluid node x, link i: if x + c_i is fluid, f_i(x + c_i) = f*_i(x); if it is
        a boundary node, f_ibar(x) = f*_i(x) - 6 w_i rho_0 c_i.v_b(x + c_i).
        Reading: the bounce-back's rho factor is rho_0 (Ladd), and v_b is taken
        at the boundary node.  The particle receives the momentum
        c_i (f*_i(x) + f_ibar(x)) per link (Eq. 11), the torque (r_b - r) x that.
        Returns new populations, velocity u, and per-particle force and torque.
        """
        fluid = self.owner == FLUID
        force = fext + self.g.reshape(3, 1, 1, 1)
        # boundary nodes hold no fluid; give them rest populations so the
        # (discarded) collision there stays finite
        rest = feq(np.full(self.shape, self.rho0), np.zeros((3,) + self.shape))
        fs, rho, u = collide(np.where(fluid[None], self.f, rest), force, self.lam_e, self.lam_o)
        vb, arm = self.boundary_velocity_field()
        fnew = np.zeros_like(self.f)
        P = len(self.particles)
        Fh = np.zeros((P, 3))
        Th = np.zeros((P, 3))
        fnew[0] = np.where(fluid, fs[0], 0.0)
        for i in range(1, Q):
            c = CV[i]
            ib = OPP[i]
            nb_owner = shift_from(self.owner, c)
            push = fluid & (nb_owner == FLUID)
            bounce = fluid & (nb_owner != FLUID)
            fnew[i] += shift_to(np.where(push, fs[i], 0.0), c)
            vbn = shift_from(vb, c)
            cvb = c[0] * vbn[0] + c[1] * vbn[1] + c[2] * vbn[2]
            refl = fs[i] - 6.0 * WT[i] * self.rho0 * cvb
            fnew[ib] += np.where(bounce, refl, 0.0)
            if P:
                armn = shift_from(arm, c)
                mom = fs[i] + refl  # scalar per link; times c_i below
                for pid in range(P):
                    m = bounce & (nb_owner == pid)
                    if not m.any():
                        continue
                    dp = np.array([c[0] * mom[m], c[1] * mom[m], c[2] * mom[m]])
                    Fh[pid] += dp.sum(axis=1)
                    ax, ay, az = armn[0][m], armn[1][m], armn[2][m]
                    Th[pid] += np.array([(ay * dp[2] - az * dp[1]).sum(),
                                         (az * dp[0] - ax * dp[2]).sum(),
                                         (ax * dp[1] - ay * dp[0]).sum()])
        u = np.where(fluid[None], u, 0.0)
        return fnew, u, Fh, Th

    # ----- S3: species update ---------------------------------------------------
    def advection(self, u):
        """Volume-of-fluid advection (Sec. III.C): the cell at r is displaced by
        u(r) and intersected with its 26 neighbours.  The fraction moved to
        offset s is prod_a w_a(s_a): w = 1 - |u_a| for s_a = 0, |u_a| for
        s_a = sign(u_a), 0 otherwise.  Reading: only fluid cells move solute,
        and a share aimed at a boundary node stays in its source cell.
        Returns d rho per species."""
        fluid = self.owner == FLUID
        au = np.abs(u)
        out = np.zeros_like(self.rho)
        for s in OFFS26:
            frac = np.ones(self.shape)
            for a in range(3):
                if s[a] == 0:
                    frac = frac * (1.0 - au[a])
                else:
                    frac = frac * np.where(np.sign(u[a]) == s[a], au[a], 0.0)
            moves = fluid & shift_from(fluid, s)
            for k in range(self.K):
                amt = np.where(moves, self.rho[k] * frac, 0.0)
                out[k] -= amt
                out[k] += shift_to(amt, s)
        return out

    # ----- S4: particles ---------------------------------------------------------
    def charge_field_force(self, pid):
        """Force and torque of the external field E on the particle's own
        charge distribution q_p(r) (Eq. 21 / the simple scheme's spread)."""
        p = self.particles[pid]
        lo, hi, ps, inside = self.psi_p[pid]
        qv = self.particle_charge(pid)
        Z, Y, X = np.meshgrid(np.arange(lo[2], hi[2]), np.arange(lo[1], hi[1]),
                              np.arange(lo[0], hi[0]), indexing="ij")
        d = [X - p.pos[0], Y - p.pos[1], Z - p.pos[2]]
        F = qv.sum() * self.E
        T = np.array([((d[1] * self.E[2] - d[2] * self.E[1]) * qv).sum(),
                      ((d[2] * self.E[0] - d[0] * self.E[2]) * qv).sum(),
                      ((d[0] * self.E[1] - d[1] * self.E[0]) * qv).sum()])
        return F, T

    def min_image(self, coord, r, n):
        """x - r wrapped to the nearest periodic image (|d| <= n/2)."""
        d = coord - r
        d = np.where(d > 0.5 * n, d - n, d)
        d = np.where(d < -0.5 * n, d + n, d)
        return d

    def surface_distance(self, pid, X, Y, Z):
        """Distance from node centres (X, Y, Z) (integer lattice coordinates,
        0 <= X < nx ...) to the surface of particle pid, in FP64:
        s = sqrt(dx*dx + dy*dy + dz*dz) - R with d the minimum-image offset
        node - centre, the squares summed left to right.  Also returns d."""
        p = self.particles[pid]
        nx, ny, nz = self.n
        dx = self.min_image(np.asarray(X, dtype=np.float64), p.pos[0], nx)
        dy = self.min_image(np.asarray(Y, dtype=np.float64), p.pos[1], ny)
        dz = self.min_image(np.asarray(Z, dtype=np.float64), p.pos[2], nz)
        return np.sqrt(dx * dx + dy * dy + dz * dz) - p.radius, dx, dy, dz

    def nearest_particle(self):
        """Nearest-surface partition of the widened boxes (the regions V_p of
        solute_forces).  Every node of particle p's box widened by ceil(R) + 4
        cells is a candidate of p; a node belongs to the candidate with the
        smallest FP64 surface distance, equal distances to the lower index.
        Returns (nearest, regions): nearest[n] is the particle of flat node n
        (-1 outside every widened box); regions[p] = (flat nodes of p's widened
        box, each once, and their minimum-image offsets dx, dy, dz)."""
        nx, ny, nz = self.n
        best = np.full(self.shape, np.inf).ravel()
        nearest = np.full(self.shape, -1, dtype=np.int64).ravel()
        regions = []
        # particles visited in index order; a node changes hands only to a
        # strictly smaller distance
        for pid, p in enumerate(self.particles):
            lo, hi = particle_box(p.pos, p.radius)
            m = int(math.ceil(p.radius)) + FORCE_MARGIN
            iz = np.mod(np.arange(lo[2] - m, hi[2] + m), nz)
            iy = np.mod(np.arange(lo[1] - m, hi[1] + m), ny)
            ix = np.mod(np.arange(lo[0] - m, hi[0] + m), nx)
            Zc, Yc, Xc = np.meshgrid(iz, iy, ix, indexing="ij")
            flat = (Xc + nx * (Yc + ny * Zc)).ravel()
            # a widened box wider than the lattice lists a node more than once
            flat, first = np.unique(flat, return_index=True)
            s, dx, dy, dz = self.surface_distance(pid, Xc.ravel()[first], Yc.ravel()[first],
                                                  Zc.ravel()[first])
            closer = s < best[flat]
            best[flat[closer]] = s[closer]
            nearest[flat[closer]] = pid
            regions.append((flat, dx, dy, dz))
        return nearest, regions

    def solute_forces(self, fext):
        """Force and torque of the solute on every particle.

        Reading: the paper adds "a force from electrostatics" to the drag
        without a formula (Sec. III.C).  The solute is massless, so the force it
        exerts on the particles (Coulomb force on the particle charge and the
        ions' contact pressure on the surface) is the reaction of its internal
        force on the fluid.  With i(r) = f_ext(r) - q_ions(r) E (the coupling
        force of Eq. 16 minus the external field's direct push on the local ion
        charge), particle p receives
            F_p = Z_p E - sum_{r in V_p} i(r) - (unassigned remainder) / P,
        where V_p are the fluid nodes of p's box widened by ceil(R) + 4 cells
        for which p is the particle with the nearest surface, and the remainder
        is the sum of i over fluid nodes in no V_p.  "Nearest" compares the FP64
        surface distances of surface_distance(); equal values go to the lower
        particle index.  Total momentum then changes only by E times the total
        charge (zero in a neutral box).  Torque: that of Z_p E on q_p(r) minus
        sum (r - r_p) x i.
        Returns (F, T) arrays of shape (P, 3).
        """
        P = len(self.particles)
        F = np.zeros((P, 3))
        T = np.zeros((P, 3))
        if P == 0:
            return F, T
        nx, ny, nz = self.n
        fluid = self.owner == FLUID
        q_ions = np.tensordot(self.valence, self.rho, axes=(0, 0)) if self.K else np.zeros(self.shape)
        ifield = np.where(fluid[None], fext - q_ions[None] * self.E.reshape(3, 1, 1, 1), 0.0)
        nearest, regions = self.nearest_particle()
        assigned = np.zeros(3)
        for pid, p in enumerate(self.particles):
            flat, dx, dy, dz = regions[pid]
            mine = (nearest[flat] == pid) & fluid.ravel()[flat]
            ix_ = ifield[0].ravel()[flat][mine]
            iy_ = ifield[1].ravel()[flat][mine]
            iz_ = ifield[2].ravel()[flat][mine]
            s = np.array([ix_.sum(), iy_.sum(), iz_.sum()])
            assigned += s
            Fq, Tq = self.charge_field_force(pid)
            F[pid] = Fq - s
            ax, ay, az = dx[mine], dy[mine], dz[mine]
            T[pid] = Tq - np.array([(ay * iz_ - az * iy_).sum(), (az * ix_ - ax * iz_).sum(),
                                    (ax * iy_ - ay * ix_).sum()])
        remainder = ifield.reshape(3, -1).sum(axis=1) - assigned
        F -= remainder / P
        return F, T

    def integrate(self, Fh, Th, Fs, Ts):
        """Symplectic Euler (Sec. III.B): v += F/m, r += v, omega += T/I, with
        F = momentum exchange + solute force + last step's create/destroy
        momentum.  Fixed particles keep their position and velocity."""
        for pid, p in enumerate(self.particles):
            p.force = Fh[pid] + Fs[pid] + p.f_trans
            p.torque = Th[pid] + Ts[pid]
            p.f_trans = np.zeros(3)
            if p.fixed:
                continue
            p.vel = p.vel + p.force / p.mass
            p.omega = p.omega + p.torque / p.inertia
            p.pos = p.pos + p.vel
            for a in range(3):
                if p.pos[a] >= self.n[a]:
                    p.pos[a] -= self.n[a]
                elif p.pos[a] < 0.0:
                    p.pos[a] += self.n[a]

    # ----- S5: re-flag and transitions ------------------------------------------
    def transitions(self, old_owner):
        """Create/destroy fluid (Sec. III.B) and expel/refill solute (Sec. III.D.1).

        Newly covered node: its fluid momentum sum_i f_i c_i goes to the particle;
        its solute is split equally among its N_f receiving neighbours.  Newly
        uncovered node: f = f^eq(mean neighbour density, v_b), whose momentum is
        taken from the particle; solute refilled by Eq. (17), each neighbour
        giving up rho/(N_f + 1) (Eq. 18), or left empty with VACATE_ZERO.
        Reading: neighbours are the 18 D3Q19 neighbours that are fluid both
        before and after the re-flag; all transfers use the values from before
        the transitions and are applied together.
        """
        nx, ny, nz = self.n
        new = self.owner
        covered = np.argwhere((old_owner == FLUID) & (new >= 0))
        uncovered = np.argwhere((old_owner >= 0) & (new == FLUID))
        if len(covered) == 0 and len(uncovered) == 0:
            return
        steady = (old_owner == FLUID) & (new == FLUID)
        rho_old = self.rho.copy()
        f_old = self.f.copy()
        drho = np.zeros_like(self.rho)

        def receivers(z, y, x):
            out = []
            for i in range(1, Q):
                c = CV[i]
                zz, yy, xx = (z + c[2]) % nz, (y + c[1]) % ny, (x + c[0]) % nx
                if steady[zz, yy, xx]:
                    out.append((zz, yy, xx))
            return out

        for z, y, x in covered:
            pid = int(new[z, y, x])
            mom = np.array([np.dot(CV[:, a].astype(np.float64), f_old[:, z, y, x]) for a in range(3)])
            self.particles[pid].f_trans += mom
            rec = receivers(z, y, x)
            if not rec:
                raise OracleError("expel: covered node has no fluid neighbour")
            for k in range(self.K):
                share = rho_old[k, z, y, x] / len(rec)
                drho[k, z, y, x] -= rho_old[k, z, y, x]
                for zz, yy, xx in rec:
                    drho[k, zz, yy, xx] += share
            self.f[:, z, y, x] = 0.0
        for z, y, x in uncovered:
            pid = int(old_owner[z, y, x])
            p = self.particles[pid]
            rec = receivers(z, y, x)
            rbar = np.mean([f_old[:, zz, yy, xx].sum() for zz, yy, xx in rec]) if rec else self.rho0
            lo, _ = particle_box(p.pos, p.radius)
            X = lo[0] + (x - lo[0]) % nx
            Y = lo[1] + (y - lo[1]) % ny
            Z = lo[2] + (z - lo[2]) % nz
            d = np.array([X - p.pos[0], Y - p.pos[1], Z - p.pos[2]])
            w = p.omega
            vb = np.array([p.vel[0] + (w[1] * d[2] - w[2] * d[1]),
                           p.vel[1] + (w[2] * d[0] - w[0] * d[2]),
                           p.vel[2] + (w[0] * d[1] - w[1] * d[0])])
            fn = feq(np.array(rbar), vb.reshape(3))
            self.f[:, z, y, x] = fn
            mom = np.array([np.dot(CV[:, a].astype(np.float64), fn) for a in range(3)])
            p.f_trans -= mom
            if self.flags & VACATE_ZERO:
                continue
            nf = len(rec)
            for k in range(self.K):
                for zz, yy, xx in rec:
                    share = rho_old[k, zz, yy, xx] / (nf + 1)
                    drho[k, z, y, x] += share
                    drho[k, zz, yy, xx] -= share
        self.rho += drho

    # ----- the whole step -----------------------------------------------------------
    def step(self, nsteps=1):
        for _ in range(nsteps):
            # S1
            self.phi = poisson(self.charge_density(), self.bjerrum)
            # S2a
            J = self.link_fluxes()
            fext = self.coupling_force(J)
            Fs, Ts = self.solute_forces(fext)
            # S2b
            fnew, u, Fh, Th = self.lb_step(fext)
            # S3
            adv = self.advection(u)
            div = J[:, 1:].sum(axis=1)
            self.rho = self.rho - div + adv
            self.f = fnew
            self.u = u
            # S4
            self.integrate(Fh, Th, Fs, Ts)
            # S5
            old = self.owner
            self._reflag_setup()
            self.transitions(old)
            self.steps_done += 1

    # ----- observables ------------------------------------------------------------------
    def density(self):
        return self.f.sum(axis=0)

    def total_species(self):
        return self.rho.reshape(self.K, -1).sum(axis=1)

    def total_charge(self):
        return float(np.dot(self.valence, self.total_species())) + \
            sum(p.charge for p in self.particles) + float(self.qwall.sum())

    def fluid_momentum(self):
        return np.array([np.tensordot(CV[:, a].astype(np.float64), self.f, axes=(0, 0)).sum()
                         for a in range(3)])
