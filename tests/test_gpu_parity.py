"""Parity of the CUDA FP64 path with the FP64 oracle, element by element, on
the same seeded inputs (tolerance 1e-11 relative, see tests/pairs.py)."""
import numpy as np
import pytest

import workloads
from oracle import ek_oracle as O
from pairs import TOL, compare, make_pair, rel_err

pytestmark = pytest.mark.gpu


# --------------------------------------------------------------------------
# S1 alone: the standalone Poisson entry point against the oracle's solve
# --------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(8, 8, 8), (16, 12, 8), (24, 16, 18), (48, 32, 64), (32, 32, 32),
                                   (128, 8, 16), (12, 96, 27)])
def test_poisson_standalone(gpu_lib, shape):
    import torch
    ek = gpu_lib
    nx, ny, nz = shape
    rng = np.random.default_rng(7)
    q = rng.standard_normal((nz, ny, nx))
    ref = O.poisson(q, 0.7)
    qd = torch.from_numpy(q.ravel()).cuda()
    phi = torch.empty_like(qd)
    spec = torch.empty(ek.poisson_scratch_bytes(nx, ny, nz) // 8, dtype=torch.float64, device="cuda")
    ek.poisson_solve(qd, phi, shape, 0.7, spec)
    torch.cuda.synchronize()
    got = phi.cpu().numpy().reshape(nz, ny, nx)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # in place (q and phi alias)
    ek.poisson_solve(qd, qd, shape, 0.7, spec)
    torch.cuda.synchronize()
    assert np.max(np.abs(qd.cpu().numpy().reshape(nz, ny, nx) - ref)) <= 1e-12 * np.max(np.abs(ref))


# --------------------------------------------------------------------------
# each stage alone on a perturbed state with a moving, rotating particle
# --------------------------------------------------------------------------
def test_stages_one_by_one(gpu_lib):
    ek = gpu_lib
    case = workloads.small_case(n=(16, 16, 16), radius=3.2, charge=-15.0)
    o, s = make_pair(ek, case, vel=[(0.02, -0.01, 0.015)], omega=[(0.003, -0.002, 0.004)])
    # S1
    o.phi = O.poisson(o.charge_density(), o.bjerrum)
    s.run_stage(1)
    assert rel_err(s.get_fields(ek.FIELD_PHI), o.phi) <= TOL
    assert rel_err(s.get_fields(ek.FIELD_CHARGE), o.charge_density()) <= TOL
    # S2 + S3
    J = o.link_fluxes()
    fext = o.coupling_force(J)
    Fs, Ts = o.solute_forces(fext)
    fnew, u, Fh, Th = o.lb_step(fext)
    adv = o.advection(u)
    o.rho = o.rho - J[:, 1:].sum(axis=1) + adv
    o.f, o.u = fnew, u
    s.run_stage(2)
    compare(ek, o, s, what=("species", "populations", "velocity", "phi", "owner", "psi"))
    # S4
    o.integrate(Fh, Th, Fs, Ts)
    s.run_stage(4)
    compare(ek, o, s, what=("particles",))
    # S5
    old = o.owner.copy()
    o._reflag_setup()
    o.transitions(old)
    s.run_stage(5)
    compare(ek, o, s)


# --------------------------------------------------------------------------
# whole steps
# --------------------------------------------------------------------------
def test_steps_small_box(gpu_lib):
    ek = gpu_lib
    case = workloads.small_case(n=(16, 16, 16), radius=3.0, charge=-20.0)
    o, s = make_pair(ek, case)
    for _ in range(4):
        o.step(5)
        s.step(5)
        compare(ek, o, s)


def test_workload_small_100_steps(gpu_lib):
    """The 32^3 single-sphere workload (R=4, Z=-50, E=0.01), 100 steps."""
    ek = gpu_lib
    case = workloads.workload("small")
    o, s = make_pair(ek, case, perturb=0.0)
    o.step(100)
    s.step(100)
    errs = compare(ek, o, s)
    assert max(errs.values()) <= TOL


@pytest.mark.parametrize("variant", ["simple", "vacate_zero", "norm_vp", "trt", "three_species",
                                     "no_neutralize"])
def test_scheme_variants(gpu_lib, variant):
    ek = gpu_lib
    case = workloads.small_case(n=(16, 16, 16), radius=3.0, charge=-20.0)
    flags = O.PV | O.NEUTRALIZE
    magic = None
    if variant == "simple":
        flags = O.NEUTRALIZE
    elif variant == "vacate_zero":
        flags |= O.VACATE_ZERO
    elif variant == "norm_vp":
        flags |= O.CHARGE_NORM_VP
    elif variant == "trt":
        magic = 3.0 / 16.0
    elif variant == "three_species":
        case["valence"], case["D"], case["bulk"] = (1, -1, 2), (0.2, 0.3, 0.15), (1e-3, 1e-3, 5e-4)
    elif variant == "no_neutralize":
        flags = O.PV
    o, s = make_pair(ek, case, flags=flags, magic=magic, vel=[(0.05, 0.02, -0.01)], rho_p=50.0)
    for _ in range(3):
        o.step(6)
        s.step(6)
        compare(ek, o, s)


def test_covering_and_uncovering(gpu_lib):
    """A heavy sphere dragged across several cells: transitions every few steps."""
    ek = gpu_lib
    case = workloads.small_case(n=(16, 16, 16), radius=3.0, charge=-10.0)
    o, s = make_pair(ek, case, vel=[(0.06, 0.025, -0.015)], rho_p=1e9, perturb=0.0)
    N0 = o.total_species().copy()
    flips = 0
    for _ in range(10):
        old = o.owner.copy()
        o.step(5)
        s.step(5)
        flips += int((old != o.owner).sum())
        compare(ek, o, s)
        tot = np.array([s.get_fields(ek.FIELD_SPECIES, k).sum() for k in range(o.K)])
        assert np.allclose(tot, N0, rtol=1e-12, atol=0)
    assert flips > 20


def test_several_particles_ragged_box(gpu_lib):
    ek = gpu_lib
    case = workloads.small_case(n=(24, 18, 32), radius=2.5, charge=-12.0, nparticles=3, seed=5)
    o, s = make_pair(ek, case, vel=[(0.01, 0.0, 0.02), (-0.02, 0.01, 0.0), (0.0, -0.015, 0.01)])
    o.step(8)
    s.step(8)
    compare(ek, o, s)


def test_fixed_particle_co_moving_frame(gpu_lib):
    ek = gpu_lib
    case = workloads.small_case(n=(16, 16, 16), radius=3.0, charge=-20.0)
    o, s = make_pair(ek, case, fixed=True)
    o.step(10)
    s.step(10)
    compare(ek, o, s)
    assert np.allclose(s.get_particles()[0]["pos"], np.mod(case["particles"][0]["pos"], 16))


def test_charged_walls_and_body_force(gpu_lib):
    """Slit between two charged walls (static boundaries, wall charge) with a
    body force: exercises wall bounce-back, zero-flux walls and rho_b."""
    ek = gpu_lib
    case = workloads.small_case(n=(16, 8, 8), radius=1.0, charge=0.0, nparticles=0)
    nz, ny, nx = 8, 8, 16
    walls = np.zeros((nz, ny, nx), dtype=bool)
    walls[:, :, 0] = True
    walls[:, :, 15] = True
    qw = np.where(walls, -0.01, 0.0)
    o, s = make_pair(ek, case, walls=walls, wall_charge=qw, magic=3.0 / 16.0, g=(0.0, 1e-5, 0.0))
    o.step(15)
    s.step(15)
    compare(ek, o, s)


def test_fluid_only(gpu_lib):
    ek = gpu_lib
    case = workloads.small_case(n=(16, 8, 12), nparticles=0)
    case["valence"], case["D"], case["bulk"] = (), (), ()
    o, s = make_pair(ek, case, g=(1e-5, 0.0, -2e-5), magic=3.0 / 16.0)
    o.step(10)
    s.step(10)
    compare(ek, o, s)


# --------------------------------------------------------------------------
# the benchmark workload at full size (128^3, R=8, Z=-300): full-field parity
# every 5 of the first 20 steps from the same state, and conservation over 50
# more steps
# --------------------------------------------------------------------------
def test_single_workload_full_size(gpu_lib):
    ek = gpu_lib
    case = workloads.workload("single")
    o, s = make_pair(ek, case, perturb=0.0)
    for _ in range(4):
        o.step(5)
        s.step(5)
        compare(ek, o, s)
    N0 = o.total_species()
    s.step(50)
    tot = np.array([s.get_fields(ek.FIELD_SPECIES, k).sum() for k in range(2)])
    assert np.allclose(tot, N0, rtol=1e-12, atol=0)
    p = s.get_particles()[0]
    assert p["vel"][0] < 0.0  # negative sphere in +E moves along -x


def test_errors_are_status_codes(gpu_lib):
    ek = gpu_lib
    s = ek.EKSystem((16, 16, 16))
    with pytest.raises(ek.EKError):
        s.add_particle((8, 8, 8), radius=6.0)  # 2R + 6 > 16
    s.add_particle((8, 8, 8), radius=3.0)
    s.add_particle((9, 8, 8), radius=3.0)  # overlaps the first
    with pytest.raises(ek.EKError) as e:
        s.step(1)
    assert e.value.code == -5
    with pytest.raises(ek.EKError):
        ek.EKSystem((10, 16, 16))  # 10 = 2 * 5 is not 2^a 3^b


def test_particle_crosses_periodic_boundary(gpu_lib):
    """A heavy sphere pushed across the x = 0 seam (and y): the boxes of the
    previous and the current position lie in different periodic images."""
    ek = gpu_lib
    case = workloads.small_case(n=(16, 16, 16), radius=3.0, charge=-10.0)
    case["particles"][0]["pos"] = [0.9, 15.6, 7.3]
    o, s = make_pair(ek, case, vel=[(-0.09, 0.08, 0.01)], rho_p=1e9, perturb=0.0)
    N0 = o.total_species().copy()
    for _ in range(6):
        o.step(5)
        s.step(5)
        compare(ek, o, s)
    assert o.particles[0].pos[0] > 8.0  # wrapped to the far side
    tot = np.array([s.get_fields(ek.FIELD_SPECIES, k).sum() for k in range(o.K)])
    assert np.allclose(tot, N0, rtol=1e-12, atol=0)


@pytest.mark.parametrize("flags", [0, 16])
def test_nonfinite_state_is_reported_not_propagated_silently(gpu_lib, flags):
    """A NaN written into the populations of one node (host fault injection)
    makes the next step return EK_ERR_UNSTABLE; the context then refuses
    further steps instead of running on."""
    ek = gpu_lib
    s = ek.EKSystem((16, 16, 16), flags=flags)
    s.step(2)
    f = s.get_fields(ek.FIELD_POPULATIONS)
    f = np.array(f, dtype=np.float64)
    f.reshape(19, -1)[3, 1234] = np.nan
    s.set_field(ek.FIELD_POPULATIONS, f.ravel())
    with pytest.raises(ek.EKError) as e:
        s.step(1)
    assert e.value.code == -4  # EK_ERR_UNSTABLE
    with pytest.raises(ek.EKError):
        s.step(1)
    s.close()


def test_allocation_failure_is_reported_and_cleaned_up(gpu_lib):
    """The allocation-failure hook: the fifth field allocation of the next
    ek_create fails; ek_create returns EK_ERR_NOMEM after freeing the rest,
    and the next ek_create succeeds."""
    ek = gpu_lib
    ek.debug_fail_alloc(5)
    with pytest.raises(ek.EKError) as e:
        ek.EKSystem((32, 32, 32), flags=16)
    assert e.value.code == -2  # EK_ERR_NOMEM
    s = ek.EKSystem((32, 32, 32), flags=16)
    s.step(2)
    s.close()
    ek.debug_fail_alloc(0)
