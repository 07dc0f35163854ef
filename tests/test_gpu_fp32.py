"""FP32-storage form (populations as float deviations, int32 fixed-point
species): exact species conservation, agreement with the FP64 oracle at FP32
tolerance, and the particle mobility within 1e-3 of the FP64 form."""
import numpy as np
import pytest

import workloads
from oracle import ek_oracle as O
from pairs import make_pair, perm_to_oracle, rel_err

pytestmark = pytest.mark.gpu

FP32 = 16
TOL32 = 2e-4  # per element, floor 1e-3 of the field's max (FP32 rounding ~6e-8 per op, species units 2^-20 of bulk)


def totals(ek, s, K):
    return np.array([s.get_fields(ek.FIELD_SPECIES, k).sum() for k in range(K)])


def test_fp32_fields_match_oracle(gpu_lib):
    ek = gpu_lib
    case = workloads.small_case(n=(16, 16, 16), radius=3.0, charge=-20.0)
    o, s = make_pair(ek, case, flags=O.PV | O.NEUTRALIZE | FP32, vel=[(0.02, -0.01, 0.01)])
    for _ in range(2):
        o.step(5)
        s.step(5)
        assert np.array_equal(s.get_fields(ek.FIELD_OWNER), o.owner.astype(float))
        fluid = o.owner == O.FLUID
        for k in range(o.K):
            assert rel_err(s.get_fields(ek.FIELD_SPECIES, k), o.rho[k]) < TOL32
        fg = s.get_fields(ek.FIELD_POPULATIONS)[perm_to_oracle(ek)]
        assert rel_err(fg[:, fluid], o.f[:, fluid]) < 1e-5
        assert rel_err(s.get_fields(ek.FIELD_PHI), o.phi) < TOL32
        assert rel_err(s.get_fields(ek.FIELD_PSI), o.psi) == 0.0
        u = s.get_fields(ek.FIELD_VELOCITY)
        assert rel_err(u[:, fluid], o.u[:, fluid], floor=1.0) < 1e-3
        p = s.get_particles()[0]
        assert np.max(np.abs(p["pos"] - o.particles[0].pos)) < 1e-6
        assert np.max(np.abs(p["vel"] - o.particles[0].vel)) < 1e-3 * np.max(np.abs(o.particles[0].vel))


def test_fp32_fields_match_oracle_workload_small_100_steps(gpu_lib):
    """The 32^3 single-sphere workload (R = 4, Z = -50, E = 0.01) for 100 steps in
    the FP32-storage form against the FP64 oracle, field by field: species
    and Phi per element (floor 1e-3 of the field's max), populations of fluid
    nodes, Psi exactly, the particle's position and velocity."""
    ek = gpu_lib
    case = workloads.workload("small")
    o, s = make_pair(ek, case, flags=O.PV | O.NEUTRALIZE | FP32, perturb=0.0)
    for _ in range(4):
        o.step(25)
        s.step(25)
        assert np.array_equal(s.get_fields(ek.FIELD_OWNER), o.owner.astype(float))
        fluid = o.owner == O.FLUID
        for k in range(o.K):
            assert rel_err(s.get_fields(ek.FIELD_SPECIES, k), o.rho[k]) < 1e-3
        fg = s.get_fields(ek.FIELD_POPULATIONS)[perm_to_oracle(ek)]
        assert rel_err(fg[:, fluid], o.f[:, fluid]) < 1e-5
        assert rel_err(s.get_fields(ek.FIELD_PHI), o.phi) < 1e-3
        assert rel_err(s.get_fields(ek.FIELD_PSI), o.psi) == 0.0
        p = s.get_particles()[0]
        assert np.max(np.abs(p["pos"] - o.particles[0].pos)) < 1e-5
        assert np.max(np.abs(p["vel"] - o.particles[0].vel)) < 2e-3 * np.max(np.abs(o.particles[0].vel))


def test_fp32_species_conserved_exactly(gpu_lib):
    """A heavy sphere dragged across cells: every covering, uncovering, flux and
    advection moves whole units, so the totals never change, bit for bit."""
    ek = gpu_lib
    case = workloads.small_case(n=(16, 16, 16), radius=3.0, charge=-10.0)
    o, s = make_pair(ek, case, flags=O.PV | O.NEUTRALIZE | FP32, vel=[(0.06, 0.025, -0.015)],
                     rho_p=1e9, perturb=0.0)
    N0 = totals(ek, s, 2)
    owner0 = s.get_fields(ek.FIELD_OWNER)
    flips = 0
    for _ in range(12):
        s.step(5)
        assert np.array_equal(totals(ek, s, 2), N0)
        ow = s.get_fields(ek.FIELD_OWNER)
        flips += int((ow != owner0).sum())
        owner0 = ow
    assert flips > 20


@pytest.mark.parametrize("flags", [O.NEUTRALIZE | FP32, O.PV | O.NEUTRALIZE | O.VACATE_ZERO | FP32])
def test_fp32_conservation_scheme_variants(gpu_lib, flags):
    ek = gpu_lib
    case = workloads.small_case(n=(16, 16, 16), radius=3.0, charge=-10.0)
    o, s = make_pair(ek, case, flags=flags, vel=[(0.07, 0.0, 0.02)], rho_p=1e9, perturb=0.01)
    N0 = totals(ek, s, 2)
    s.step(40)
    assert np.array_equal(totals(ek, s, 2), N0)


def _system(ek, w, flags, fixed=False):
    s = ek.EKSystem(w["shape"], nu=w["nu"], rho0=w["rho0"], bjerrum=w["bjerrum"],
                    valence=w["valence"], D=w["D"], bulk=w["bulk"], flags=flags)
    for p in w["particles"]:
        s.add_particle(p["pos"], radius=p["radius"], charge=p["charge"], rho_p=w["rho_p"],
                       fixed=fixed)
    s.set_field(ek.FIELD_E_EXT, np.array(w["E"]))
    return s


def mobility_velocity(ek, w, flags, fixed, steps, every=50):
    """Particle velocity relative to the mean fluid velocity, averaged over the
    second half of the run (the electrophoretic velocity; for a fixed sphere
    the particle is at rest and the fluid streams past it)."""
    s = _system(ek, w, flags, fixed)
    N0 = totals(ek, s, len(w["valence"]))
    rel = []
    for _ in range(steps // every):
        s.step(every)
        v = s.get_particles()[0]["vel"][0]
        u = s.get_fields(ek.FIELD_VELOCITY)[0]
        rel.append(v - u[s.get_fields(ek.FIELD_OWNER) == -1].mean())
    return float(np.mean(rel[len(rel) // 2:])), s, N0


def test_fp32_mobility_matches_fp64(gpu_lib):
    """32^3, R = 4, Z = -50, E = 0.01: the time-averaged electrophoretic
    velocity of the FP32 form within 1e-3 of the FP64 form, species exact."""
    ek = gpu_lib
    w = workloads.workload("small")
    v64, _, _ = mobility_velocity(ek, w, ek.EK_PV | ek.EK_NEUTRALIZE, False, 3000)
    v32, s32, N0 = mobility_velocity(ek, w, ek.EK_PV | ek.EK_NEUTRALIZE | FP32, False, 3000)
    assert abs(v32 - v64) <= 1e-3 * abs(v64)
    assert np.array_equal(totals(ek, s32, 2), N0)
    assert v64 < 0.0


def test_moving_matches_co_moving_fixed_sphere(gpu_lib):
    """The paper's validation (Sec. IV.A): the electrophoretic velocity of the
    moving sphere equals the electro-osmotic flow past the same sphere held
    fixed, to a few per cent (the paper: 1.4% and 2.4%)."""
    ek = gpu_lib
    w = workloads.workload("small")
    # the co-moving frame needs the momentum diffusion time L^2/nu (~6000 steps)
    vm, _, _ = mobility_velocity(ek, w, ek.EK_PV | ek.EK_NEUTRALIZE, False, 6000)
    vf, _, _ = mobility_velocity(ek, w, ek.EK_PV | ek.EK_NEUTRALIZE, True, 6000)
    assert abs(vm - vf) <= 0.03 * abs(vf)


def test_fp32_mobility_many_spheres_matches_fp64(gpu_lib):
    """The many-colloid workload at full size (256^3, 64 spheres R = 5 with
    charges in [-100, -50], species z = +1, -1, +2, E = 0.005): the mean
    electrophoretic velocity of the spheres along E, averaged over steps
    1000-2000 (the double layers have formed after a few hundred steps; the
    window average takes out their slow drift), of the FP32 form within 1e-3
    of the FP64 form; the FP32 species totals stay exact."""
    ek = gpu_lib
    w = workloads.workload("many")
    K = len(w["valence"])

    def run(flags):
        s = _system(ek, w, flags)
        N0 = totals(ek, s, K)
        s.step(1000)
        vs = []
        for _ in range(10):
            s.step(100)
            vs.append(np.mean([p["vel"][0] for p in s.get_particles()]))
        v = float(np.mean(vs))
        tot = totals(ek, s, K)
        s.close()
        return v, N0, tot

    v64, _, _ = run(ek.EK_PV | ek.EK_NEUTRALIZE)
    v32, N0, tot = run(ek.EK_PV | ek.EK_NEUTRALIZE | FP32)
    assert v64 < 0.0
    assert abs(v32 - v64) <= 1e-3 * abs(v64), (v32, v64)
    assert np.array_equal(tot, N0)


def test_fp32_mobility_single_128_stationary(gpu_lib):
    """The 128^3 single-sphere workload: the electrophoretic velocity averaged
    over steps 2000-3000 (past the start-up transient), FP32 form within 1e-3
    of the FP64 form."""
    ek = gpu_lib
    w = workloads.workload("single")

    def run(flags):
        s = _system(ek, w, flags)
        s.step(2000)
        vs = []
        for _ in range(10):
            s.step(100)
            vs.append(s.get_particles()[0]["vel"][0])
        s.close()
        return float(np.mean(vs))

    v64 = run(ek.EK_PV | ek.EK_NEUTRALIZE)
    v32 = run(ek.EK_PV | ek.EK_NEUTRALIZE | FP32)
    assert v64 < 0.0
    assert abs(v32 - v64) <= 1e-3 * abs(v64), (v32, v64)


def test_fp32_single_workload_full_size(gpu_lib):
    ek = gpu_lib
    w = workloads.workload("single")
    s64 = _system(ek, w, ek.EK_PV | ek.EK_NEUTRALIZE)
    s32 = _system(ek, w, ek.EK_PV | ek.EK_NEUTRALIZE | FP32)
    N0 = totals(ek, s32, 2)
    s64.step(100)
    s32.step(100)
    v64 = s64.get_particles()[0]["vel"]
    v32 = s32.get_particles()[0]["vel"]
    assert np.linalg.norm(v32 - v64) <= 1e-3 * np.linalg.norm(v64)
    assert np.array_equal(totals(ek, s32, 2), N0)
    assert v32[0] < 0.0


@pytest.mark.parametrize("shape", [(32, 32, 32), (64, 32, 128), (128, 64, 32), (256, 32, 64),
                                   (512, 32, 32), (128, 128, 128), (32, 256, 32), (64, 32, 256),
                                   (48, 32, 32), (32, 48, 64), (96, 24, 48), (192, 48, 96),
                                   (36, 32, 32), (32, 512, 32), (32, 32, 512), (48, 256, 512)])
def test_fp32_poisson_shapes(gpu_lib, shape):
    """S1 of the FP32 form against the oracle's Poisson solve of the same
    charge, within FP32 rounding of the spectrum: edges 2^k and 3 2^k from 24
    to 512 take the specialised line transforms (with n_y, n_z in {32, 48, 64,
    128} the y and z passes of a kx plane run on a cluster of two CTAs that
    exchange halves through distributed shared memory; 256- and 512-point y
    and z lines run as four-step 16 x 16 and 16 x 32 transforms), other edges
    (36) the generic ones."""
    ek = gpu_lib
    nx, ny, nz = shape
    s = ek.EKSystem(shape, nu=1.0 / 6.0, rho0=1.0, bjerrum=0.7, valence=(1, -1), D=(0.3, 0.3),
                    bulk=(1e-3, 1e-3), flags=FP32)
    for k in range(2):
        r = 1e-3 * (1.0 + workloads.perturbation(nx * ny * nz, 0.5, 100 + k))
        s.set_field(ek.FIELD_SPECIES, r, component=k)
    rho = [s.get_fields(ek.FIELD_SPECIES, k).reshape(nz, ny, nx) for k in range(2)]
    ref = O.poisson(rho[0] - rho[1], 0.7)
    s.run_stage(1)
    got = s.get_fields(ek.FIELD_PHI).reshape(nz, ny, nx)
    assert np.max(np.abs(got - ref)) <= 2e-5 * np.max(np.abs(ref))


def test_fp32_steps_are_deterministic_with_many_particles(gpu_lib):
    """Two identical systems with many particles, stepped asynchronously
    (graphs, the particle chain beside S3): bit-identical fields and particle
    records, transitions included (the transitions' momentum is summed in a
    fixed order, not by atomic adds)."""
    import torch
    ek = gpu_lib
    w = workloads.small_case((96, 96, 96), radius=5.0, charge=-60.0, nparticles=14, seed=11, E=0.02)

    def run():
        s = ek.EKSystem(w["shape"], nu=w["nu"], rho0=w["rho0"], bjerrum=w["bjerrum"],
                        valence=w["valence"], D=w["D"], bulk=w["bulk"],
                        flags=ek.EK_PV | ek.EK_NEUTRALIZE | ek.EK_FP32)
        for p in w["particles"]:
            s.add_particle(p["pos"], radius=p["radius"], charge=p["charge"], rho_p=w["rho_p"])
        s.set_field(ek.FIELD_E_EXT, np.array(w["E"], dtype=np.float64))
        st = torch.cuda.Stream()
        s.set_stream(st)
        s.step(120)
        out = [s.get_fields(ek.FIELD_SPECIES, k) for k in range(2)]
        out += [s.get_fields(ek.FIELD_POPULATIONS), s.get_fields(ek.FIELD_OWNER)]
        parts = s.get_particles()
        out += [np.array([p["pos"] for p in parts]), np.array([p["vel"] for p in parts]),
                np.array([p["omega"] for p in parts])]
        s.close()
        return out

    a, b = run(), run()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("species,flags", [
    (((1,), (0.3,), (1e-3,)), O.PV | FP32),  # one species cannot neutralise the box
    (((1, -1, 2, -2), (0.3, 0.2, 0.15, 0.1), (1e-3, 1e-3, 5e-4, 5e-4)), O.PV | O.NEUTRALIZE | FP32)])
def test_fp32_species_counts_match_oracle(gpu_lib, species, flags):
    """One and four species (the S2 and S3 kernels are instantiated per species
    count) on a 16^3 box, narrower than the 32-node tile: boundary flags and Psi
    exactly, species and Phi per element within 2e-4 of the FP64 oracle after
    ten steps of a moving sphere, species totals exact."""
    ek = gpu_lib
    case = workloads.small_case(n=(16, 16, 16), radius=3.0, charge=-20.0)
    case["valence"], case["D"], case["bulk"] = species
    o, s = make_pair(ek, case, flags=flags, vel=[(0.03, -0.02, 0.01)])
    K = len(species[0])
    N0 = totals(ek, s, K)
    o.step(10)
    s.step(10)
    assert np.array_equal(s.get_fields(ek.FIELD_OWNER), o.owner.astype(float))
    for k in range(K):
        assert rel_err(s.get_fields(ek.FIELD_SPECIES, k), o.rho[k]) < TOL32, k
    assert rel_err(s.get_fields(ek.FIELD_PHI), o.phi) < TOL32
    assert rel_err(s.get_fields(ek.FIELD_PSI), o.psi) == 0.0
    fluid = o.owner == O.FLUID
    fg = s.get_fields(ek.FIELD_POPULATIONS)[perm_to_oracle(ek)]
    assert rel_err(fg[:, fluid], o.f[:, fluid]) < 1e-5
    assert np.array_equal(totals(ek, s, K), N0)
