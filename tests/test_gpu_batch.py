"""Batched ensemble: systems of different box sizes, salts, fields and
particles advanced together by one graph launch per step must end where the
same systems stepped one by one end, and the autotuner's trials are real,
conserving steps."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

FP32 = 16


def make(ek, w, flags):
    s = ek.EKSystem(w["shape"], nu=w["nu"], rho0=w["rho0"], bjerrum=w["bjerrum"],
                    valence=w["valence"], D=w["D"], bulk=w["bulk"], flags=flags)
    for p in w["particles"]:
        s.add_particle(p["pos"], radius=p["radius"], charge=p["charge"], rho_p=w["rho_p"])
    s.set_field(ek.FIELD_E_EXT, np.array(w["E"], dtype=np.float64))
    return s


def ensemble():
    # small boxes (edges 16..32) so that the spheres of R <= 4 fit (2R + 6 <= edge)
    return workloads.batch_ensemble(6, seed=77, edges=(16, 24, 32), radius=(2.5, 4.0),
                                    charge=(-30.0, -10.0), bulk=(1e-3, 1e-2))


def state(ek, s):
    out = {k: s.get_fields(ek.FIELD_SPECIES, k) for k in range(2)}
    out["f"] = s.get_fields(ek.FIELD_POPULATIONS)
    out["phi"] = s.get_fields(ek.FIELD_PHI)
    out["owner"] = s.get_fields(ek.FIELD_OWNER)
    p = s.get_particles()[0]
    out["pos"] = np.array(p["pos"])
    out["vel"] = np.array(p["vel"])
    return out


def test_batch_matches_systems_stepped_alone(gpu_lib):
    ek = gpu_lib
    ws = ensemble()
    # five FP32-form systems and one FP64-form system in the same batch
    flags = [ek.EK_PV | ek.EK_NEUTRALIZE | (FP32 if i < 5 else 0) for i in range(len(ws))]
    batched = [make(ek, w, f) for w, f in zip(ws, flags)]
    alone = [make(ek, w, f) for w, f in zip(ws, flags)]
    b = ek.EKBatch(batched)
    assert len(b) == len(ws)
    b.step(3)
    b.step(4)  # odd total: both ping-pong parities captured and replayed
    for s in alone:
        s.step(7)
    for i, (sb, sa) in enumerate(zip(batched, alone)):
        x, y = state(ek, sb), state(ek, sa)
        assert np.array_equal(x["owner"], y["owner"]), i
        for key in x:
            scale = max(np.max(np.abs(y[key])), 1e-300)
            assert np.max(np.abs(x[key] - y[key])) <= 1e-12 * scale, (i, key)
        if flags[i] & FP32:
            for k in range(2):  # int units: the same arithmetic gives the same integers
                assert np.array_equal(x[k], y[k]), (i, k)
    assert sum(s.kernel_launches() for s in batched) == sum(s.kernel_launches() for s in alone)
    b.close()


def test_batch_tuner_steps_conserve_and_choose_a_candidate(gpu_lib):
    ek = gpu_lib
    ws = ensemble()
    systems = [make(ek, w, ek.EK_PV | ek.EK_NEUTRALIZE | FP32) for w in ws]
    totals = [[s.get_fields(ek.FIELD_SPECIES, k).sum() for k in range(2)] for s in systems]
    b = ek.EKBatch(systems)
    cfg, ms = b.tune(1)
    assert cfg["branches"] in (len(ws), 8, 16, 32, 64) and cfg["planes_per_block"] in (2, 4, 8)
    assert ms > 0.0
    b.step(5)
    for s, t in zip(systems, totals):
        for k in range(2):
            assert s.get_fields(ek.FIELD_SPECIES, k).sum() == t[k]
        p = s.get_particles()[0]
        assert np.all(np.isfinite(p["pos"])) and np.all(np.isfinite(p["vel"]))
    b.close()


def compare(ek, batched, alone, fp32):
    for i, (sb, sa) in enumerate(zip(batched, alone)):
        x, y = state(ek, sb), state(ek, sa)
        assert np.array_equal(x["owner"], y["owner"]), i
        for key in x:
            scale = max(np.max(np.abs(y[key])), 1e-300)
            assert np.max(np.abs(x[key] - y[key])) <= 1e-12 * scale, (i, key)
        if fp32:
            for k in range(2):  # int units: the same arithmetic gives the same integers
                assert np.array_equal(x[k], y[k]), (i, k)


@pytest.mark.parametrize("edges,overlap,form", [((16, 24, 32), 1, 1), ((32, 48, 64), 1, 1),
                                               ((32, 48, 64), 0, 1), ((16, 24, 32), 1, 2),
                                               ((32, 48, 64), 0, 2)])
def test_fused_batch_matches_systems_stepped_alone(gpu_lib, edges, overlap, form):
    """The fused forms (each kernel once over all systems' (system, block)
    ranges; form 2 with the particle kernels as persistent launches whose
    phases meet at grid barriers) against the same FP32 systems stepped
    alone: edges 32, 48 and 64 take the batched S1 passes, 16 and 24 their own
    S1 inside the fused step."""
    ek = gpu_lib
    ws = workloads.batch_ensemble(6, seed=78, edges=edges, radius=(2.5, 4.0),
                                  charge=(-30.0, -10.0), bulk=(1e-3, 1e-2))
    flags = ek.EK_PV | ek.EK_NEUTRALIZE | FP32
    batched = [make(ek, w, flags) for w in ws]
    alone = [make(ek, w, flags) for w in ws]
    b = ek.EKBatch(batched)
    assert b.config()["fused"] == 1  # the default where the batch allows it
    b.set_config(particle_chain_beside_s3=overlap, fused=form)
    assert b.config()["fused"] == form
    b.step(3)
    b.step(4)
    for s in alone:
        s.step(7)
    compare(ek, batched, alone, True)
    # a step is one set of launches for the whole batch
    assert sum(s.kernel_launches() for s in batched) < sum(s.kernel_launches() for s in alone)
    b.close()


def test_fused_and_branch_forms_agree_over_a_change_of_form(gpu_lib):
    """Steps of the fused form, then of the branch form, then fused again end
    where the systems stepped alone end (the forms share every system's state)."""
    ek = gpu_lib
    ws = workloads.batch_ensemble(4, seed=79, edges=(32, 48), radius=(2.5, 4.0),
                                  charge=(-30.0, -10.0), bulk=(1e-3, 1e-2))
    flags = ek.EK_PV | ek.EK_NEUTRALIZE | FP32
    batched = [make(ek, w, flags) for w in ws]
    alone = [make(ek, w, flags) for w in ws]
    b = ek.EKBatch(batched)
    b.step(2)
    b.set_config(fused=0, branches=2)
    b.step(3)
    b.set_config(fused=1)
    b.step(2)
    for s in alone:
        s.step(7)
    compare(ek, batched, alone, True)
    b.close()


def test_fused_form_refused_for_a_mixed_batch(gpu_lib):
    ek = gpu_lib
    ws = ensemble()[:2]
    systems = [make(ek, ws[0], ek.EK_PV | FP32), make(ek, ws[1], ek.EK_PV)]
    b = ek.EKBatch(systems)
    assert not b.config()["fused"]
    with pytest.raises(ek.EKError):
        b.set_config(fused=1)
    b.step(1)
    b.close()


def test_grid_barrier_wait_is_bounded_and_reported(gpu_lib):
    """Failure detection of the persistent particle chain without a fault: one
    CTA of each persistent launch leaves before the first grid barrier, so the
    others' waits run out (after 20 ms); the kernel ends, the batch reports
    EK_ERR_TIMEOUT and its systems refuse further work, and the device stays
    usable (a new system steps normally)."""
    ek = gpu_lib
    ws = workloads.batch_ensemble(4, seed=80, edges=(32, 48), radius=(2.5, 4.0),
                                  charge=(-30.0, -10.0), bulk=(1e-3, 1e-2))
    flags = ek.EK_PV | ek.EK_NEUTRALIZE | FP32
    systems = [make(ek, w, flags) for w in ws]
    b = ek.EKBatch(systems)
    b.set_config(fused=2)
    b.step(2)  # the barriers pass when every CTA arrives
    b.wait_test(leave_cta=0, limit_ms=20.0)
    with pytest.raises(ek.EKError) as e:
        b.step(1)
    assert e.value.code == -7  # EK_ERR_TIMEOUT
    with pytest.raises(ek.EKError):
        b.step(1)  # the systems stopped part way through a step
    b.close()
    s = make(ek, ws[0], flags)
    s.step(3)
    p = s.get_particles()[0]
    assert np.all(np.isfinite(p["pos"]))


def _oracle_members(ek, ws, flags):
    from oracle import ek_oracle as O  # noqa: F401  (the pairs helper builds both sides)
    from pairs import make_pair
    return [make_pair(ek, w, flags=flags, perturb=0.0) for w in ws]


def test_batch_members_match_oracle_fp64(gpu_lib):
    """Three ensemble members (ragged boxes of edges 16..32, one sphere each,
    their own salt, charge and field) in the FP64 form, advanced by the batch,
    against the FP64 oracle stepped member by member: every field at the
    parity tolerance of the single-system path (1e-11)."""
    from pairs import compare as oracle_compare
    ek = gpu_lib
    ws = workloads.batch_ensemble(3, seed=81, edges=(16, 24, 32), radius=(2.5, 4.0),
                                  charge=(-30.0, -10.0), bulk=(1e-3, 1e-2))
    pairs = _oracle_members(ek, ws, ek.EK_PV | ek.EK_NEUTRALIZE)
    b = ek.EKBatch([s for _, s in pairs])
    b.step(3)
    b.step(4)
    for o, s in pairs:
        o.step(7)
        oracle_compare(ek, o, s)
    b.close()


@pytest.mark.parametrize("form", [1, 2])
def test_batch_members_match_oracle_fp32_fused(gpu_lib, form):
    """Three FP32-form members on the fused batch path (edges 32 and 48 take
    the batched S1 passes; form 2 runs the particle kernels as persistent
    launches with grid barriers) against the FP64 oracle: boundary flags and
    Psi exactly, species and Phi per element within 2e-4 (floor 1e-3 of the
    field's max), fluid populations within 1e-5, the particle within 1e-6 in
    position and 2e-3 of its speed in velocity."""
    from pairs import perm_to_oracle, rel_err
    from oracle import ek_oracle as O
    ek = gpu_lib
    ws = workloads.batch_ensemble(3, seed=82, edges=(32, 48), radius=(2.5, 4.0),
                                  charge=(-30.0, -10.0), bulk=(1e-3, 1e-2))
    pairs = _oracle_members(ek, ws, ek.EK_PV | ek.EK_NEUTRALIZE | FP32)
    b = ek.EKBatch([s for _, s in pairs])
    b.set_config(fused=form)
    assert b.config()["fused"] == form
    b.step(3)
    b.step(4)
    perm = perm_to_oracle(ek)
    for i, (o, s) in enumerate(pairs):
        o.step(7)
        assert np.array_equal(s.get_fields(ek.FIELD_OWNER), o.owner.astype(float)), i
        fluid = o.owner == O.FLUID
        for k in range(o.K):
            assert rel_err(s.get_fields(ek.FIELD_SPECIES, k), o.rho[k]) < 2e-4, (i, k)
        fg = s.get_fields(ek.FIELD_POPULATIONS)[perm]
        assert rel_err(fg[:, fluid], o.f[:, fluid]) < 1e-5, i
        assert rel_err(s.get_fields(ek.FIELD_PHI), o.phi) < 2e-4, i
        assert rel_err(s.get_fields(ek.FIELD_PSI), o.psi) == 0.0, i
        p = s.get_particles()[0]
        assert np.max(np.abs(p["pos"] - o.particles[0].pos)) < 1e-6, i
        vmax = np.max(np.abs(o.particles[0].vel))
        assert np.max(np.abs(p["vel"] - o.particles[0].vel)) < 2e-3 * vmax, i
    b.close()
