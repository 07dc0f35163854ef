"""Checkpoint and resume through the C ABI (ek_get_state / ek_set_state): a
system restored from a checkpoint, into a fresh context or into the same one
later, continues as the checkpointed system continued (species and node
owners bit for bit, the rest to the rounding of the FP64 form's atomic
transfer sums); a checkpoint of another system, or a damaged one, is refused."""
import numpy as np
import pytest

import workloads
from oracle import ek_oracle as O
from pairs import make_pair

pytestmark = pytest.mark.gpu

FP32 = 16
ERR_ARG, ERR_STATE = -1, -8


def snapshot(ek, s, K):
    out = {"owner": s.get_fields(ek.FIELD_OWNER), "phi": s.get_fields(ek.FIELD_PHI),
           "f": s.get_fields(ek.FIELD_POPULATIONS), "psi": s.get_fields(ek.FIELD_PSI),
           "u": s.get_fields(ek.FIELD_VELOCITY)}
    for k in range(K):
        out["rho%d" % k] = s.get_fields(ek.FIELD_SPECIES, k)
    for j, p in enumerate(s.get_particles()):
        for key in ("pos", "vel", "omega", "force", "torque"):
            out["p%d_%s" % (j, key)] = np.array(p[key], dtype=np.float64)
    return out


def same(a, b, exact_species):
    assert np.array_equal(a["owner"], b["owner"])
    for key in a:
        if exact_species and key.startswith("rho"):
            assert np.array_equal(a[key], b[key]), key
        scale = max(np.max(np.abs(b[key])), 1e-300)
        assert np.max(np.abs(a[key] - b[key])) <= 1e-12 * scale, key


@pytest.mark.parametrize("flags", [O.PV | O.NEUTRALIZE, O.PV | O.NEUTRALIZE | FP32])
def test_resume_continues_the_checkpointed_run(gpu_lib, flags):
    import torch
    ek = gpu_lib
    case = workloads.small_case(n=(24, 18, 16), radius=3.0, charge=-20.0, nparticles=2)
    vel = [(0.03, -0.01, 0.01), (-0.02, 0.015, 0.0)]
    K = len(case["valence"])
    E2 = np.array([0.0, 0.02, -0.01])
    _, a = make_pair(ek, case, flags=flags, vel=vel)
    a.step(5)
    ck = a.get_state()
    a.set_field(ek.FIELD_E_EXT, E2)
    a.step(7)
    want = snapshot(ek, a, K)
    # a fresh context with the same set-up, stepping through replayed graphs
    _, b = make_pair(ek, case, flags=flags, vel=vel)
    b.set_stream(torch.cuda.Stream())
    b.step(2)  # a different state (and captured steps) before the restore
    b.set_state(ck)
    b.set_field(ek.FIELD_E_EXT, E2)
    b.step(3)
    b.step(4)
    same(snapshot(ek, b, K), want, flags & FP32)
    # the checkpointed context itself, rewound
    a.set_state(ck)
    a.set_field(ek.FIELD_E_EXT, E2)
    a.step(7)
    same(snapshot(ek, a, K), want, flags & FP32)
    # the checkpoint carries E: without the change the runs part
    b.set_state(ck)
    b.step(7)
    assert not np.array_equal(snapshot(ek, b, K)["p0_pos"], want["p0_pos"])


def test_checkpoint_of_another_system_is_refused(gpu_lib):
    ek = gpu_lib
    case = workloads.small_case(n=(24, 18, 16), radius=3.0, charge=-20.0, nparticles=2)
    _, a = make_pair(ek, case, flags=O.PV | O.NEUTRALIZE | FP32)
    ck = a.get_state()
    # the size query agrees with the checkpoint
    assert ck.size > 19 * 24 * 18 * 16 * 4
    # another shape, another storage form, another particle count
    other = dict(case, shape=(24, 18, 32))
    _, b = make_pair(ek, other, flags=O.PV | O.NEUTRALIZE | FP32)
    _, c = make_pair(ek, case, flags=O.PV | O.NEUTRALIZE)
    one = dict(case, particles=case["particles"][:1])
    _, d = make_pair(ek, one, flags=O.PV | O.NEUTRALIZE | FP32)
    for s in (b, c, d):
        with pytest.raises(ek.EKError) as e:
            s.set_state(ck)
        assert e.value.code == ERR_STATE
    # truncated or not a checkpoint
    with pytest.raises(ek.EKError) as e:
        a.set_state(ck[:-1])
    assert e.value.code == ERR_ARG
    with pytest.raises(ek.EKError) as e:
        a.set_state(np.zeros(ck.size, dtype=np.uint8))
    assert e.value.code == ERR_ARG
    # the refusals left the system usable and unchanged
    a.set_state(ck)
    a.step(2)
