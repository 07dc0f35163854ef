"""A step on a caller-provided stream is captured once per ping-pong parity as
a CUDA graph and replayed; the replay must give what the same kernels give
launched one by one on the default stream, also after E changes (the captured
launch arguments are rebuilt) and after the stream changes."""
import numpy as np
import pytest

import workloads
from oracle import ek_oracle as O
from pairs import make_pair

pytestmark = pytest.mark.gpu

FP32 = 16


def snapshot(ek, s, K):
    out = {"owner": s.get_fields(ek.FIELD_OWNER), "phi": s.get_fields(ek.FIELD_PHI),
           "f": s.get_fields(ek.FIELD_POPULATIONS), "psi": s.get_fields(ek.FIELD_PSI)}
    for k in range(K):
        out["rho%d" % k] = s.get_fields(ek.FIELD_SPECIES, k)
    for j, p in enumerate(s.get_particles()):
        for key in ("pos", "vel", "omega", "force"):
            out["p%d_%s" % (j, key)] = np.array(p[key], dtype=np.float64)
    return out


def same(a, b, rtol):
    for key in a:
        x, y = a[key], b[key]
        scale = max(np.max(np.abs(y)), 1e-300)
        assert np.max(np.abs(x - y)) <= rtol * scale, key


@pytest.mark.parametrize("flags", [O.PV | O.NEUTRALIZE, O.PV | O.NEUTRALIZE | FP32])
def test_graph_replay_matches_direct_launches(gpu_lib, flags):
    import torch
    ek = gpu_lib
    case = workloads.small_case(n=(24, 18, 16), radius=3.0, charge=-20.0, nparticles=2)
    vel = [(0.03, -0.01, 0.01), (-0.02, 0.015, 0.0)]
    _, direct = make_pair(ek, case, flags=flags, vel=vel)
    _, graphed = make_pair(ek, case, flags=flags, vel=vel)
    stream = torch.cuda.Stream()
    graphed.set_stream(stream)
    # odd counts so that both parities are captured and replayed
    for n in (3, 4):
        direct.step(n)
        graphed.step(n)
    E2 = np.array([0.0, 0.02, -0.01])
    direct.set_field(ek.FIELD_E_EXT, E2)
    graphed.set_field(ek.FIELD_E_EXT, E2)
    direct.step(5)
    graphed.step(5)
    other = torch.cuda.Stream()
    graphed.set_stream(other)
    direct.step(2)
    graphed.step(2)
    assert graphed.kernel_launches() == direct.kernel_launches()
    a = snapshot(ek, graphed, len(case["valence"]))
    b = snapshot(ek, direct, len(case["valence"]))
    assert np.array_equal(a["owner"], b["owner"])
    same(a, b, 1e-12)


def test_async_particle_records_match(gpu_lib):
    """ek_get_particles_async (packed on the device, copied into pinned host
    memory on the stream) gives the records ek_get_particles gives."""
    import ctypes
    import torch
    ek = gpu_lib
    case = workloads.small_case(n=(24, 18, 16), radius=3.0, charge=-20.0, nparticles=2)
    _, s = make_pair(ek, case, flags=O.PV | O.NEUTRALIZE | FP32, vel=[(0.03, 0.0, 0.0), (0.0, -0.02, 0.0)])
    stream = torch.cuda.Stream()
    s.set_stream(stream)
    n = s.num_particles()
    buf = torch.zeros(n * ctypes.sizeof(ek.ParticleRec), dtype=torch.uint8).pin_memory()
    for _ in range(2):
        s.step_async(3)
        s.get_particles_async(buf)
        stream.synchronize()
        got = ek.particles_from_buffer(buf, n)
        want = s.get_particles()
        for g, w in zip(got, want):
            for key in ("pos", "vel", "omega", "force", "torque"):
                assert np.array_equal(g[key], w[key]), key
            assert g["radius"] == w["radius"] and g["charge"] == w["charge"] and g["fixed"] == w["fixed"]

