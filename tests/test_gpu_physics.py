"""Closed-form physics through the C ABI, both storage forms: the
Poisson-Boltzmann profile of counter-ions between two charged walls."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FP32 = 16


@pytest.mark.parametrize("fp32", [False, True])
def test_poisson_boltzmann_slit(gpu_lib, fp32):
    """Counter-ions only (z = +1) between walls of charge density -sigma:
    rho(z) = rho_m / cos^2(alpha (z - z_c)), alpha^2 = 2 pi l_B rho_m,
    sigma = (rho_m / alpha) tan(alpha d), fluid cells filling
    [z_c - d, z_c + d] (the oracle's pin of the same closed form agrees to
    0.2%)."""
    ek = gpu_lib
    nx = ny = 8
    nz = 36                      # walls at z = 0 and 35, fluid cells 1..34: d = 17
    lB, d = 0.7, 17.0
    alpha = 1.0 / 17.0
    rho_m = alpha ** 2 / (2.0 * math.pi * lB)
    sigma = rho_m * math.tan(alpha * d) / alpha
    flags = ek.EK_NEUTRALIZE | (FP32 if fp32 else 0)
    s = ek.EKSystem((nx, ny, nz), bjerrum=lB, valence=(1,), D=(0.3,), bulk=(0.0,), flags=flags)
    walls = np.zeros((nz, ny, nx))
    walls[0] = walls[nz - 1] = 1.0
    s.set_field(ek.FIELD_WALL_CHARGE, np.where(walls > 0, -sigma, 0.0).ravel())
    s.set_field(ek.FIELD_WALL, walls.ravel())
    total0 = s.get_fields(ek.FIELD_SPECIES, 0).sum()
    s.step(2000)
    rho = s.get_fields(ek.FIELD_SPECIES, 0).reshape(nz, ny, nx)[1:nz - 1]
    z = np.arange(1, nz - 1) - 0.5 * (nz - 1)
    expect = rho_m / np.cos(alpha * z) ** 2
    prof = rho.mean(axis=(1, 2))
    # laterally uniform (the FP32 form's float FFT leaves rounding noise of a few units)
    assert np.max(np.abs(rho - prof[:, None, None])) <= (1e-4 if fp32 else 1e-10) * prof.max()
    assert np.max(np.abs(prof / expect - 1.0)) < 0.01
    # the ions stay in the box: exact in the FP32 form's integer units
    total = s.get_fields(ek.FIELD_SPECIES, 0).sum()
    if fp32:
        assert total == total0
    else:
        assert abs(total - total0) <= 1e-12 * total0
