"""Python binding of the C ABI in include/ek.h (libek.so): argument marshalling only.

Every step of the time step runs in the CUDA library; this module converts
numpy arrays and torch tensors to pointers and status codes to exceptions.
There is no CPU fallback: if libek.so is missing or cannot be loaded, every
call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libek.so")

EK_MAX_SPECIES = 4

# ek_params.flags
EK_PV = 1
EK_VACATE_ZERO = 2
EK_CHARGE_NORM_VP = 4
EK_NEUTRALIZE = 8
EK_FP32 = 16

# ek_field
FIELD_SPECIES = 0
FIELD_POPULATIONS = 1
FIELD_VELOCITY = 2
FIELD_E_EXT = 3
FIELD_BODY_FORCE = 4
FIELD_WALL = 5
FIELD_WALL_CHARGE = 6
FIELD_DENSITY = 7
FIELD_PHI = 8
FIELD_PSI = 9
FIELD_OWNER = 10
FIELD_CHARGE = 11

STATUS = {0: "EK_OK", -1: "EK_ERR_ARG", -2: "EK_ERR_NOMEM", -3: "EK_ERR_CUDA",
          -4: "EK_ERR_UNSTABLE", -5: "EK_ERR_OVERLAP", -6: "EK_ERR_EXPEL", -7: "EK_ERR_TIMEOUT",
          -8: "EK_ERR_STATE"}

# entry points declared in include/ek.h
EXPORTS = ["ek_create", "ek_destroy", "ek_add_particle", "ek_set_field", "ek_get_fields",
           "ek_step", "ek_step_async", "ek_run_stage", "ek_get_particles", "ek_get_particles_async",
           "ek_num_particles", "ek_get_state", "ek_set_state",
           "ek_set_stream", "ek_sync", "ek_last_error", "ek_lattice_dirs",
           "ek_poisson_scratch_bytes", "ek_poisson_solve", "ek_step_timed",
           "ek_kernel_launches", "ek_poisson_solve_static", "ek_poisson_mg_scratch_bytes",
           "ek_poisson_solve_mg", "ek_poisson_cg_scratch_bytes", "ek_poisson_solve_cg",
           "ek_batch_create", "ek_batch_destroy", "ek_batch_set_stream", "ek_batch_step_async",
           "ek_batch_step", "ek_batch_sync", "ek_batch_tune", "ek_batch_config", "ek_batch_set_config",
           "ek_batch_wait_test", "ek_batch_size", "ek_debug_fail_alloc",
           "ek_batch_last_error"]


class EKError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__(f"{STATUS.get(code, code)}: {msg}")


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("nu", ctypes.c_double), ("rho0", ctypes.c_double), ("bjerrum", ctypes.c_double),
                ("magic", ctypes.c_double), ("nspecies", ctypes.c_int),
                ("valence", ctypes.c_int * EK_MAX_SPECIES),
                ("D", ctypes.c_double * EK_MAX_SPECIES),
                ("bulk", ctypes.c_double * EK_MAX_SPECIES),
                ("flags", ctypes.c_uint)]


class ParticleRec(ctypes.Structure):
    _fields_ = [("pos", ctypes.c_double * 3), ("vel", ctypes.c_double * 3),
                ("omega", ctypes.c_double * 3), ("force", ctypes.c_double * 3),
                ("torque", ctypes.c_double * 3), ("radius", ctypes.c_double),
                ("charge", ctypes.c_double), ("rho_p", ctypes.c_double), ("fixed", ctypes.c_int)]


_lib = None


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libek.so (building it first if the CUDA toolkit is present)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        from . import build as _build
        path = _build.build()
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.ek_create.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(vp)]
    lib.ek_destroy.argtypes = [vp]
    lib.ek_add_particle.argtypes = [vp, ctypes.POINTER(dp), ctypes.POINTER(dp), ctypes.POINTER(dp),
                                    dp, dp, dp, ip, ctypes.POINTER(ip)]
    lib.ek_set_field.argtypes = [vp, ip, ip, vp, ctypes.c_size_t, ip]
    lib.ek_get_fields.argtypes = [vp, ip, ip, vp, ctypes.c_size_t, ip]
    lib.ek_step.argtypes = [vp, ip]
    lib.ek_step_async.argtypes = [vp, ip]
    lib.ek_run_stage.argtypes = [vp, ip]
    lib.ek_get_particles.argtypes = [vp, ctypes.POINTER(ParticleRec), ip]
    lib.ek_get_particles_async.argtypes = [vp, vp, ip]
    lib.ek_num_particles.argtypes = [vp]
    lib.ek_num_particles.restype = ip
    lib.ek_get_state.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t)]
    lib.ek_set_state.argtypes = [vp, vp, ctypes.c_size_t]
    lib.ek_set_stream.argtypes = [vp, vp]
    lib.ek_sync.argtypes = [vp]
    lib.ek_last_error.argtypes = [vp]
    lib.ek_last_error.restype = ctypes.c_char_p
    lib.ek_lattice_dirs.argtypes = [ctypes.POINTER(ip)]
    lib.ek_lattice_dirs.restype = None
    lib.ek_poisson_scratch_bytes.argtypes = [ip, ip, ip]
    lib.ek_poisson_scratch_bytes.restype = ctypes.c_size_t
    lib.ek_poisson_solve.argtypes = [vp, vp, ip, ip, ip, dp, vp, vp]
    lib.ek_step_timed.argtypes = [vp, ip, ctypes.POINTER(dp)]
    lib.ek_poisson_solve_static.argtypes = [vp, vp, ip, ip, ip, dp, vp]
    lib.ek_poisson_mg_scratch_bytes.argtypes = [ip, ip, ip]
    lib.ek_poisson_mg_scratch_bytes.restype = ctypes.c_size_t
    lib.ek_poisson_solve_mg.argtypes = [vp, vp, ip, ip, ip, dp, dp, ip, vp, vp,
                                        ctypes.POINTER(ip), ctypes.POINTER(dp)]
    lib.ek_poisson_cg_scratch_bytes.argtypes = [ip, ip, ip]
    lib.ek_poisson_cg_scratch_bytes.restype = ctypes.c_size_t
    lib.ek_poisson_solve_cg.argtypes = [vp, vp, vp, vp, vp, ip, ip, ip, dp, dp, ip, vp, vp,
                                        ctypes.POINTER(ip), ctypes.POINTER(dp)]
    lib.ek_kernel_launches.argtypes = [vp]
    lib.ek_kernel_launches.restype = ctypes.c_longlong
    lib.ek_batch_create.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(vp)]
    lib.ek_batch_destroy.argtypes = [vp]
    lib.ek_batch_set_stream.argtypes = [vp, vp]
    lib.ek_batch_step_async.argtypes = [vp, ip]
    lib.ek_batch_step.argtypes = [vp, ip]
    lib.ek_batch_sync.argtypes = [vp]
    lib.ek_batch_tune.argtypes = [vp, ip, ctypes.POINTER(dp)]
    lib.ek_batch_config.argtypes = [vp, ctypes.POINTER(ip)]
    lib.ek_batch_set_config.argtypes = [vp, ctypes.POINTER(ip)]
    lib.ek_batch_wait_test.argtypes = [vp, ip, dp]
    lib.ek_debug_fail_alloc.argtypes = [ip]
    lib.ek_debug_fail_alloc.restype = None
    lib.ek_batch_size.argtypes = [vp]
    lib.ek_batch_size.restype = ip
    lib.ek_batch_last_error.argtypes = [vp]
    lib.ek_batch_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("ek_num_particles", "ek_last_error", "ek_lattice_dirs",
                        "ek_poisson_scratch_bytes", "ek_kernel_launches", "ek_batch_size",
                        "ek_poisson_mg_scratch_bytes", "ek_debug_fail_alloc",
                        "ek_poisson_cg_scratch_bytes",
                        "ek_batch_last_error"):
            getattr(lib, name).restype = ip
    _lib = lib
    return lib


def debug_fail_alloc(n: int) -> None:
    """Test hook: the n-th field allocation of ek_create from now on fails (see
    ek_debug_fail_alloc in include/ek.h); n <= 0 clears it."""
    load_library().ek_debug_fail_alloc(int(n))


def lattice_dirs() -> np.ndarray:
    """The (19, 3) D3Q19 velocity set in the library's population order."""
    lib = load_library()
    c = (ctypes.c_int * 57)()
    lib.ek_lattice_dirs(c)
    return np.array(list(c), dtype=np.int64).reshape(19, 3)


def _buf(values, on_device_ok=True):
    """(pointer, count, on_device, keepalive) of a numpy array or torch tensor."""
    try:
        import torch
        if isinstance(values, torch.Tensor):
            if values.dtype != torch.float64 or not values.is_contiguous():
                raise TypeError("torch tensors must be contiguous float64")
            return values.data_ptr(), values.numel(), int(values.is_cuda), values
    except ImportError:
        pass
    arr = np.ascontiguousarray(values, dtype=np.float64)
    return arr.ctypes.data, arr.size, 0, arr


class EKSystem:
    """One electrokinetic box on the GPU (an ek_ctx)."""

    def __init__(self, shape, nu=1.0 / 6.0, rho0=1.0, bjerrum=0.7, valence=(1, -1),
                 D=(0.3, 0.3), bulk=(1e-3, 1e-3), flags=EK_PV | EK_NEUTRALIZE, magic=0.0):
        self.lib = load_library()
        p = Params()
        p.nx, p.ny, p.nz = (int(v) for v in shape)
        p.nu, p.rho0, p.bjerrum = float(nu), float(rho0), float(bjerrum)
        p.magic = float(magic or 0.0)
        K = len(valence)
        p.nspecies = K
        for k in range(K):
            p.valence[k] = int(valence[k])
            p.D[k] = float(D[k])
            p.bulk[k] = float(bulk[k])
        p.flags = int(flags)
        self.params = p
        self.shape = (p.nx, p.ny, p.nz)
        self.N = p.nx * p.ny * p.nz
        self.K = K
        self.ctx = ctypes.c_void_p()
        st = self.lib.ek_create(ctypes.byref(p), ctypes.byref(self.ctx))
        if st != 0:
            raise EKError(st, "ek_create failed")

    # -- helpers ---------------------------------------------------------------
    def _check(self, st):
        if st != 0:
            raise EKError(st, self.lib.ek_last_error(self.ctx).decode())

    def close(self):
        if self.ctx:
            self.lib.ek_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def field_size(self, which):
        if which == FIELD_POPULATIONS:
            return 19 * self.N
        if which == FIELD_VELOCITY:
            return 3 * self.N
        if which in (FIELD_E_EXT, FIELD_BODY_FORCE):
            return 3
        return self.N

    # -- ABI calls ---------------------------------------------------------------
    def add_particle(self, pos, vel=(0, 0, 0), radius=4.0, charge=0.0, rho_p=2.0, fixed=False,
                     omega=(0, 0, 0)):
        D3 = ctypes.c_double * 3
        out = ctypes.c_int(-1)
        self._check(self.lib.ek_add_particle(self.ctx, D3(*pos), D3(*vel), D3(*omega),
                                             float(radius), float(charge), float(rho_p),
                                             int(bool(fixed)), ctypes.byref(out)))
        return out.value

    def set_field(self, which, values, component=0):
        ptr, n, dev, keep = _buf(values)
        self._check(self.lib.ek_set_field(self.ctx, which, component, ctypes.c_void_p(ptr), n, dev))
        del keep

    def get_fields(self, which, component=0, out=None):
        """Read a field; returns a numpy array shaped like the field, or fills
        `out` (numpy array or torch tensor, host or device)."""
        n = self.field_size(which)
        if out is None:
            arr = np.empty(n, dtype=np.float64)
            self._check(self.lib.ek_get_fields(self.ctx, which, component,
                                               ctypes.c_void_p(arr.ctypes.data), n, 0))
            nx, ny, nz = self.shape
            if n == 3:
                return arr
            if n == self.N:
                return arr.reshape(nz, ny, nx)
            return arr.reshape(n // self.N, nz, ny, nx)
        ptr, cnt, dev, keep = _buf(out)
        if cnt != n:
            raise ValueError("output size does not match the field")
        self._check(self.lib.ek_get_fields(self.ctx, which, component, ctypes.c_void_p(ptr), n, dev))
        return out

    def step(self, n=1):
        self._check(self.lib.ek_step(self.ctx, int(n)))

    def step_async(self, n=1):
        self._check(self.lib.ek_step_async(self.ctx, int(n)))

    def step_timed(self, n=1):
        """Run n steps; returns device ms per stage: S1, S2 (fused LB kernel),
        S3 (advection), S4, S5, total."""
        acc = (ctypes.c_double * 6)()
        self._check(self.lib.ek_step_timed(self.ctx, int(n), acc))
        return list(acc)

    def kernel_launches(self):
        return int(self.lib.ek_kernel_launches(self.ctx))

    def run_stage(self, stage):
        self._check(self.lib.ek_run_stage(self.ctx, int(stage)))

    def sync(self):
        self._check(self.lib.ek_sync(self.ctx))

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an integer handle, or None."""
        h = 0
        if stream is not None:
            h = getattr(stream, "cuda_stream", stream)
        self._check(self.lib.ek_set_stream(self.ctx, ctypes.c_void_p(int(h))))

    def num_particles(self):
        return self.lib.ek_num_particles(self.ctx)

    def get_state(self) -> np.ndarray:
        """A checkpoint of the system (ek_get_state) as a uint8 array."""
        n = ctypes.c_size_t(0)
        self._check(self.lib.ek_get_state(self.ctx, None, ctypes.byref(n)))
        buf = np.empty(n.value, dtype=np.uint8)
        self._check(self.lib.ek_get_state(self.ctx, ctypes.c_void_p(buf.ctypes.data), ctypes.byref(n)))
        return buf

    def set_state(self, buf):
        """Restore a checkpoint from get_state (ek_set_state)."""
        b = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(self.lib.ek_set_state(self.ctx, ctypes.c_void_p(b.ctypes.data), b.nbytes))

    def get_particles_async(self, buf):
        """Enqueue a copy of the particle records into `buf`, a page-locked
        host (or device) buffer of at least num_particles() records, e.g.
        torch.empty(n * ctypes.sizeof(ParticleRec), dtype=torch.uint8).pin_memory();
        decode with particles_from_buffer once the stream has passed the call."""
        ptr = buf.data_ptr() if hasattr(buf, "data_ptr") else int(buf)
        self._check(self.lib.ek_get_particles_async(self.ctx, ctypes.c_void_p(ptr),
                                                     self.num_particles()))

    def get_particles(self):
        P = self.num_particles()
        recs = (ParticleRec * max(P, 1))()
        self._check(self.lib.ek_get_particles(self.ctx, recs, P))
        out = []
        for r in recs[:P]:
            out.append(dict(pos=np.array(r.pos[:]), vel=np.array(r.vel[:]),
                            omega=np.array(r.omega[:]), force=np.array(r.force[:]),
                            torque=np.array(r.torque[:]), radius=r.radius, charge=r.charge,
                            rho_p=r.rho_p, fixed=bool(r.fixed)))
        return out


def particles_from_buffer(buf, count):
    """Decode `count` ek_particle records from a host buffer (bytes-like, or a
    pinned torch uint8 tensor filled by EKSystem.get_particles_async)."""
    if count <= 0:
        return []
    raw = bytes(buf.numpy()) if hasattr(buf, "numpy") else bytes(buf)
    recs = (ParticleRec * count).from_buffer_copy(raw[:count * ctypes.sizeof(ParticleRec)])
    return [dict(pos=np.array(r.pos[:]), vel=np.array(r.vel[:]), omega=np.array(r.omega[:]),
                 force=np.array(r.force[:]), torque=np.array(r.torque[:]), radius=r.radius,
                 charge=r.charge, rho_p=r.rho_p, fixed=bool(r.fixed)) for r in recs[:count]]


def poisson_scratch_bytes(nx, ny, nz):
    return load_library().ek_poisson_scratch_bytes(nx, ny, nz)


def poisson_solve(q, phi, shape, bjerrum, spectrum, stream=None):
    """Standalone Poisson solve on device tensors (torch, float64): see ek.h."""
    lib = load_library()
    nx, ny, nz = shape
    h = 0 if stream is None else getattr(stream, "cuda_stream", stream)
    st = lib.ek_poisson_solve(ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(phi.data_ptr()),
                              nx, ny, nz, float(bjerrum), ctypes.c_void_p(spectrum.data_ptr()),
                              ctypes.c_void_p(int(h)))
    if st != 0:
        raise EKError(st, "ek_poisson_solve failed")


def poisson_mg_scratch_bytes(shape):
    return int(load_library().ek_poisson_mg_scratch_bytes(*(int(v) for v in shape)))


def poisson_solve_mg(q, phi, shape, bjerrum, scratch, tol=1e-12, max_cycles=50, stream=None):
    """Multigrid Poisson solve on device tensors (torch, float64; scratch a
    device tensor of at least poisson_mg_scratch_bytes(shape) bytes): see
    ek_poisson_solve_mg in include/ek.h.  Returns (V-cycles, relative residual)."""
    lib = load_library()
    nx, ny, nz = shape
    h = 0 if stream is None else getattr(stream, "cuda_stream", stream)
    cyc = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    st = lib.ek_poisson_solve_mg(ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(phi.data_ptr()),
                                 nx, ny, nz, float(bjerrum), float(tol), int(max_cycles),
                                 ctypes.c_void_p(scratch.data_ptr()), ctypes.c_void_p(int(h)),
                                 ctypes.byref(cyc), ctypes.byref(res))
    if st != 0:
        raise EKError(st, "ek_poisson_solve_mg failed")
    return cyc.value, res.value


def poisson_cg_scratch_bytes(shape):
    return int(load_library().ek_poisson_cg_scratch_bytes(*(int(v) for v in shape)))


def poisson_solve_cg(q, phi, shape, bjerrum, scratch, eps=None, fixed=None, phi_fixed=None,
                     tol=1e-12, max_iter=20000, stream=None):
    """Poisson solve with an inhomogeneous permittivity and fixed-potential
    nodes by conjugate gradients (see ek_poisson_solve_cg in include/ek.h).
    q, phi, eps, phi_fixed: float64 device tensors; fixed: uint8 device
    tensor; scratch: a device tensor of at least poisson_cg_scratch_bytes(shape)
    bytes.  Returns (iterations, relative residual)."""
    lib = load_library()
    nx, ny, nz = shape
    h = 0 if stream is None else getattr(stream, "cuda_stream", stream)
    ptr = (lambda t: ctypes.c_void_p(None) if t is None else ctypes.c_void_p(t.data_ptr()))
    it = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    st = lib.ek_poisson_solve_cg(ptr(q), ptr(eps), ptr(fixed), ptr(phi_fixed), ptr(phi), nx, ny, nz,
                                 float(bjerrum), float(tol), int(max_iter), ptr(scratch),
                                 ctypes.c_void_p(int(h)), ctypes.byref(it), ctypes.byref(res))
    if st != 0:
        raise EKError(st, "ek_poisson_solve_cg failed")
    return it.value, res.value


POISSON_STATIC_MAX = 1 << 19  # complex doubles of the fixed scratch of ek_poisson_solve_static


def poisson_solve_static(q, phi, shape, bjerrum, stream=None):
    """Poisson solve that allocates no device memory (see ek_poisson_solve_static
    in include/ek.h): for callers that cannot call cudaMalloc.  q and phi are
    float64 device tensors; calls that overlap on the GPU race."""
    lib = load_library()
    nx, ny, nz = shape
    h = 0 if stream is None else getattr(stream, "cuda_stream", stream)
    st = lib.ek_poisson_solve_static(ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(phi.data_ptr()),
                                     nx, ny, nz, float(bjerrum), ctypes.c_void_p(int(h)))
    if st != 0:
        raise EKError(st, "ek_poisson_solve_static failed (box too large for the fixed scratch?)")


class EKBatch:
    """Many EKSystem objects advanced together, one CUDA graph launch per step
    of all of them (see ek_batch_* in include/ek.h).  The systems must outlive
    the batch; call sync() before reading a system or stepping it alone."""

    def __init__(self, systems):
        self.lib = load_library()
        self.systems = list(systems)
        arr = (ctypes.c_void_p * len(self.systems))(*[s.ctx.value for s in self.systems])
        self.ptr = ctypes.c_void_p()
        st = self.lib.ek_batch_create(arr, len(self.systems), ctypes.byref(self.ptr))
        if st != 0:
            raise EKError(st, "ek_batch_create failed")

    def _check(self, st):
        if st != 0:
            raise EKError(st, self.lib.ek_batch_last_error(self.ptr).decode())

    def step(self, n=1):
        self._check(self.lib.ek_batch_step(self.ptr, int(n)))

    def step_async(self, n=1):
        self._check(self.lib.ek_batch_step_async(self.ptr, int(n)))

    def sync(self):
        self._check(self.lib.ek_batch_sync(self.ptr))

    def set_stream(self, stream):
        h = getattr(stream, "cuda_stream", stream)
        self._check(self.lib.ek_batch_set_stream(self.ptr, ctypes.c_void_p(int(h))))

    def tune(self, trial_steps=2):
        """Run the autotuner; returns (config dict, ms per batch step)."""
        best = ctypes.c_double(0.0)
        self._check(self.lib.ek_batch_tune(self.ptr, int(trial_steps), ctypes.byref(best)))
        return self.config(), best.value

    def config(self):
        cfg = (ctypes.c_int * 4)()
        self._check(self.lib.ek_batch_config(self.ptr, cfg))
        return {"branches": cfg[0], "planes_per_block": cfg[1], "particle_chain_beside_s3": bool(cfg[2]),
                "fused": cfg[3]}

    def set_config(self, branches=None, planes_per_block=None, particle_chain_beside_s3=None, fused=None):
        """Change part of the configuration (the rest stays as it is)."""
        c = self.config()
        vals = [c["branches"] if branches is None else branches,
                c["planes_per_block"] if planes_per_block is None else planes_per_block,
                int(c["particle_chain_beside_s3"] if particle_chain_beside_s3 is None else particle_chain_beside_s3),
                int(c["fused"] if fused is None else fused)]
        cfg = (ctypes.c_int * 4)(*vals)
        self._check(self.lib.ek_batch_set_config(self.ptr, cfg))

    def wait_test(self, leave_cta=-1, limit_ms=1000.0):
        """Failure-detection hook of the persistent particle chain (form 2):
        one CTA leaves before the first grid barrier, the waits give up after
        limit_ms (see ek_batch_wait_test in include/ek.h)."""
        self._check(self.lib.ek_batch_wait_test(self.ptr, int(leave_cta), float(limit_ms)))

    def __len__(self):
        return self.lib.ek_batch_size(self.ptr)

    def close(self):
        if self.ptr:
            self.lib.ek_batch_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
