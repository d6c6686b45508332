"""Python binding of the GB300 Yee + embedded-ROM library (``libfdtdrom.so``).

Argument marshalling only: every step of the time-marching path runs in the
library's CUDA kernels, and the one-time reduced-model build runs in its FP64
host code.  There is no fallback: if the shared library is missing, importing
the functions raises.  Build it with ``paper_1609_07114_gb300.build.build()``.

Names follow the C ABI in include/fdtd.h.  PyTorch is used only to hand over
device buffers (``tensor.data_ptr()``) and the current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfdtdrom.so")

FDTD_OK = 0
ERRORS = {-1: "FDTD_EINVAL", -2: "FDTD_ENOMEM", -3: "FDTD_ECFL", -4: "FDTD_ENOTPASSIVE",
          -5: "FDTD_ESINGULAR", -6: "FDTD_EUNSTABLE", -7: "FDTD_ETIMEOUT", -8: "FDTD_ECUDA"}
FDTD_RULE_DUAL = 0
FDTD_RULE_PAPER = 1
FDTD_SRC_JX = 0
FDTD_SRC_JY = 1
FDTD_ENERGY_STATIC_MAX = 32768   # capacity of fdtd_energy_noalloc (include/fdtd.h)

_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)


class fdtd_sim_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("eps_r", _dp), ("sigma", _dp)]


class fdtd_grid_desc(C.Structure):
    _fields_ = [("dx", C.c_double), ("dy", C.c_double), ("dt", C.c_double),
                ("nsim", C.c_int), ("sims", C.POINTER(fdtd_sim_desc))]


class rom_desc(C.Structure):
    _fields_ = [("a", C.c_int), ("b", C.c_int), ("r", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dt", C.c_double),
                ("eps_r", _dp), ("sigma", _dp), ("q", C.c_int), ("rule", C.c_int),
                ("f0", C.c_double), ("gamma", C.c_double), ("defl_tol", C.c_double)]


class rom_build_report(C.Structure):
    _fields_ = [("qE", C.c_int), ("qH", C.c_int), ("n_inputs", C.c_int), ("n_clamped", C.c_int),
                ("smax_before", C.c_double), ("smax_after", C.c_double),
                ("min_eig_R", C.c_double), ("cond3_residual", C.c_double),
                ("seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fdtd_pml_desc(C.Structure):
    _fields_ = [("sides", C.c_int), ("ncells", C.c_int), ("m", C.c_double), ("sigma_max", C.c_double),
                ("kappa_max", C.c_double), ("alpha_max", C.c_double)]


FDTD_PML_W, FDTD_PML_E, FDTD_PML_S, FDTD_PML_N = 1, 2, 4, 8


class fdtd_tune_report(C.Structure):
    _fields_ = [("steps_per_launch", C.c_int), ("tile_rows", C.c_int), ("march_rows", C.c_int),
                ("march_ring", C.c_int), ("march_prefetch", C.c_int),
                ("gemm_min", C.c_int), ("gemm_rows_per_warp", C.c_int), ("chain", C.c_int),
                ("chained_models", C.c_int), ("candidates", C.c_int), ("ms_default", C.c_double),
                ("ms_best", C.c_double), ("march_ctas", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fdtd_source(C.Structure):
    _fields_ = [("sim", C.c_int), ("comp", C.c_int), ("i", C.c_int), ("j", C.c_int),
                ("len", C.c_int), ("wave", _fp)]


class fdtd_probe(C.Structure):
    _fields_ = [("sim", C.c_int), ("i", C.c_int), ("j", C.c_int)]


_lib = None


def lib() -> C.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} not found: build it with paper_1609_07114_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, i, d, ll = C.c_void_p, C.c_int, C.c_double, C.c_longlong
    sig = {
        "fdtd_create": (i, [C.POINTER(fdtd_grid_desc), vp, C.POINTER(vp)]),
        "fdtd_destroy": (None, [vp]),
        "fdtd_cfl_limit": (i, [d, d, _dp]),
        "rom_build": (i, [C.POINTER(rom_desc), C.POINTER(vp), C.POINTER(rom_build_report)]),
        "rom_build_gpu": (i, [C.POINTER(rom_desc), vp, C.POINTER(vp), C.POINTER(rom_build_report)]),
        "rom_free": (None, [vp]),
        "rom_get_info": (i, [vp, C.POINTER(i), C.POINTER(i), C.POINTER(i)]),
        "rom_get_blocks": (i, [vp, _dp, _dp, _dp, _dp, _dp]),
        "rom_embed": (i, [vp, vp, i, i, i, C.POINTER(i)]),
        "rom_couple": (i, [vp, _dp, _dp, _dp, _dp]),
        "fdtd_get_rom_map": (i, [vp, i, C.POINTER(i), C.POINTER(i), _dp, _dp]),
        "fdtd_run": (i, [vp, ll, C.POINTER(fdtd_source), i, C.POINTER(fdtd_probe), i, vp]),
        "fdtd_run_host": (i, [vp, ll, C.POINTER(fdtd_source), i, C.POINTER(fdtd_probe), i, _fp]),
        "fdtd_get_fields": (i, [vp, i, _fp, _fp, _fp]),
        "fdtd_set_fields": (i, [vp, i, _fp, _fp, _fp]),
        "fdtd_get_rom_state": (i, [vp, i, _fp]),
        "fdtd_set_rom_state": (i, [vp, i, _fp]),
        "fdtd_get_step": (i, [vp, C.POINTER(ll)]),
        "fdtd_save_state": (i, [vp, vp, C.POINTER(C.c_size_t)]),
        "fdtd_load_state": (i, [vp, vp, C.c_size_t]),
        "fdtd_energy": (i, [vp, _dp]),
        "fdtd_grad": (i, [vp, ll, C.POINTER(fdtd_source), i, C.POINTER(fdtd_probe), i, i,
                          vp, vp, vp, _dp]),
        "fdtd_energy_noalloc": (i, [vp, _dp]),
        "fdtd_vjp": (i, [vp, ll, C.POINTER(fdtd_source), i, C.POINTER(fdtd_probe), i, i,
                         vp, vp, vp, vp, vp]),
        "fdtd_dft_set": (i, [vp, C.POINTER(fdtd_probe), i, _dp, i, _dp]),
        "fdtd_dft_get": (i, [vp, _dp]),
        "fdtd_fine_fields": (i, [vp, i, vp, vp, vp, vp]),
        "fdtd_set_pml": (i, [vp, i, C.POINTER(fdtd_pml_desc)]),
        "fdtd_selftest_timeout": (i, [vp]),
        "rom_get_basis": (i, [vp, C.POINTER(i), C.POINTER(i), _dp, _dp]),
        "fdtd_set_timing": (i, [vp, i]),
        "fdtd_get_kernel_times": (i, [vp, _dp, C.POINTER(ll), _dp, C.POINTER(ll)]),
        "fdtd_steps_per_launch": (i, [vp]),
        "fdtd_time_stencil": (i, [vp, i, i, _dp]),
        "fdtd_autotune": (i, [vp, C.c_char_p, C.POINTER(fdtd_tune_report)]),
        "fdtd_get_plan": (i, [vp, C.POINTER(fdtd_tune_report)]),
        "fdtd_last_error": (C.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class FdtdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def _check(rc, ctx=None):
    if rc != FDTD_OK:
        msg = lib().fdtd_last_error(ctx)
        raise FdtdError(rc, msg.decode() if msg else "")


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def fdtd_cfl_limit(dx: float, dy: float) -> float:
    out = C.c_double()
    _check(lib().fdtd_cfl_limit(dx, dy, C.byref(out)))
    return out.value


class RomModel:
    """A reduced model built on the host in FP64 (``rom_build``)."""

    def __init__(self, handle, report, a, b, r):
        self._h = handle
        self.report = report
        self.a, self.b, self.r = a, b, r
        qE, qH, nu = C.c_int(), C.c_int(), C.c_int()
        _check(lib().rom_get_info(self._h, C.byref(qE), C.byref(qH), C.byref(nu)))
        self.qE, self.qH, self.nu = qE.value, qH.value, nu.value

    @property
    def q(self):
        return self.qE + self.qH

    def blocks(self):
        """R11, R22, Kt, Sig, LE (FP64, Eq. (12) blocks)."""
        qE, qH, nu = self.qE, self.qH, self.nu
        R11, R22 = np.zeros((qE, qE)), np.zeros((qH, qH))
        Kt, Sig, LE = np.zeros((qE, qH)), np.zeros((qE, qE)), np.zeros((qE, nu))
        ptr = lambda a: a.ctypes.data_as(_dp)
        _check(lib().rom_get_blocks(self._h, ptr(R11), ptr(R22), ptr(Kt), ptr(Sig), ptr(LE)))
        return R11, R22, Kt, Sig, LE

    def basis(self):
        """(V1, V2): the projection bases (``rom_get_basis``), FP64."""
        nE, nH = C.c_int(), C.c_int()
        _check(lib().rom_get_basis(self._h, C.byref(nE), C.byref(nH), None, None))
        V1, V2 = np.zeros((nE.value, self.qE)), np.zeros((nH.value, self.qH))
        _check(lib().rom_get_basis(self._h, None, None, V1.ctypes.data_as(_dp), V2.ctypes.data_as(_dp)))
        return V1, V2

    def couple(self, ring_eps_r, ring_sigma):
        """Host-only run-time map (P, Q) of Eq. (23) for the given outside
        half-cell materials (``rom_couple``)."""
        ny = 2 * (self.a + self.b)
        e, s = _f64(ring_eps_r), _f64(ring_sigma)
        assert e.size == ny and s.size == ny
        n = ny + self.q
        P, Q = np.zeros((n, n)), np.zeros((n, ny))
        _check(lib().rom_couple(self._h, e.ctypes.data_as(_dp), s.ctypes.data_as(_dp),
                                P.ctypes.data_as(_dp), Q.ctypes.data_as(_dp)))
        return P, Q

    def close(self):
        if self._h:
            lib().rom_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rom_build(a, b, r, dx, dy, dt, eps_r, sigma, q, rule=FDTD_RULE_DUAL, f0=30e9,
              gamma=0.99, defl_tol=0.0) -> RomModel:
    e, s = _f64(eps_r), _f64(sigma)
    assert e.size == r * a * r * b and s.size == e.size
    d = rom_desc(a, b, r, dx, dy, dt, e.ctypes.data_as(_dp), s.ctypes.data_as(_dp), q, rule,
                 f0, gamma, defl_tol)
    h = C.c_void_p()
    rep = rom_build_report()
    _check(lib().rom_build(C.byref(d), C.byref(h), C.byref(rep)))
    return RomModel(h, rep, a, b, r)


def rom_build_gpu(a, b, r, dx, dy, dt, eps_r, sigma, q, rule=FDTD_RULE_DUAL, f0=30e9,
                  gamma=0.99, defl_tol=0.0, stream=None) -> RomModel:
    """``rom_build_gpu``: the same model built with the Krylov basis and the
    congruences on the GPU (FP64)."""
    e, s = _f64(eps_r), _f64(sigma)
    assert e.size == r * a * r * b and s.size == e.size
    d = rom_desc(a, b, r, dx, dy, dt, e.ctypes.data_as(_dp), s.ctypes.data_as(_dp), q, rule,
                 f0, gamma, defl_tol)
    h = C.c_void_p()
    rep = rom_build_report()
    _check(lib().rom_build_gpu(C.byref(d), _stream_handle(stream), C.byref(h), C.byref(rep)))
    return RomModel(h, rep, a, b, r)


def _stream_handle(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


class FdtdContext:
    """``fdtd_create``: one or more coarse simulations sharing dx, dy, dt."""

    def __init__(self, dx, dy, dt, sims, stream=None):
        self._keep = [(_f64(e), _f64(s)) for e, s in sims]
        descs = (fdtd_sim_desc * len(sims))()
        for k, (e, s) in enumerate(self._keep):
            ny, nx = e.shape
            descs[k] = fdtd_sim_desc(nx, ny, e.ctypes.data_as(_dp), s.ctypes.data_as(_dp))
        self.shapes = [e.shape for e, _ in self._keep]
        g = fdtd_grid_desc(dx, dy, dt, len(sims), descs)
        h = C.c_void_p()
        _check(lib().fdtd_create(C.byref(g), _stream_handle(stream), C.byref(h)))
        self._h = h
        self.dx, self.dy, self.dt = dx, dy, dt
        self._keep = None

    def _ck(self, rc):
        _check(rc, self._h)

    def rom_embed(self, model: RomModel, sim: int, i0: int, j0: int) -> int:
        inst = C.c_int()
        self._ck(lib().rom_embed(self._h, model._h, sim, i0, j0, C.byref(inst)))
        return inst.value

    def get_rom_map(self, inst):
        n, ny = C.c_int(), C.c_int()
        self._ck(lib().fdtd_get_rom_map(self._h, inst, C.byref(n), C.byref(ny), None, None))
        P = np.zeros((n.value, n.value))
        Q = np.zeros((n.value, ny.value))
        self._ck(lib().fdtd_get_rom_map(self._h, inst, None, None, P.ctypes.data_as(_dp),
                                        Q.ctypes.data_as(_dp)))
        return P, Q

    @staticmethod
    def _sources(sources, host):
        arr = (fdtd_source * max(len(sources), 1))()
        keep = []
        for k, s in enumerate(sources):
            w = s["wave"]
            if host:
                w = _f32(w)
                keep.append(w)
                ptr = w.ctypes.data_as(_fp)
            else:
                assert w.is_cuda and w.dtype.itemsize == 4 and w.is_contiguous()
                ptr = C.cast(C.c_void_p(w.data_ptr()), _fp)
            arr[k] = fdtd_source(s.get("sim", 0), s["comp"], s["i"], s["j"], s.get("len", 1), ptr)
        return arr, keep

    @staticmethod
    def _probes(probes):
        arr = (fdtd_probe * max(len(probes), 1))()
        for k, p in enumerate(probes):
            if len(p) == 2:
                arr[k] = fdtd_probe(0, p[0], p[1])
            else:
                arr[k] = fdtd_probe(p[0], p[1], p[2])
        return arr

    def fdtd_run(self, nsteps, sources=(), probes=(), probe_out=None):
        """Device buffers: source waves are CUDA float32 tensors of length
        >= nsteps; probe_out a CUDA float32 tensor [nsteps, nprobe]."""
        src, _ = self._sources(sources, host=False)
        pr = self._probes(probes)
        out = C.c_void_p(probe_out.data_ptr()) if probe_out is not None else C.c_void_p()
        self._ck(lib().fdtd_run(self._h, nsteps, src, len(sources), pr, len(probes), out))

    def fdtd_run_host(self, nsteps, sources=(), probes=()):
        """Host buffers: numpy waves in, numpy probe samples [nsteps, nprobe] out."""
        src, keep = self._sources(sources, host=True)
        pr = self._probes(probes)
        out = np.zeros((nsteps, max(len(probes), 1)), dtype=np.float32)
        self._ck(lib().fdtd_run_host(self._h, nsteps, src, len(sources), pr, len(probes),
                                     out.ctypes.data_as(_fp)))
        return out[:, :len(probes)]

    def get_fields(self, sim=0):
        ny, nx = self.shapes[sim]
        Ex = np.zeros((ny + 1, nx), np.float32)
        Ey = np.zeros((ny, nx + 1), np.float32)
        Hz = np.zeros((ny, nx), np.float32)
        self._ck(lib().fdtd_get_fields(self._h, sim, Ex.ctypes.data_as(_fp), Ey.ctypes.data_as(_fp),
                                       Hz.ctypes.data_as(_fp)))
        return Ex, Ey, Hz

    def set_fields(self, sim, Ex, Ey, Hz):
        Ex, Ey, Hz = _f32(Ex), _f32(Ey), _f32(Hz)
        self._ck(lib().fdtd_set_fields(self._h, sim, Ex.ctypes.data_as(_fp), Ey.ctypes.data_as(_fp),
                                       Hz.ctypes.data_as(_fp)))

    def get_rom_state(self, inst, q):
        x = np.zeros(q, np.float32)
        self._ck(lib().fdtd_get_rom_state(self._h, inst, x.ctypes.data_as(_fp)))
        return x

    def set_rom_state(self, inst, x):
        x = _f32(x)
        self._ck(lib().fdtd_set_rom_state(self._h, inst, x.ctypes.data_as(_fp)))

    def save_state(self) -> bytes:
        """``fdtd_save_state``: the whole marching state as bytes."""
        n = C.c_size_t()
        self._ck(lib().fdtd_save_state(self._h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._ck(lib().fdtd_save_state(self._h, buf, C.byref(n)))
        return buf.raw

    def load_state(self, data: bytes):
        """``fdtd_load_state``."""
        buf = C.create_string_buffer(data, len(data))
        self._ck(lib().fdtd_load_state(self._h, buf, len(data)))

    def selftest_timeout(self):
        """``fdtd_selftest_timeout``: the status code of the bounded-wait
        failure path (FDTD_ETIMEOUT when it works)."""
        return lib().fdtd_selftest_timeout(self._h)

    def set_pml(self, sim, sides, ncells, m=3.0, sigma_max=0.0, kappa_max=1.0, alpha_max=0.0):
        """Convolutional PML layers of simulation `sim` (``fdtd_set_pml``);
        sides = FDTD_PML_* bits, 0 removes them; sigma_max <= 0 selects the
        default 0.8 (m + 1) / (eta0 h)."""
        d = fdtd_pml_desc(sides, ncells, m, sigma_max, kappa_max, alpha_max)
        self._ck(lib().fdtd_set_pml(self._h, sim, C.byref(d)))

    def fine_fields(self, inst, model):
        """Fine-region (Ex, Ey, Hz) of instance `inst` rebuilt from its state
        (``fdtd_fine_fields``), as CUDA float32 tensors."""
        import torch
        nxf, nyf = model.r * model.a, model.r * model.b
        Ex = torch.empty((nyf + 1, nxf), dtype=torch.float32, device="cuda")
        Ey = torch.empty((nyf, nxf + 1), dtype=torch.float32, device="cuda")
        Hz = torch.empty((nyf, nxf), dtype=torch.float32, device="cuda")
        self._ck(lib().fdtd_fine_fields(self._h, inst, model._h, C.c_void_p(Ex.data_ptr()),
                                        C.c_void_p(Ey.data_ptr()), C.c_void_p(Hz.data_ptr())))
        return Ex, Ey, Hz

    def dft_set(self, monitors, freqs, init=None):
        """Running DFT monitors of Hz (``fdtd_dft_set``): monitors are
        (sim, i, j) or (i, j); freqs in Hz; init an optional complex
        [nmon, nfreq] array of starting sums (as returned by dft_get)."""
        f = _f64(freqs)
        nmon = len(monitors)
        if init is not None:
            a = np.asarray(init, dtype=np.complex128).reshape(nmon, f.size)
            acc = np.ascontiguousarray(np.stack([a.real, a.imag], axis=-1))
            self._dft_init = acc
            ip = acc.ctypes.data_as(_dp)
        else:
            ip = None
        self._ck(lib().fdtd_dft_set(self._h, self._probes(monitors), nmon, f.ctypes.data_as(_dp),
                                    f.size if nmon else 0, ip))
        self._dft_shape = (nmon, f.size if nmon else 0)

    def dft_get(self):
        """X[m, f] = sum_n Hz^{n+1/2}(m) exp(-i 2 pi f (n + 1/2) dt) dt (complex)."""
        nmon, nf = getattr(self, "_dft_shape", (0, 0))
        out = np.zeros((nmon, nf, 2))
        self._ck(lib().fdtd_dft_get(self._h, out.ctypes.data_as(_dp)))
        return out[..., 0] + 1j * out[..., 1]

    def step_count(self):
        n = C.c_longlong()
        self._ck(lib().fdtd_get_step(self._h, C.byref(n)))
        return n.value

    def fdtd_grad(self, nsteps, sources=(), probes=(), ckpt_every=500, need_src=True):
        """Gradient of J = sum of probe Hz^2 over the next nsteps steps (``fdtd_grad``).
        Returns (J, dJ/deps_r per simulation [ny, nx], dJ/dsigma likewise,
        dJ/dJ^n [nsrc, nsteps]) as CUDA float32 tensors (J a float)."""
        import torch
        src, _ = self._sources(sources, host=False)
        pr = self._probes(probes)
        ncell = sum(ny * nx for ny, nx in self.shapes)
        geps = torch.zeros(ncell, dtype=torch.float32, device="cuda")
        gsig = torch.zeros(ncell, dtype=torch.float32, device="cuda")
        gsrc = torch.zeros((max(len(sources), 1), nsteps), dtype=torch.float32, device="cuda")
        J = C.c_double()
        self._ck(lib().fdtd_grad(self._h, nsteps, src, len(sources), pr, len(probes), ckpt_every,
                                 C.c_void_p(geps.data_ptr()), C.c_void_p(gsig.data_ptr()),
                                 C.c_void_p(gsrc.data_ptr()) if need_src else C.c_void_p(),
                                 C.byref(J)))
        out_e, out_s, off = [], [], 0
        for ny, nx in self.shapes:
            out_e.append(geps[off:off + ny * nx].view(ny, nx))
            out_s.append(gsig[off:off + ny * nx].view(ny, nx))
            off += ny * nx
        return J.value, out_e, out_s, gsrc[:len(sources)]

    def fdtd_vjp(self, nsteps, sources, probes, cotangent, ckpt_every=500, need_src=True,
                 probe_out=None):
        """Vector-Jacobian product of the probe series (``fdtd_vjp``): the
        gradient of L = sum cotangent * probes over the next nsteps steps.
        cotangent: CUDA float32 [nsteps, nprobe]; probe_out: optional CUDA
        float32 [nsteps, nprobe] for the forward samples.  Returns
        (dL/deps_r per simulation [ny, nx], dL/dsigma likewise,
        dL/dJ^n [nsrc, nsteps]) as CUDA float32 tensors."""
        import torch
        src, _ = self._sources(sources, host=False)
        pr = self._probes(probes)
        if len(probes):
            assert (cotangent.is_cuda and cotangent.dtype == torch.float32 and cotangent.is_contiguous()
                    and cotangent.numel() == nsteps * len(probes))
        ncell = sum(ny * nx for ny, nx in self.shapes)
        geps = torch.zeros(ncell, dtype=torch.float32, device="cuda")
        gsig = torch.zeros(ncell, dtype=torch.float32, device="cuda")
        gsrc = torch.zeros((max(len(sources), 1), nsteps), dtype=torch.float32, device="cuda")
        ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p()
        self._ck(lib().fdtd_vjp(self._h, nsteps, src, len(sources), pr, len(probes), ckpt_every,
                                ptr(cotangent if len(probes) else None), ptr(geps), ptr(gsig),
                                ptr(gsrc) if need_src else C.c_void_p(), ptr(probe_out)))
        out_e, out_s, off = [], [], 0
        for ny, nx in self.shapes:
            out_e.append(geps[off:off + ny * nx].view(ny, nx))
            out_s.append(gsig[off:off + ny * nx].view(ny, nx))
            off += ny * nx
        return out_e, out_s, gsrc[:len(sources)]

    def energy(self):
        """Storage function W of every simulation (``fdtd_energy``)."""
        out = np.zeros(len(self.shapes))
        self._ck(lib().fdtd_energy(self._h, out.ctypes.data_as(_dp)))
        return out

    def energy_noalloc(self):
        """Same result as ``energy`` without any device allocation
        (``fdtd_energy_noalloc``: partial sums in a fixed library array)."""
        out = np.zeros(len(self.shapes))
        self._ck(lib().fdtd_energy_noalloc(self._h, out.ctypes.data_as(_dp)))
        return out

    def set_timing(self, on: bool):
        self._ck(lib().fdtd_set_timing(self._h, int(bool(on))))

    def steps_per_launch(self) -> int:
        """2 when runs step in pairs (temporal blocking), else 1."""
        r = lib().fdtd_steps_per_launch(self._h)
        if r < 0:
            self._ck(r)
        return r

    def autotune(self, cache_path=None):
        """``fdtd_autotune``: time the bit-identical launch configurations on
        this context and keep the fastest; returns the report as a dict."""
        rep = fdtd_tune_report()
        p = cache_path.encode() if cache_path else None
        self._ck(lib().fdtd_autotune(self._h, p, C.byref(rep)))
        return rep.as_dict()

    def plan(self):
        """The current launch configuration (``fdtd_get_plan``) as a dict."""
        rep = fdtd_tune_report()
        self._ck(lib().fdtd_get_plan(self._h, C.byref(rep)))
        return rep.as_dict()

    def time_stencil(self, launches=16, reps=8):
        """Device ms of one stencil launch alone, from graph replays without
        per-kernel events (``fdtd_time_stencil``); the state is unchanged."""
        ms = C.c_double()
        self._ck(lib().fdtd_time_stencil(self._h, launches, reps, C.byref(ms)))
        return ms.value

    def kernel_times(self):
        """(stencil ms, stencil launches, ROM/probe ms, ROM/probe launches);
        a launch advances steps_per_launch() steps."""
        a, b = C.c_double(), C.c_double()
        na, nb = C.c_longlong(), C.c_longlong()
        self._ck(lib().fdtd_get_kernel_times(self._h, C.byref(a), C.byref(na), C.byref(b), C.byref(nb)))
        return a.value, na.value, b.value, nb.value

    def close(self):
        if getattr(self, "_h", None):
            lib().fdtd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
