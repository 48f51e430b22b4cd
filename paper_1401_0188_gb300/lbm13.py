"""ctypes binding of the lbm13 C ABI (include/lbm13.h).

Argument marshalling only: every step of the time step, the read-outs and the
reductions run in the CUDA library.  The functions mirror the C names
(lbm13_create, lbm13_step, ...); `Lattice` wraps one handle.  PyTorch supplies
device memory (its caching allocator, through the C allocator callback) and
streams.  The library must have been built (paper_1401_0188_gb300.build); a
missing library is an error, there is no fallback.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

Q = 13
PARAM_FIELDS = ("E0", "c1", "k2", "c_epsE", "c_vpi_rho", "c_vpi_E", "Pr", "nu",
                "s_eps", "s_vpi", "s_r", "s_XXe")
PERIODIC, WALL_BB, WALL_MIXED, HALO = 0, 1, 2, 3
HALO_SOUTH, HALO_NORTH = 2, 3
FP64, FP32_DEVIATION = 0, 1
WALL_DENSITY_EXTRAPOLATE, WALL_DENSITY_ZERO_FLUX = 0, 1
PERSISTENT_AUTO, PERSISTENT_OFF, PERSISTENT_ON = 0, 1, 2
PAIR_AUTO, PAIR_OFF, PAIR_ON = 0, 1, 2
DERIVED_COUNT = 48

FIELD_UX, FIELD_UY, FIELD_T, FIELD_P, FIELD_E_SEC7 = 1 << 13, 1 << 14, 1 << 15, 1 << 16, 1 << 17
ALL_MOMENTS = 0x1FFF

STATUS = {0: "LBM13_OK", 1: "LBM13_EINVAL", 2: "LBM13_ENOMEM", 3: "LBM13_EUNSTABLE",
          4: "LBM13_EDIVERGED", 5: "LBM13_ETIMEOUT", 6: "LBM13_ECUDA"}

# Symbols declared in include/lbm13.h.
EXPORTS = ("lbm13_version", "lbm13_status_string", "lbm13_derive", "lbm13_create", "lbm13_destroy",
           "lbm13_last_error", "lbm13_set_stream", "lbm13_info", "lbm13_set_state", "lbm13_set_state_device",
           "lbm13_set_raw_state", "lbm13_get_raw_state", "lbm13_checkpoint_bytes", "lbm13_save",
           "lbm13_restore", "lbm13_step", "lbm13_moments", "lbm13_moments_device",
           "lbm13_residual", "lbm13_time", "lbm13_synchronize", "lbm13_plan_create", "lbm13_plan_destroy",
           "lbm13_plan_last_error", "lbm13_plan_step", "lbm13_plan_tune", "lbm13_plan_set_config",
           "lbm13_plan_config", "lbm13_plan_residual", "lbm13_totals_noalloc", "lbm13_project",
           "lbm13_set_persistent", "lbm13_barrier_check", "lbm13_linear_growth", "lbm13_debug_violations",
           "lbm13_plan_tma_check", "lbm13_fp64_fma_rate", "lbm13_plan_add", "lbm13_plan_remove",
           "lbm13_halo_bytes", "lbm13_halo_pack", "lbm13_halo_unpack", "lbm13_linear_growth_batch",
           "lbm13_set_pair_steps", "lbm13_step_launches", "lbm13_pair_check")


class Lbm13Error(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [(n, C.c_double) for n in PARAM_FIELDS]


class Wall(C.Structure):
    _fields_ = [("kind", C.c_int), ("u_t", C.c_double), ("T", C.c_double)]


class Boundary(C.Structure):
    _fields_ = [("west", Wall), ("east", Wall), ("south", Wall), ("north", Wall),
                ("gx", C.c_double), ("gy", C.c_double), ("rho_ref", C.c_double), ("wall_density", C.c_int),
                ("heat", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


_lib = None


def library_path():
    """The release library, or the bounds-checked one (built with
    build.build(debug=True)) when LBM13_DEBUG_BUILD=1."""
    return _build.DEBUG_LIB if os.environ.get("LBM13_DEBUG_BUILD") == "1" else _build.LIB


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run paper_1401_0188_gb300.build.build() first")
    L = C.CDLL(path)
    dp, vp, i64 = C.POINTER(C.c_double), C.c_void_p, C.c_int64
    sig = {
        "lbm13_version": (C.c_char_p, []),
        "lbm13_status_string": (C.c_char_p, [C.c_int]),
        "lbm13_derive": (C.c_int, [C.POINTER(Params), dp]),
        "lbm13_create": (C.c_int, [C.c_int, C.c_int, C.POINTER(Params), C.POINTER(Boundary), C.c_int,
                                   C.POINTER(Allocator), vp, C.POINTER(vp)]),
        "lbm13_destroy": (None, [vp]),
        "lbm13_last_error": (C.c_char_p, [vp]),
        "lbm13_set_stream": (C.c_int, [vp, vp]),
        "lbm13_info": (C.c_int, [vp, C.POINTER(i64)]),
        "lbm13_set_state": (C.c_int, [vp, dp, dp, dp, dp]),
        "lbm13_set_state_device": (C.c_int, [vp, vp, vp, vp, vp]),
        "lbm13_set_raw_state": (C.c_int, [vp, dp, i64]),
        "lbm13_get_raw_state": (C.c_int, [vp, dp, C.POINTER(i64)]),
        "lbm13_checkpoint_bytes": (C.c_int, [vp, C.POINTER(C.c_size_t)]),
        "lbm13_save": (C.c_int, [vp, vp, C.c_size_t]),
        "lbm13_restore": (C.c_int, [vp, vp, C.c_size_t]),
        "lbm13_step": (C.c_int, [vp, i64]),
        "lbm13_moments": (C.c_int, [vp, dp, C.c_uint]),
        "lbm13_moments_device": (C.c_int, [vp, vp, C.c_uint]),
        "lbm13_residual": (C.c_int, [vp, dp]),
        "lbm13_project": (C.c_int, [vp, C.c_int, C.c_int, dp]),
        "lbm13_set_persistent": (C.c_int, [vp, C.c_int]),
        "lbm13_set_pair_steps": (C.c_int, [vp, C.c_int]),
        "lbm13_step_launches": (C.c_int, [vp, i64, C.POINTER(i64)]),
        "lbm13_pair_check": (C.c_int, [vp, C.c_double, C.c_int, C.POINTER(C.c_int)]),
        "lbm13_linear_growth": (C.c_int, [C.POINTER(Params), C.c_double, C.c_double, C.c_int, C.POINTER(C.c_double)]),
        "lbm13_barrier_check": (C.c_int, [C.c_int, C.c_int, C.c_double, C.POINTER(C.c_int)]),
        "lbm13_linear_growth_batch": (C.c_int, [C.POINTER(Params), dp, dp, C.c_int, C.c_int, dp, vp]),
        "lbm13_debug_violations": (C.c_int, [vp, C.POINTER(C.c_ulonglong)]),
        "lbm13_plan_tma_check": (C.c_int, [vp, C.c_double, C.c_int, C.POINTER(C.c_int)]),
        "lbm13_time": (i64, [vp]),
        "lbm13_synchronize": (C.c_int, [vp]),
        "lbm13_totals_noalloc": (C.c_int, [vp, vp]),
        "lbm13_fp64_fma_rate": (C.c_int, [C.c_int, dp, dp]),
        "lbm13_plan_create": (C.c_int, [C.POINTER(vp), C.c_int, C.POINTER(Allocator), vp, C.POINTER(vp)]),
        "lbm13_plan_destroy": (None, [vp]),
        "lbm13_plan_last_error": (C.c_char_p, [vp]),
        "lbm13_plan_step": (C.c_int, [vp, i64]),
        "lbm13_plan_add": (C.c_int, [vp, vp]),
        "lbm13_halo_bytes": (C.c_int, [vp, C.POINTER(C.c_size_t)]),
        "lbm13_halo_pack": (C.c_int, [vp, C.c_int, vp]),
        "lbm13_halo_unpack": (C.c_int, [vp, C.c_int, vp]),
        "lbm13_plan_remove": (C.c_int, [vp, vp]),
        "lbm13_plan_tune": (C.c_int, [vp, C.c_int, dp]),
        "lbm13_plan_set_config": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
        "lbm13_plan_config": (C.c_int, [vp, C.POINTER(i64)]),
        "lbm13_plan_residual": (C.c_int, [vp, dp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(status, h=None):
    if status != 0:
        msg = lib().lbm13_last_error(h)
        raise Lbm13Error(status, msg.decode() if msg else "")


def make_params(p):
    return Params(*[float(p[n]) for n in PARAM_FIELDS])


def wall(kind=PERIODIC, u_t=0.0, T=0.0):
    return {"kind": kind, "u_t": u_t, "T": T}


def boundary(west=None, east=None, south=None, north=None, gx=0.0, gy=0.0, rho_ref=0.0, wall_density=0,
             heat=0.0):
    w = lambda d: d if d is not None else wall()
    return {"west": w(west), "east": w(east), "south": w(south), "north": w(north),
            "gx": gx, "gy": gy, "rho_ref": rho_ref, "wall_density": wall_density, "heat": heat}


def make_boundary(b):
    mk = lambda d: Wall(int(d["kind"]), float(d.get("u_t", 0.0)), float(d.get("T", 0.0)))
    return Boundary(mk(b["west"]), mk(b["east"]), mk(b["south"]), mk(b["north"]),
                    float(b.get("gx", 0.0)), float(b.get("gy", 0.0)), float(b.get("rho_ref", 0.0)),
                    int(b.get("wall_density", 0)), float(b.get("heat", 0.0)))


def linear_growth(params, ux=0.0, uy=0.0, n=9):
    """max |z| - 1 of the linearised step about rho = 1, u = (ux, uy), T = T0
    over an n x n grid of wave vectors in [-pi, pi]^2 (host only, no GPU)."""
    out = C.c_double(0.0)
    pp = make_params(params)
    _check(lib().lbm13_linear_growth(C.byref(pp), float(ux), float(uy), int(n), C.byref(out)))
    return out.value


def linear_growth_batch(params_list, velocities, n=9, stream=None):
    """max |z| - 1 of the linearised step for every (params_list[c],
    velocities[c]) on an n x n k-grid, scanned on the current CUDA device."""
    count = len(params_list)
    if count != len(velocities) or count < 1:
        raise ValueError("one velocity per parameter set, at least one case")
    arr = (Params * count)(*[make_params(p) for p in params_list])
    ux = np.ascontiguousarray([float(u[0]) for u in velocities])
    uy = np.ascontiguousarray([float(u[1]) for u in velocities])
    out = np.zeros(count)
    _check(lib().lbm13_linear_growth_batch(arr, _dp(ux), _dp(uy), count, int(n), _dp(out),
                                           C.c_void_p(stream.cuda_stream if stream is not None else 0)))
    return out


def barrier_check(blocks, extra_blocks, timeout_s):
    """Self-check of the grid barrier's bounded wait: True when the waits ran
    out (expected exactly when extra_blocks > 0)."""
    out = C.c_int(0)
    _check(lib().lbm13_barrier_check(int(blocks), int(extra_blocks), float(timeout_s), C.byref(out)))
    return bool(out.value)


def fp64_fma_rate(iters=1 << 15):
    """Measured FP64 FMAs per second of the current device, and the timed
    launch's duration in seconds."""
    rate, sec = C.c_double(), C.c_double()
    _check(lib().lbm13_fp64_fma_rate(int(iters), C.byref(rate), C.byref(sec)))
    return rate.value, sec.value


def lbm13_version():
    return lib().lbm13_version().decode()


def lbm13_derive(params):
    """Derived constants of Sec. 2 (host only); returns (status, out[48])."""
    out = np.zeros(DERIVED_COUNT)
    p = make_params(params)
    st = lib().lbm13_derive(C.byref(p), _dp(out))
    return st, out


class _TorchAllocator:
    """Routes the library's device allocations to PyTorch's caching allocator."""

    def __init__(self, device, stream):
        import torch
        self._torch = torch
        self.device = device
        self.stream = stream
        self.live = {}

        def _alloc(size, ctx):
            try:
                ptr = torch.cuda.caching_allocator_alloc(int(size), device=self.device, stream=self.stream)
            except RuntimeError:
                return None
            self.live[ptr] = size
            return ptr

        def _free(ptr, ctx):
            if ptr in self.live:
                del self.live[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        self._a = ALLOC_FN(_alloc)
        self._f = FREE_FN(_free)
        self.struct = Allocator(self._a, self._f, None)


class Lattice:
    """One lattice handle.

    params:    dict with the 12 free parameters (PARAM_FIELDS).
    bnd:       dict from `boundary(...)` (default: fully periodic, no force).
    precision: FP64 or FP32_DEVIATION.
    stream:    a torch.cuda.Stream (default: torch's current stream).
    allocator: "torch" (caching allocator) or None (cudaMalloc).
    """

    def __init__(self, nx, ny, params, bnd=None, precision=FP64, stream=None, allocator="torch", device=None):
        import torch
        self.nx, self.ny = int(nx), int(ny)
        self.params = dict(params)
        self.bnd = bnd if bnd is not None else boundary()
        self.precision = precision
        self.device = torch.cuda.current_device() if device is None else int(device)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self._alloc = _TorchAllocator(self.device, self.stream) if allocator == "torch" else None
            h = C.c_void_p()
            p, b = make_params(self.params), make_boundary(self.bnd)
            st = lib().lbm13_create(self.nx, self.ny, C.byref(p), C.byref(b), int(precision),
                                    C.byref(self._alloc.struct) if self._alloc else None,
                                    C.c_void_p(self.stream.cuda_stream), C.byref(h))
            _check(st)
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().lbm13_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def info(self):
        out = (C.c_int64 * 8)()
        _check(lib().lbm13_info(self._h, out), self._h)
        keys = ("nx", "ny", "pitch", "precision", "elem_bytes", "device_bytes", "step", "persistent_grid")
        return {k: int(out[i]) for i, k in enumerate(keys)}

    @property
    def t(self):
        return int(lib().lbm13_time(self._h))

    def set_stream(self, stream):
        self.stream = stream
        _check(lib().lbm13_set_stream(self._h, C.c_void_p(stream.cuda_stream)), self._h)

    def set_state(self, rho=None, ux=None, uy=None, T=None):
        """Equilibrium of host fields (scalars broadcast; None = rest value)."""
        shape = (self.ny, self.nx)
        arrs = []
        for a in (rho, ux, uy, T):
            if a is None:
                arrs.append(None)
            else:
                arrs.append(np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), shape)))
        ptrs = [_dp(a) if a is not None else None for a in arrs]
        _check(lib().lbm13_set_state(self._h, *ptrs), self._h)

    def set_state_device(self, rho, ux, uy, T):
        """Equilibrium of device fields: torch float64 CUDA tensors of shape (ny, nx)."""
        for a in (rho, ux, uy, T):
            if not (a.is_cuda and a.dtype.is_floating_point and a.element_size() == 8 and a.is_contiguous()):
                raise ValueError("fields must be contiguous float64 CUDA tensors")
            if tuple(a.shape) != (self.ny, self.nx):
                raise ValueError("field shape must be (ny, nx)")
        _check(lib().lbm13_set_state_device(self._h, *[C.c_void_p(a.data_ptr()) for a in (rho, ux, uy, T)]),
               self._h)

    def set_raw_state(self, f, step=0):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(Q, self.ny, self.nx)
        _check(lib().lbm13_set_raw_state(self._h, _dp(f), int(step)), self._h)

    def get_raw_state(self):
        f = np.zeros((Q, self.ny, self.nx))
        st = C.c_int64()
        _check(lib().lbm13_get_raw_state(self._h, _dp(f), C.byref(st)), self._h)
        return f

    def save(self):
        """Bit-exact checkpoint image (bytes)."""
        n = C.c_size_t()
        _check(lib().lbm13_checkpoint_bytes(self._h, C.byref(n)), self._h)
        buf = (C.c_ubyte * n.value)()
        _check(lib().lbm13_save(self._h, buf, n.value), self._h)
        return bytes(buf)

    def restore(self, image):
        buf = (C.c_ubyte * len(image)).from_buffer_copy(image)
        _check(lib().lbm13_restore(self._h, buf, len(image)), self._h)

    def step(self, n=1):
        _check(lib().lbm13_step(self._h, int(n)), self._h)

    def moments(self, mask=ALL_MOMENTS):
        k = bin(mask & 0x3FFFF).count("1")
        out = np.zeros((k, self.ny, self.nx))
        _check(lib().lbm13_moments(self._h, _dp(out), int(mask)), self._h)
        return out

    def macro(self):
        """(rho, ux, uy, T), each (ny, nx)."""
        return self.moments(1 | FIELD_UX | FIELD_UY | FIELD_T)

    def moments_device(self, out, mask=ALL_MOMENTS):
        k = bin(mask & 0x3FFFF).count("1")
        if not (out.is_cuda and out.element_size() == 8 and out.is_contiguous() and out.numel() >= k * self.nx * self.ny):
            raise ValueError("out must be a contiguous float64 CUDA tensor with room for the selected planes")
        _check(lib().lbm13_moments_device(self._h, C.c_void_p(out.data_ptr()), int(mask)), self._h)

    def residual(self, raise_on_divergence=True):
        out = np.zeros(16)
        st = lib().lbm13_residual(self._h, _dp(out))
        if st == 4 and not raise_on_divergence:
            return out
        _check(st, self._h)
        return out

    def debug_violations(self):
        """Out-of-lattice population accesses counted by a bounds-checked
        build (raises on a release build, which checks nothing)."""
        n = C.c_ulonglong(0)
        _check(lib().lbm13_debug_violations(self._h, C.byref(n)), self._h)
        return int(n.value)

    def halo_bytes(self):
        """Bytes of one packed halo: [2 rows][4 populations][nx] in the storage type."""
        n = C.c_size_t()
        _check(lib().lbm13_halo_bytes(self._h, C.byref(n)), self._h)
        return n.value

    def halo_pack(self, side, out):
        """Pack the rows next to halo side `side` (HALO_SOUTH / HALO_NORTH) into
        `out`, a contiguous CUDA tensor of halo_bytes() bytes (stream-ordered)."""
        _check(lib().lbm13_halo_pack(self._h, int(side), C.c_void_p(out.data_ptr())), self._h)

    def halo_unpack(self, side, buf):
        """Write a neighbour's packed halo into the halo rows of `side`."""
        _check(lib().lbm13_halo_unpack(self._h, int(side), C.c_void_p(buf.data_ptr())), self._h)

    def set_persistent(self, mode):
        """PERSISTENT_AUTO (default), PERSISTENT_OFF or PERSISTENT_ON: whether
        step(n) runs many steps per cooperative launch."""
        _check(lib().lbm13_set_persistent(self._h, int(mode)), self._h)

    def set_pair_steps(self, mode):
        """PAIR_AUTO (default: from 2^20 nodes), PAIR_ON or PAIR_OFF: whether
        step(n) advances a lattice periodic in x and y (FP32-deviation) two
        steps per launch."""
        _check(lib().lbm13_set_pair_steps(self._h, int(mode)), self._h)

    def step_launches(self, n):
        """Kernel launches step(n) makes with the current modes."""
        out = C.c_int64()
        _check(lib().lbm13_step_launches(self._h, int(n), C.byref(out)), self._h)
        return out.value

    def pair_check(self, timeout_s, withhold=True):
        """Self-check of the paired steps' bounded wait; True when it ran out."""
        out = C.c_int()
        _check(lib().lbm13_pair_check(self._h, float(timeout_s), int(bool(withhold)), C.byref(out)), self._h)
        return bool(out.value)

    def project(self, kx, ky=0):
        """Fourier aggregates (Sec. 6): [field][harmonic][cos, sin] for the
        fields (rho - 1, ux, uy, T - T0, E - E0, p - T0), harmonics k and 2k of
        k = 2 pi (kx/nx, ky/ny); sums over all nodes."""
        out = np.zeros(24)
        _check(lib().lbm13_project(self._h, int(kx), int(ky), _dp(out)), self._h)
        return out.reshape(6, 2, 2)

    def synchronize(self):
        _check(lib().lbm13_synchronize(self._h), self._h)


def _pcheck(status, p=None):
    if status != 0:
        msg = lib().lbm13_plan_last_error(p)
        raise Lbm13Error(status, msg.decode() if msg else "")


class Plan:
    """Batched stepping of many lattices (one launch per step, CUDA graphs for
    runs of 32 steps).  The Lattice objects must outlive the plan."""

    def __init__(self, lattices, stream=None, allocator="torch"):
        import torch
        if not lattices:
            raise ValueError("empty lattice list")
        self.lattices = list(lattices)
        dev = self.lattices[0].device
        with torch.cuda.device(dev):
            self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
            self._alloc = _TorchAllocator(dev, self.stream) if allocator == "torch" else None
            arr = (C.c_void_p * len(self.lattices))(*[l.handle for l in self.lattices])
            h = C.c_void_p()
            _pcheck(lib().lbm13_plan_create(arr, len(self.lattices),
                                            C.byref(self._alloc.struct) if self._alloc else None,
                                            C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().lbm13_plan_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        _pcheck(lib().lbm13_plan_step(self._h, int(n)), self._h)

    def add(self, lattice):
        """Admit one more lattice (ordered after the work on its own stream)."""
        _pcheck(lib().lbm13_plan_add(self._h, lattice.handle), self._h)
        self.lattices.append(lattice)

    def remove(self, lattice):
        """Retire a lattice: the last one takes its row in residual()."""
        _pcheck(lib().lbm13_plan_remove(self._h, lattice.handle), self._h)
        i = next(k for k, l in enumerate(self.lattices) if l is lattice)
        self.lattices[i] = self.lattices[-1]
        self.lattices.pop()

    def tune(self, steps_per_candidate=4):
        best = C.c_double()
        _pcheck(lib().lbm13_plan_tune(self._h, int(steps_per_candidate), C.byref(best)), self._h)
        return best.value

    def set_config(self, R=2, BY=4, ctas_per_sm=8, order=0, groups=1):
        _pcheck(lib().lbm13_plan_set_config(self._h, int(R), int(BY), int(ctas_per_sm), int(order), int(groups)),
                self._h)

    def residual(self, raise_on_divergence=True):
        """(count, 16) FP64 read-outs of every lattice, one synchronisation."""
        out = np.zeros((len(self.lattices), 16))
        st = lib().lbm13_plan_residual(self._h, _dp(out))
        if st == 4 and not raise_on_divergence:
            return out
        _pcheck(st, self._h)
        return out

    def tma_check(self, timeout_s, withhold=True):
        """Self-check of the staged tiles' bounded wait: True when the waits
        ran out (expected exactly when the copies are withheld)."""
        out = C.c_int(0)
        _pcheck(lib().lbm13_plan_tma_check(self._h, float(timeout_s), 1 if withhold else 0, C.byref(out)), self._h)
        return bool(out.value)

    def config(self):
        out = (C.c_int64 * 9)()
        _pcheck(lib().lbm13_plan_config(self._h, out), self._h)
        keys = ("R", "BY", "ctas_per_sm", "order", "tiles", "grid", "nodes", "tried", "groups")
        return {k: int(out[i]) for i, k in enumerate(keys)}
