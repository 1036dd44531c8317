"""Thin ctypes binding of liblee (include/lee.h): same names as the C ABI,
argument marshalling only.  Every step of the path runs in the library's CUDA
kernels; there is no CPU fallback: importing this module without a built
``liblee.so`` raises.

``Solver`` bundles the calls of one solve: it allocates the device arena that
``lee_plan`` asks for with PyTorch and binds it with a dedicated CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblee.so")

LEE_OK, LEE_ERR_ARG, LEE_ERR_GEOMETRY, LEE_ERR_RANK, LEE_ERR_ADE_UNSTABLE, LEE_ERR_BUDGET, LEE_ERR_CUDA, \
    LEE_ERR_DIVERGED, LEE_ERR_TIMEOUT = range(9)
LEE_FP64, LEE_FP32 = 0, 1
LEE_BC_RADIATION, LEE_BC_PERIODIC = 0, 1
LEE_P, LEE_U, LEE_V = 0, 1, 2
STATUS_TIMEOUT, STATUS_DIVERGED = 1, 2      # bits of a member's status word (Batch.status)
_STATUS = {1: "ARG", 2: "GEOMETRY", 3: "RANK", 4: "ADE_UNSTABLE", 5: "BUDGET", 6: "CUDA", 7: "DIVERGED", 8: "TIMEOUT"}


class LeeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"LEE_ERR_{_STATUS.get(code, code)}: {msg}")
        self.code = code


class lee_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("h", C.c_double), ("cfl", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double), ("precision", C.c_int),
                ("bc_x", C.c_int), ("bc_y", C.c_int)]


class lee_sizes(C.Structure):
    _fields_ = [("device_bytes", C.c_longlong), ("n_ghost", C.c_int), ("n_fluid", C.c_int),
                ("n_entries", C.c_longlong), ("n_reduced", C.c_int), ("regime", C.c_int),
                ("dt", C.c_double), ("ade_amplification", C.c_double), ("n_tiles", C.c_int),
                ("n_states", C.c_int)]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_llp = C.POINTER(C.c_longlong)
_vp = C.c_void_p

# name: (restype, argtypes) -- mirrors include/lee.h
SIGNATURES = {
    "lee_create": (C.c_int, [C.POINTER(_vp), C.POINTER(lee_grid)]),
    "lee_destroy": (C.c_int, [_vp]),
    "lee_last_error": (C.c_char_p, [_vp]),
    "lee_set_wall_none": (C.c_int, [_vp]),
    "lee_set_wall_line": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double]),
    "lee_set_wall_cylinder": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double]),
    "lee_set_impedance": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double]),
    "lee_set_rigid": (C.c_int, [_vp]),
    "lee_set_tile": (C.c_int, [_vp, C.c_int, C.c_int]),
    "lee_set_sponge": (C.c_int, [_vp, C.c_int, C.c_double]),
    "lee_fill_ghosts_with_bc": (C.c_int, [_vp, _dp]),
    "lee_set_impedance_rational": (C.c_int, [_vp, C.c_int, _dp, C.c_int, _dp]),
    "lee_batch_set_stage_fusion": (C.c_int, [_vp, C.c_int]),
    "lee_batch_fused_tiles": (C.c_int, [_vp, _llp, _llp]),
    "lee_batch_set_band_in_tile": (C.c_int, [_vp, C.c_int]),
    "lee_batch_read_latest_probes_async": (C.c_int, [_vp, _dp, _llp]),
    "lee_batch_band_in_tile": (C.c_int, [_vp, C.POINTER(C.c_int)]),
    "lee_fp64_fma_probe": (C.c_int, [C.c_int, C.c_longlong, _vp, _vp]),
    "lee_plan": (C.c_int, [_vp, C.POINTER(lee_sizes)]),
    "lee_bind": (C.c_int, [_vp, _vp, C.c_longlong, _vp]),
    "lee_init_pulse": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double, C.c_double]),
    "lee_init_packet": (C.c_int, [_vp] + [C.c_double] * 6),
    "lee_set_monopole": (C.c_int, [_vp] + [C.c_double] * 5),
    "lee_write_field": (C.c_int, [_vp, C.c_int, _dp]),
    "lee_set_probes": (C.c_int, [_vp, C.c_int, _dp, C.c_int]),
    "lee_read_probes": (C.c_int, [_vp, _dp, _llp]),
    "lee_step": (C.c_int, [_vp, C.c_longlong]),
    "lee_sync": (C.c_int, [_vp]),
    "lee_read_field": (C.c_int, [_vp, C.c_int, _dp]),
    "lee_read_mask": (C.c_int, [_vp, C.POINTER(C.c_ubyte)]),
    "lee_tile_flags": (C.c_int, [_vp, C.POINTER(C.c_uint), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "lee_read_ade": (C.c_int, [_vp, _dp]),
    "lee_get_step": (C.c_int, [_vp, _llp]),
    "lee_energy": (C.c_int, [_vp, _dp]),
    "lee_state_bytes": (C.c_int, [_vp, _llp]),
    "lee_read_state": (C.c_int, [_vp, _vp]),
    "lee_write_state": (C.c_int, [_vp, _vp]),
    "lee_upload_state_async": (C.c_int, [_vp, _vp]),
    "lee_download_probes_async": (C.c_int, [_vp, _dp, C.c_longlong, C.c_longlong]),
    "lee_ghost_info": (C.c_int, [_vp, C.c_int, _ip, _dp, _ip, _ip]),
    "lee_ghost_weights": (C.c_int, [_vp, C.c_int, _ip, _dp, _dp]),
    "lee_batch_create": (C.c_int, [C.POINTER(_vp), C.c_int]),
    "lee_batch_destroy": (C.c_int, [_vp]),
    "lee_batch_add": (C.c_int, [_vp, _vp]),
    "lee_batch_remove": (C.c_int, [_vp, _vp]),
    "lee_batch_plan": (C.c_int, [_vp, _llp]),
    "lee_batch_bind": (C.c_int, [_vp, _vp, C.c_longlong, _vp]),
    "lee_batch_step": (C.c_int, [_vp, C.c_longlong]),
    "lee_batch_last_error": (C.c_char_p, [_vp]),
    "lee_batch_launch": (C.c_int, [_vp, C.c_int, C.c_int]),
    "lee_batch_status": (C.c_int, [_vp, _llp, C.c_int]),
    "lee_batch_stencil_kernel": (C.c_char_p, [_vp]),
    "lee_batch_set_strips_per_sm": (C.c_int, [_vp, C.c_int]),
    "lee_energy_noalloc": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int, C.c_int, C.c_longlong, C.c_int, C.c_double,
                                      _vp, _vp]),
    "lee_launch_count": (C.c_longlong, []),
    "lee_version": (C.c_char_p, []),
}

_lib = None


def load():
    """Load liblee.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc, ctx=None, batch=None):
    if rc != LEE_OK:
        L = load()
        if batch is not None:
            msg = L.lee_batch_last_error(batch)
        else:
            msg = L.lee_last_error(ctx)
        raise LeeError(rc, (msg or b"").decode())


def _d(a):
    return a.ctypes.data_as(_dp)


class Solver:
    """One solve behind the C ABI: create -> wall/impedance/probes -> plan ->
    bind (device arena from PyTorch, dedicated stream) -> init -> step -> read."""

    def __init__(self, nx, ny, h, cfl=0.5, x0=0.0, y0=0.0, precision="fp64",
                 periodic_x=False, periodic_y=False, device=None):
        self.L = load()
        self.nx, self.ny, self.h = nx, ny, h
        self.precision = LEE_FP32 if precision in ("fp32", LEE_FP32) else LEE_FP64
        g = lee_grid(nx, ny, h, cfl, x0, y0, self.precision,
                     LEE_BC_PERIODIC if periodic_x else LEE_BC_RADIATION,
                     LEE_BC_PERIODIC if periodic_y else LEE_BC_RADIATION)
        self.ctx = _vp()
        _check(self.L.lee_create(C.byref(self.ctx), C.byref(g)), None)
        self.sizes = None
        self.arena = None
        self.stream = None
        self.device = device
        self._nprobe = 0

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx:
            try:
                if self.stream is not None:
                    self.L.lee_sync(ctx)
            finally:
                self.L.lee_destroy(ctx)
            self.ctx = None

    def _c(self, rc):
        _check(rc, self.ctx)

    # ---- set-up
    def set_wall_none(self):
        self._c(self.L.lee_set_wall_none(self.ctx)); return self

    def set_wall_line(self, xw, yw, angle):
        self._c(self.L.lee_set_wall_line(self.ctx, xw, yw, angle)); return self

    def set_wall_cylinder(self, xc, yc, r):
        self._c(self.L.lee_set_wall_cylinder(self.ctx, xc, yc, r)); return self

    def set_impedance(self, R, M, K):
        self._c(self.L.lee_set_impedance(self.ctx, R, M, K)); return self

    def set_impedance_rational(self, real=(), pairs=()):
        """Rational admittance of Sec. 2.3 (Y_inf = 0): real = [(lam, A)],
        pairs = [(alpha, beta, B, C)]."""
        r = np.ascontiguousarray(np.asarray(real, dtype=np.float64).reshape(-1, 2))
        q = np.ascontiguousarray(np.asarray(pairs, dtype=np.float64).reshape(-1, 4))
        rb = r if r.size else np.zeros(2)
        qb = q if q.size else np.zeros(4)
        self._c(self.L.lee_set_impedance_rational(self.ctx, len(r), _d(rb), len(q), _d(qb)))
        return self

    def set_rigid(self):
        self._c(self.L.lee_set_rigid(self.ctx)); return self

    def set_probes(self, xy, capacity):
        xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1)
        self._nprobe = len(xy) // 2
        self._c(self.L.lee_set_probes(self.ctx, self._nprobe, _d(xy), int(capacity)))
        return self

    def set_sponge(self, width, kappa=0.04):
        """Opt-in absorbing ramp over `width` outer layers (0 = off, the default;
        before plan); a departure from the paper, which adds no damping."""
        self._c(self.L.lee_set_sponge(self.ctx, int(width), float(kappa))); return self

    def set_tile(self, tile_w, tile_h):
        """FP32 TMA stencil tile shape (before plan); (0, 0) = default."""
        self._c(self.L.lee_set_tile(self.ctx, int(tile_w), int(tile_h))); return self

    def plan(self):
        s = lee_sizes()
        self._c(self.L.lee_plan(self.ctx, C.byref(s)))
        self.sizes = s
        return s

    def bind(self, arena=None, stream=None):
        import torch
        if self.sizes is None:
            self.plan()
        dev = self.device or torch.device("cuda", torch.cuda.current_device())
        if arena is None:
            arena = torch.empty(int(self.sizes.device_bytes), dtype=torch.uint8, device=dev)
        self.arena = arena
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        self._c(self.L.lee_bind(self.ctx, arena.data_ptr(), arena.numel(), C.c_void_p(self.stream.cuda_stream)))
        return self

    # ---- state
    def init_pulse(self, xs, ys, amp, halfwidth):
        self._c(self.L.lee_init_pulse(self.ctx, xs, ys, amp, halfwidth)); return self

    def init_packet(self, xs, ys, angle, amp, k, alpha):
        self._c(self.L.lee_init_packet(self.ctx, xs, ys, angle, amp, k, alpha)); return self

    def set_monopole(self, xs, ys, amp, halfwidth, omega):
        self._c(self.L.lee_set_monopole(self.ctx, xs, ys, amp, halfwidth, omega)); return self

    def write_field(self, which, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(-1)
        assert a.size == self.nx * self.ny
        self._c(self.L.lee_write_field(self.ctx, which, _d(a)))

    def step(self, n):
        self._c(self.L.lee_step(self.ctx, int(n))); return self

    def sync(self):
        self._c(self.L.lee_sync(self.ctx))

    # ---- read back
    def field(self, which):
        out = np.empty(self.nx * self.ny)
        self._c(self.L.lee_read_field(self.ctx, which, _d(out)))
        return out.reshape(self.ny, self.nx)

    def mask(self):
        out = np.empty(self.nx * self.ny, dtype=np.uint8)
        self._c(self.L.lee_read_mask(self.ctx, out.ctypes.data_as(C.POINTER(C.c_ubyte))))
        return out.reshape(self.ny, self.nx)

    def tile_flags(self):
        """Stencil tile classes of the plan (tiles_y x tiles_x flag words; bits
        in include/lee.h, lee_tile_flags)."""
        tx, ty = C.c_int(), C.c_int()
        self._c(self.L.lee_tile_flags(self.ctx, None, C.byref(tx), C.byref(ty)))
        out = np.zeros(max(tx.value * ty.value, 1), dtype=np.uint32)
        self._c(self.L.lee_tile_flags(self.ctx, out.ctypes.data_as(C.POINTER(C.c_uint)), C.byref(tx), C.byref(ty)))
        return out[:tx.value * ty.value].reshape(ty.value, tx.value)

    def ade(self):
        ng, ns = self.sizes.n_ghost, self.sizes.n_states
        out = np.zeros(ns * max(ng, 1))
        self._c(self.L.lee_read_ade(self.ctx, _d(out)))
        return out[:ns * ng].reshape(-1, ns)

    def steps_done(self):
        v = C.c_longlong()
        self._c(self.L.lee_get_step(self.ctx, C.byref(v)))
        return v.value

    def probes(self):
        n = C.c_longlong()
        self._c(self.L.lee_read_probes(self.ctx, None, C.byref(n)))
        out = np.empty(max(n.value * self._nprobe, 1))
        self._c(self.L.lee_read_probes(self.ctx, _d(out), C.byref(n)))
        return out[:n.value * self._nprobe].reshape(n.value, self._nprobe)

    def energy(self):
        e = C.c_double()
        self._c(self.L.lee_energy(self.ctx, C.byref(e)))
        return e.value

    def read_state(self):
        nb = C.c_longlong()
        self._c(self.L.lee_state_bytes(self.ctx, C.byref(nb)))
        blob = np.empty(nb.value, dtype=np.uint8)
        self._c(self.L.lee_read_state(self.ctx, blob.ctypes.data_as(_vp)))
        return blob

    def write_state(self, blob):
        blob = np.ascontiguousarray(blob, dtype=np.uint8)
        self._c(self.L.lee_write_state(self.ctx, blob.ctypes.data_as(_vp)))

    def fill_ghosts_with_bc(self, bc):
        """Test hook: ghost nodes of Q^n from given boundary data, bc[g] =
        (u.n, dp/dn) at ghost g's boundary point (steps 4-5 of Sec. 3.2)."""
        a = np.ascontiguousarray(bc, dtype=np.float64).reshape(-1)
        self._c(self.L.lee_fill_ghosts_with_bc(self.ctx, _d(a)))

    # ---- plan export (host; no device needed)
    def ghost(self, g):
        t = C.c_int(); m = C.c_int(); n = C.c_int()
        meta = np.empty(5)
        self._c(self.L.lee_ghost_info(self.ctx, g, C.byref(t), _d(meta), C.byref(m), C.byref(n)))
        idx = np.empty(n.value, dtype=np.int32)
        w = np.empty(4 * n.value)
        kap = np.empty(2)
        self._c(self.L.lee_ghost_weights(self.ctx, g, idx.ctypes.data_as(_ip), _d(w), _d(kap)))
        return dict(target=t.value, bp=meta[:2].copy(), n=meta[2:4].copy(), r=meta[4], m=m.value,
                    cloud=idx, w=w.reshape(-1, 4), kappa=kap)


class Batch:
    """Several bound Solvers advanced by one ghost and one stencil launch per stage."""

    def __init__(self, precision="fp32", stream=None):
        import torch
        self.L = load()
        self.b = _vp()
        self.precision = LEE_FP32 if precision in ("fp32", LEE_FP32) else LEE_FP64
        _check(self.L.lee_batch_create(C.byref(self.b), self.precision))
        self.members = []
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.arena = None

    def __del__(self):
        b = getattr(self, "b", None)
        if b:
            self.L.lee_batch_destroy(b)
            self.b = None

    def _c(self, rc):
        _check(rc, batch=self.b)

    def add(self, solver):
        self._c(self.L.lee_batch_add(self.b, solver.ctx))
        self.members.append(solver)
        self._rebind()

    def remove(self, solver):
        self._c(self.L.lee_batch_remove(self.b, solver.ctx))
        self.members.remove(solver)
        self._rebind()

    def _rebind(self):
        import torch
        nb = C.c_longlong()
        self._c(self.L.lee_batch_plan(self.b, C.byref(nb)))
        if self.arena is None or self.arena.numel() < nb.value:
            # grow geometrically so that adding members one by one stays cheap
            self.arena = torch.empty(max(int(nb.value) * 2, 1 << 16), dtype=torch.uint8, device="cuda")
            self._c(self.L.lee_batch_bind(self.b, self.arena.data_ptr(), self.arena.numel(),
                                          C.c_void_p(self.stream.cuda_stream)))

    def step(self, n):
        # members' own streams must be idle before the batch stream uses their buffers
        for s in self.members:
            s.stream.synchronize()
        self._c(self.L.lee_batch_step(self.b, int(n)))

    def sync(self):
        self.stream.synchronize()

    def status(self):
        """Members' status words after the batch stream drains (0 healthy,
        STATUS_TIMEOUT, STATUS_DIVERGED bits), in member order."""
        n = len(self.members)
        out = np.zeros(max(n, 1), dtype=np.int64)
        self._c(self.L.lee_batch_status(self.b, out.ctypes.data_as(_llp), n))
        return out[:n]

    def set_stage_fusion(self, on=True):
        """Temporal blocking of stages 1 and 2 on tiles clear of walls, band
        and ramp (FP32, 64 x 40 tiles); results bitwise those of the unfused
        stages."""
        self._c(self.L.lee_batch_set_stage_fusion(self.b, int(bool(on))))

    def latest_probe_count(self):
        """Values that read_latest_probes returns (every member's probe count)."""
        n = C.c_longlong()
        self._c(self.L.lee_batch_read_latest_probes_async(self.b, C.cast(None, _dp), C.byref(n)))
        return n.value

    def read_latest_probes_async(self, host_ptr):
        """Enqueue the gather of every member's latest probe record into host
        memory at host_ptr (latest_probe_count() doubles, pinned for an
        asynchronous copy) on the batch stream."""
        n = C.c_longlong()
        self._c(self.L.lee_batch_read_latest_probes_async(self.b, C.cast(C.c_void_p(host_ptr), _dp), C.byref(n)))
        return n.value

    def read_latest_probes(self):
        """Every member's latest probe record, members in order (synchronous)."""
        out = np.zeros(max(self.latest_probe_count(), 1))
        self.read_latest_probes_async(out.ctypes.data)
        self.sync()
        return out[:self.latest_probe_count()]

    def set_band_in_tile(self, stage_mask=-1):
        """Stages (bit k for stage k) whose band nodes the warp-specialised
        stencil updates inside its band tiles instead of a separate band pass
        (-1: the default); both give bitwise the same values."""
        self._c(self.L.lee_batch_set_band_in_tile(self.b, int(stage_mask)))

    def band_in_tile(self):
        """The stage mask in effect (see set_band_in_tile)."""
        m = C.c_int()
        self._c(self.L.lee_batch_band_in_tile(self.b, C.byref(m)))
        return m.value

    def fused_tiles(self):
        """(tiles the fused pass covers, all tiles)."""
        f, t = C.c_longlong(), C.c_longlong()
        self._c(self.L.lee_batch_fused_tiles(self.b, C.byref(f), C.byref(t)))
        return f.value, t.value

    def set_strips_per_sm(self, strips):
        """Stencil work packing: tile strips per SM (0 = default 2)."""
        self._c(self.L.lee_batch_set_strips_per_sm(self.b, int(strips)))

    def stencil_kernel(self):
        """Name of the stencil kernel variant this batch launches."""
        return (self.L.lee_batch_stencil_kernel(self.b) or b"").decode()

    def launch(self, stage, what):
        """Measurement hook: one ghost (what=0) or stencil (what=1) launch of a stage."""
        self._c(self.L.lee_batch_launch(self.b, int(stage), int(what)))


def launch_count():
    return load().lee_launch_count()


def version():
    return load().lee_version().decode()
