"""Thin ctypes binding of libm2cgpu.so (include/m2c.h).

The functions named like the C entry points marshal arguments only; every
step of the solver runs in the library's CUDA kernels. ``Grid`` is a small
convenience owner of the torch device tensors a context borrows (state,
workspace). Loading fails with an error if the library is missing: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libm2cgpu.so")

M2C_OK, M2C_EINVAL = 0, 1
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "ENONPHYS", 6: "EVACUUM",
          7: "ETIMEOUT", 8: "EOVERFLOW"}
EOS_SG, EOS_MG = 0, 1
FP64, MIXED = 0, 1
BC_TRANSMISSIVE, BC_PERIODIC, BC_SYMMETRY = 0, 1, 2
LIM_VAN_ALBADA, LIM_MC = 0, 1
FLUX_HLLC, FLUX_LLF = 0, 1
GEOM_CARTESIAN, GEOM_CYLINDRICAL, GEOM_SPHERICAL = 0, 1, 2


class M2CError(RuntimeError):
    def __init__(self, code: int, where: str, text: str = ""):
        super().__init__(f"{where}: {STATUS.get(code, code)} {text}".strip())
        self.code = code


class EosDesc(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("params", ctypes.c_double * 6)]


class Options(ctypes.Structure):
    _fields_ = [("rk", ctypes.c_int), ("limiter", ctypes.c_int), ("flux", ctypes.c_int),
                ("mc_alpha", ctypes.c_double), ("dt_fixed", ctypes.c_double), ("geom", ctypes.c_int),
                ("x0", ctypes.c_double), ("band_beta", ctypes.c_double), ("band_gamma", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("interface_faces", ctypes.c_long), ("interface_cells", ctypes.c_long),
                ("flipped_cells", ctypes.c_long), ("dt", ctypes.c_double)]


_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        p, i, d, z, L_ = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_long
        L.m2c_workspace_bytes.restype = z
        L.m2c_workspace_bytes.argtypes = [i, i, i, i]
        L.m2c_workspace_bytes_rk.restype = z
        L.m2c_workspace_bytes_rk.argtypes = [i, i, i, i, i]
        L.m2c_set_options.argtypes = [p, ctypes.POINTER(Options)]
        L.m2c_batch_workspace_bytes.restype = z
        L.m2c_batch_workspace_bytes.argtypes = [i]
        L.m2c_batch_create.argtypes = [ctypes.POINTER(p), p, i, p, z, p]
        L.m2c_batch_step.argtypes = [p, i]
        L.m2c_batch_capture.argtypes = [p, i, ctypes.POINTER(p)]
        L.m2c_batch_launch_graph.argtypes = [p, p]
        L.m2c_graph_destroy.argtypes = [p]
        L.m2c_graph_destroy.restype = None
        L.m2c_batch_destroy.argtypes = [p]
        L.m2c_batch_destroy.restype = None
        L.m2c_init_grid.argtypes = [ctypes.POINTER(p), i, i, i, p, d, p, i, p, z, p]
        L.m2c_set_eos.argtypes = [p, i, i, p, i]
        L.m2c_set_scheme.argtypes = [p, d, i, i]
        L.m2c_set_tiling.argtypes = [p, i, i]
        L.m2c_set_riemann_start.argtypes = [p, i]
        L.m2c_set_state.argtypes = [p, p, p, d, L_]
        L.m2c_prims_to_state.argtypes = [p, p]
        L.m2c_state_to_prims.argtypes = [p, p]
        L.m2c_upload_state.argtypes = [p, p, p]
        L.m2c_download_state.argtypes = [p, p, p]
        L.m2c_step_host.argtypes = [p, p, p, i]
        L.m2c_step.argtypes = [p, i]
        L.m2c_residual.argtypes = [p, p, p]
        L.m2c_sync.argtypes = [p, p, p, p]
        L.m2c_get_stats.argtypes = [p, ctypes.POINTER(Stats)]
        L.m2c_riemann_workspace_bytes.restype = z
        L.m2c_riemann_workspace_bytes.argtypes = [i]
        L.m2c_solve_riemann.argtypes = [i, ctypes.POINTER(EosDesc), p, ctypes.POINTER(EosDesc), p, p, p, p, i, p, z,
                                        p]
        L.m2c_solve_riemann_mixed.argtypes = L.m2c_solve_riemann.argtypes
        L.m2c_shock_state.argtypes = [ctypes.POINTER(EosDesc), p, d, p, p, z, p]
        L.m2c_residual_noalloc_scratch_bytes.restype = z
        L.m2c_residual_noalloc_scratch_bytes.argtypes = []
        L.m2c_residual_noalloc.argtypes = [i, i, i, d, p, ctypes.POINTER(EosDesc), ctypes.POINTER(EosDesc), i,
                                           p, p, p, p, p]
        L.m2c_profile.argtypes = [p, i]
        L.m2c_profile_read.argtypes = [p, ctypes.POINTER(d), ctypes.POINTER(L_)]
        L.m2c_profile_read_kernels.argtypes = [p, p, p]
        L.m2c_destroy.argtypes = [p]
        L.m2c_destroy.restype = None
        L.m2c_last_error.argtypes = [p]
        L.m2c_last_error.restype = ctypes.c_char_p
        L.m2c_status_string.argtypes = [i]
        L.m2c_status_string.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(code: int, where: str, ctx=None):
    """Raises M2CError with the library's text for the context (or, without one, for the last
    call on this thread that has no context)."""
    if code != M2C_OK:
        raise M2CError(code, where, lib().m2c_last_error(ctx).decode())


def eos_desc(eos) -> EosDesc:
    """eos = (type, params) as in workloads.py."""
    t, prm = eos
    e = EosDesc()
    e.type = t
    vals = list(prm) + [0.0] * (6 - len(prm))
    if t == EOS_MG and len(prm) < 6:
        vals[5] = -math.inf
    for k in range(6):
        e.params[k] = vals[k]
    return e


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _buf(t, numel, name, cuda):
    """Pointer of t after checking that it is a contiguous float64 torch tensor of numel
    elements on the device (cuda) or on the host: the library reads or writes numel doubles
    through the pointer and has no other way to know the buffer's extent."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: a torch tensor is required, got {type(t).__name__}")
    where = "device" if cuda else "host"
    if t.is_cuda != cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{name}: a contiguous float64 {where} tensor of {numel} elements is required, got "
                         f"{t.dtype} {tuple(t.shape)} on {t.device}{'' if t.is_contiguous() else ' (strided)'}")
    return _ptr(t)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------- C entry points

def m2c_workspace_bytes(nx, ny, nz, precision=FP64) -> int:
    return lib().m2c_workspace_bytes(nx, ny, nz, precision)


def m2c_workspace_bytes_rk(nx, ny, nz, precision=FP64, rk=2) -> int:
    return lib().m2c_workspace_bytes_rk(nx, ny, nz, precision, rk)


def m2c_batch_workspace_bytes(k) -> int:
    return lib().m2c_batch_workspace_bytes(k)


def m2c_solve_riemann(eosL, L, eosR, R, stream=None, mixed=False):
    """Batch Riemann solve on device tensors L, R of shape (3, n) float64 (rho, u, p).
    Returns (out (4, n): p*, u*, rho*_L, rho*_R; iters (n,); status (n,)).
    mixed=True: the mixed path's solve (m2c_solve_riemann_mixed)."""
    import torch
    if not (isinstance(L, torch.Tensor) and isinstance(R, torch.Tensor)) or L.dim() != 2 or L.shape[0] != 3 \
            or tuple(R.shape) != tuple(L.shape):
        raise ValueError(f"L and R of shape (3, n) are required, got {tuple(L.shape)} and {tuple(R.shape)}")
    n = L.shape[1]
    # contiguous copies (if any) stay referenced until the call returns: the
    # kernel reads them on the stream after the launch
    Lc, Rc = L.contiguous(), R.contiguous()
    out = torch.empty((4, n), dtype=torch.float64, device=L.device)
    iters = torch.zeros(n, dtype=torch.int32, device=L.device)
    status = torch.zeros(n, dtype=torch.int32, device=L.device)
    eL, eR = eos_desc(eosL), eos_desc(eosR)
    fn = lib().m2c_solve_riemann_mixed if mixed else lib().m2c_solve_riemann
    code = fn(n, ctypes.byref(eL), _buf(Lc, 3 * n, "L", True), ctypes.byref(eR), _buf(Rc, 3 * n, "R", True),
              _ptr(out), _ptr(iters), _ptr(status), 1, None, 0, _stream_handle(stream))
    _check(code, "m2c_solve_riemann_mixed" if mixed else "m2c_solve_riemann")
    return out, iters, status


def _device_workspace(nbytes):
    """A 256-byte aligned device buffer of nbytes (torch owns it): (tensor, pointer)."""
    import torch
    t = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    return t, ctypes.c_void_p(t.data_ptr() + (-t.data_ptr()) % 256)


def m2c_riemann_workspace_bytes(n) -> int:
    return lib().m2c_riemann_workspace_bytes(n)


def m2c_solve_riemann_host(eosL, L, eosR, R, mixed=False):
    """Host-array variant: L, R numpy (3, n); returns (code, out (4, n), iters, status).
    The library stages the arrays through a device workspace owned here."""
    import numpy as np
    L = np.ascontiguousarray(L, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    n = L.shape[1]
    out = np.zeros((4, n))
    iters = np.zeros(n, dtype=np.int32)
    status = np.zeros(n, dtype=np.int32)
    eL, eR = eos_desc(eosL), eos_desc(eosR)
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    nb = m2c_riemann_workspace_bytes(n)
    ws, wp = _device_workspace(nb)
    fn = lib().m2c_solve_riemann_mixed if mixed else lib().m2c_solve_riemann
    code = fn(n, ctypes.byref(eL), vp(L), ctypes.byref(eR), vp(R), vp(out), vp(iters), vp(status), 0, wp, nb, None)
    del ws
    return code, out, iters, status


def m2c_shock_state(eos, w, p1):
    import numpy as np
    e = eos_desc(eos)
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros(3)
    nb = m2c_riemann_workspace_bytes(1)
    ws, wp = _device_workspace(nb)
    _check(lib().m2c_shock_state(ctypes.byref(e), w.ctypes.data_as(ctypes.c_void_p), p1,
                                 out.ctypes.data_as(ctypes.c_void_p), wp, nb, _stream_handle(None)),
           "m2c_shock_state")
    del ws
    return tuple(out)


def m2c_residual_noalloc(n, h, bc, eos, W, phi, R, L, precision=FP64, stream=None):
    """Stage residual with no context and no workspace (library-held scratch).
    W (5, nz, ny, nx), phi, R, L: float64 device tensors. Returns the status code."""
    nx, ny, nz = n
    N = nx * ny * nz
    bcs = (ctypes.c_int * 6)(*bc)
    e0, e1 = eos_desc(eos[0]), eos_desc(eos[1])
    return lib().m2c_residual_noalloc(nx, ny, nz, h, bcs, ctypes.byref(e0), ctypes.byref(e1), precision,
                                      _buf(W, 5 * N, "W", True), _buf(phi, N, "phi", True),
                                      _buf(R, 5 * N, "R", True), _buf(L, N, "L", True), _stream_handle(stream))


def m2c_residual_noalloc_scratch_bytes() -> int:
    return lib().m2c_residual_noalloc_scratch_bytes()


@dataclass
class StepStats:
    interface_faces: int
    interface_cells: int
    flipped_cells: int
    dt: float


class Grid:
    """A context with its borrowed device state and workspace (torch tensors)."""

    def __init__(self, n, h, bc, eos, precision=FP64, cfl=0.5, reinit_every=10, reinit_iters=5,
                 device="cuda", stream=None, options=None):
        """options: None (TVD RK2, modified van Albada, HLLC, CFL time step, Cartesian) or a
        dict of m2c_set_options fields (rk, limiter, flux, mc_alpha, dt_fixed, geom, x0, band_beta,
        band_gamma);
        rk = 3 sizes the workspace for the second stage state."""
        import torch
        self.torch = torch
        self.n = tuple(n)
        nx, ny, nz = self.n
        self.N = nx * ny * nz
        self.h = h
        self.precision = precision
        self.device = torch.device(device)
        self.stream = stream
        opts = dict(rk=2, limiter=LIM_VAN_ALBADA, flux=FLUX_HLLC, mc_alpha=1.2, dt_fixed=0.0,
                    geom=GEOM_CARTESIAN, x0=0.0, band_beta=0.0, band_gamma=0.0)
        opts.update(options or {})
        wsb = m2c_workspace_bytes_rk(nx, ny, nz, precision, opts["rk"])
        self.workspace = torch.empty(wsb + 256, dtype=torch.uint8, device=self.device)
        off = (-self.workspace.data_ptr()) % 256
        self._ws_ptr = ctypes.c_void_p(self.workspace.data_ptr() + off)
        self.W = torch.zeros((5, nz, ny, nx), dtype=torch.float64, device=self.device)
        self.phi = torch.zeros((nz, ny, nx), dtype=torch.float64, device=self.device)
        bcs = (ctypes.c_int * 6)(*bc)
        lo = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
        ctx = ctypes.c_void_p()
        code = lib().m2c_init_grid(ctypes.byref(ctx), nx, ny, nz, lo, h, bcs, precision, self._ws_ptr, wsb,
                                   _stream_handle(stream))
        _check(code, "m2c_init_grid")
        self.ctx = ctx
        for m in (0, 1):
            t, prm = eos[m]
            arr = (ctypes.c_double * 6)(*(list(prm) + [0.0] * (6 - len(prm))))
            _check(lib().m2c_set_eos(ctx, m, t, arr, len(prm)), "m2c_set_eos", ctx)
        _check(lib().m2c_set_scheme(ctx, cfl, reinit_every, reinit_iters), "m2c_set_scheme", ctx)
        if options:
            self.set_options(**opts)

    def set_options(self, rk=2, limiter=LIM_VAN_ALBADA, flux=FLUX_HLLC, mc_alpha=1.2, dt_fixed=0.0,
                    geom=GEOM_CARTESIAN, x0=0.0, band_beta=0.0, band_gamma=0.0):
        o = Options(rk, limiter, flux, mc_alpha, dt_fixed, geom, x0, band_beta, band_gamma)
        _check(lib().m2c_set_options(self.ctx, ctypes.byref(o)), "m2c_set_options", self.ctx)

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx is not None and _lib is not None:
            _lib.m2c_destroy(ctx)
            self.ctx = None

    def set_tiling(self, tile_rows=8, tile_z=0):
        _check(lib().m2c_set_tiling(self.ctx, tile_rows, tile_z), "m2c_set_tiling", self.ctx)

    def set_riemann_start(self, fp32_start=True):
        _check(lib().m2c_set_riemann_start(self.ctx, 1 if fp32_start else 0), "m2c_set_riemann_start", self.ctx)

    # -- state
    def set_state(self, W=None, phi=None, t=0.0, step=0):
        torch = self.torch
        if W is not None:
            self.W.copy_(torch.as_tensor(W, dtype=torch.float64))
        if phi is not None:
            self.phi.copy_(torch.as_tensor(phi, dtype=torch.float64))
        _check(lib().m2c_set_state(self.ctx, _ptr(self.W), _ptr(self.phi), t, step), "m2c_set_state", self.ctx)

    def set_prims(self, prims, phi, t=0.0, step=0):
        """State from primitive fields (5, nz, ny, nx) and phi, converted on the device."""
        torch = self.torch
        self.phi.copy_(torch.as_tensor(phi, dtype=torch.float64))
        _check(lib().m2c_set_state(self.ctx, _ptr(self.W), _ptr(self.phi), t, step), "m2c_set_state", self.ctx)
        P = torch.as_tensor(prims, dtype=torch.float64).to(self.device).contiguous()
        _check(lib().m2c_prims_to_state(self.ctx, _buf(P, 5 * self.N, "prims", True)), "m2c_prims_to_state",
               self.ctx)

    def prims(self):
        """Primitive fields (5, nz, ny, nx) of the current state (device tensor, FP64)."""
        torch = self.torch
        nx, ny, nz = self.n
        P = torch.empty((5, nz, ny, nx), dtype=torch.float64, device=self.device)
        _check(lib().m2c_state_to_prims(self.ctx, _ptr(P)), "m2c_state_to_prims", self.ctx)
        return P

    def _host_state(self, W_host, phi_host):
        return _buf(W_host, 5 * self.N, "W_host", False), _buf(phi_host, self.N, "phi_host", False)

    def upload(self, W_host, phi_host):
        _check(lib().m2c_upload_state(self.ctx, *self._host_state(W_host, phi_host)), "m2c_upload_state", self.ctx)

    def download(self, W_host, phi_host):
        _check(lib().m2c_download_state(self.ctx, *self._host_state(W_host, phi_host)), "m2c_download_state",
               self.ctx)

    # -- stepping
    def step(self, nsteps=1):
        _check(lib().m2c_step(self.ctx, nsteps), "m2c_step", self.ctx)

    def step_host(self, W_host, phi_host, nsteps=1):
        """m2c_step_host: upload the state from the (pinned) host arrays, step, download it back
        into them; asynchronous (sync() waits)."""
        _check(lib().m2c_step_host(self.ctx, *self._host_state(W_host, phi_host), nsteps), "m2c_step_host", self.ctx)

    def sync(self):
        t = ctypes.c_double()
        s = ctypes.c_long()
        e = ctypes.c_long()
        code = lib().m2c_sync(self.ctx, ctypes.byref(t), ctypes.byref(s), ctypes.byref(e))
        if code != M2C_OK:
            raise M2CError(code, "m2c_sync", lib().m2c_last_error(self.ctx).decode())
        return t.value, s.value

    def sync_status(self):
        t = ctypes.c_double()
        s = ctypes.c_long()
        e = ctypes.c_long()
        code = lib().m2c_sync(self.ctx, ctypes.byref(t), ctypes.byref(s), ctypes.byref(e))
        return code, e.value

    def stats(self) -> StepStats:
        st = Stats()
        _check(lib().m2c_get_stats(self.ctx, ctypes.byref(st)), "m2c_get_stats", self.ctx)
        return StepStats(st.interface_faces, st.interface_cells, st.flipped_cells, st.dt)

    def profile(self, enable=True, bulk_only=False):
        mode = (2 if bulk_only else 1) if enable else 0
        _check(lib().m2c_profile(self.ctx, mode), "m2c_profile", self.ctx)

    def profile_read(self):
        ms = ctypes.c_double()
        n = ctypes.c_long()
        _check(lib().m2c_profile_read(self.ctx, ctypes.byref(ms), ctypes.byref(n)), "m2c_profile_read", self.ctx)
        return ms.value, n.value

    KERNEL_KINDS = ("stage", "fiver", "finish", "reinit", "phase_fix", "end_step")

    def profile_read_kernels(self):
        """{kernel kind: (total ms, launches)} since profiling was enabled or last read."""
        ms = (ctypes.c_double * 6)()
        n = (ctypes.c_long * 6)()
        _check(lib().m2c_profile_read_kernels(self.ctx, ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(n, ctypes.c_void_p)),
               "m2c_profile_read_kernels", self.ctx)
        return {k: (ms[i], n[i]) for i, k in enumerate(self.KERNEL_KINDS)}

    def residual(self):
        torch = self.torch
        nx, ny, nz = self.n
        R = torch.zeros((5, nz, ny, nx), dtype=torch.float64, device=self.device)
        L = torch.zeros((nz, ny, nx), dtype=torch.float64, device=self.device)
        _check(lib().m2c_residual(self.ctx, _ptr(R), _ptr(L)), "m2c_residual", self.ctx)
        return R, L


class Batch:
    """Several Grid contexts stepped together (one launch per kernel for all of them).
    tuning = (tile rows 4|8|16 (16: mixed precision only), tile z-length (0 auto),
    schedule 0 static | 1 dynamic, blocks per SM of a persistent grid (0 = one block per tile))."""

    def __init__(self, grids, tuning=(8, 0, 0, 0)):
        import torch
        self.grids = list(grids)
        k = len(self.grids)
        nb = m2c_batch_workspace_bytes(k)
        self.ws = torch.empty(nb + 256, dtype=torch.uint8, device=self.grids[0].device)
        off = (-self.ws.data_ptr()) % 256
        arr = (ctypes.c_void_p * k)(*[g.ctx.value for g in self.grids])
        tun = (ctypes.c_int * 4)(*tuning)
        b = ctypes.c_void_p()
        code = lib().m2c_batch_create(ctypes.byref(b), arr, k, ctypes.c_void_p(self.ws.data_ptr() + off), nb, tun)
        _check(code, "m2c_batch_create", self.grids[0].ctx)
        self.b = b
        self.graph = None
        self.graph_steps = 0

    def step(self, nsteps):
        _check(lib().m2c_batch_step(self.b, nsteps), "m2c_batch_step", self.grids[0].ctx)

    def capture(self, nsteps):
        if self.graph is not None:
            lib().m2c_graph_destroy(self.graph)
            self.graph = None
        g = ctypes.c_void_p()
        _check(lib().m2c_batch_capture(self.b, nsteps, ctypes.byref(g)), "m2c_batch_capture", self.grids[0].ctx)
        self.graph = g
        self.graph_steps = nsteps

    def launch_graph(self):
        _check(lib().m2c_batch_launch_graph(self.b, self.graph), "m2c_batch_launch_graph", self.grids[0].ctx)

    def __del__(self):
        if _lib is not None:
            if getattr(self, "graph", None) is not None:
                _lib.m2c_graph_destroy(self.graph)
                self.graph = None
            if getattr(self, "b", None) is not None:
                _lib.m2c_batch_destroy(self.b)
                self.b = None
