"""GB300 (sm_103a) D3Q27 neural-collision lattice Boltzmann library (arXiv 2412.08229).

The compute path is the C-ABI library built from csrc/ (see include/lbm.h). This
package is a thin binding with the same names: each function marshals its arguments
(torch tensors on the GPU or the host, or numpy arrays on the host) into pointers and
calls the library. Nothing is computed here.
"""

import ctypes

import numpy as np

from . import _abi
from ._abi import LbmError, OPS, STORAGES, NETS, BOUNDARIES  # noqa: F401

__all__ = [
    "lbm_create", "lbm_destroy", "lbm_init", "lbm_set_state", "lbm_get_state", "lbm_step",
    "lbm_check", "lbm_set_wait_limit", "lbm_macroscopic", "lbm_kinetic_energy", "lbm_energy_spectrum",
    "nco_set_weights", "lbm_force_draws", "lbm_get_raw_state", "lbm_set_raw_state", "lbm_get_force_state",
    "lbm_set_force_state", "lbm_check_guards", "lbm_selftest_guards", "lbm_group_tables", "lbm_spectrum_shells",
    "lbm_tgv_reduced_table", "lbm_version", "LbmContext",
    "lbm_selftest_tensor_cores", "lbm_kinetic_energy_noalloc", "lbm_record_begin", "nco_backward",
    "nco_backward_ke",
    "LbmError", "LbmBatch", "lbm_batch_create", "lbm_batch_get", "lbm_batch_set_weights",
    "lbm_batch_autotune", "lbm_batch_set_tile_shape", "lbm_batch_step", "lbm_batch_check", "lbm_batch_destroy",
]


def _ptr(x, dtype):
    """Raw pointer of a contiguous tensor/array of the given numpy dtype (no copies)."""
    if x is None:
        return None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            want = {np.float32: torch.float32, np.float64: torch.float64}[dtype]
            if x.dtype != want or not x.is_contiguous():
                raise TypeError(f"expected a contiguous {want} tensor, got {x.dtype}")
            return ctypes.c_void_p(x.data_ptr())
    except ImportError:
        pass
    if isinstance(x, np.ndarray):
        if x.dtype != dtype or not x.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a C-contiguous {np.dtype(dtype)} array, got {x.dtype}")
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(x)}")


class LbmContext:
    """Owner of an lbm_ctx* (destroyed with the object), or a view of a batch instance."""

    def __init__(self, handle, cfg, owner=None):
        self.handle = handle
        self.cfg = cfg
        self.owner = owner  # the LbmBatch that owns the context, if any

    @property
    def shape(self):
        return (self.cfg.nz, self.cfg.ny, self.cfg.nx)

    @property
    def ncell(self):
        return self.cfg.nx * self.cfg.ny * self.cfg.nz

    def __del__(self):
        try:
            if self.handle and self.owner is None:
                _abi.load().lbm_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


def _config(nx, ny, nz, nu, op="bgk", storage="f32", net="f32", boundary="periodic", forcing=None,
            rho_window=(0.0, 0.0)):
    cfg = _abi.lbm_config()
    cfg.nx, cfg.ny, cfg.nz = int(nx), int(ny), int(nz)
    cfg.nu = float(nu)
    cfg.op = OPS[op]
    cfg.storage = STORAGES[storage]
    cfg.net_precision = NETS[net]
    cfg.boundary = BOUNDARIES[boundary]
    if forcing:
        cfg.forcing = 1
        cfg.force_power = float(forcing["power"])
        cfg.force_kf = float(forcing.get("kf", 1.5))
        cfg.force_c = float(forcing.get("c", 0.5))
        cfg.force_ka = float(forcing.get("ka", 1.0))
        cfg.force_kb = float(forcing.get("kb", 2.0))
    cfg.rho_min, cfg.rho_max = (float(v) for v in rho_window)
    return cfg


def lbm_create(nx, ny, nz, nu, op="bgk", storage="f32", net="f32", boundary="periodic",
               forcing=None, rho_window=(0.0, 0.0), stream=None):
    """lbm_create: forcing is None or a dict(power, kf, c, ka, kb)."""
    lib = _abi.load()
    cfg = _config(nx, ny, nz, nu, op, storage, net, boundary, forcing, rho_window)
    handle = ctypes.c_void_p()
    st = lib.lbm_create(ctypes.byref(cfg), stream if stream is not None else _current_stream(),
                        ctypes.byref(handle))
    _abi.check(st, None, "lbm_create")
    return LbmContext(handle, cfg)


def lbm_destroy(ctx):
    if ctx.owner is not None:
        raise ValueError("lbm_destroy: this context belongs to a batch (lbm_batch_destroy frees it)")
    if ctx.handle:
        _abi.check(_abi.load().lbm_destroy(ctx.handle))
        ctx.handle = None


def lbm_init(ctx, rho, u):
    _abi.check(_abi.load().lbm_init(ctx.handle, _ptr(rho, np.float32), _ptr(u, np.float32)), ctx.handle, "lbm_init")


def lbm_set_state(ctx, f):
    _abi.check(_abi.load().lbm_set_state(ctx.handle, _ptr(f, np.float32)), ctx.handle, "lbm_set_state")


def lbm_get_state(ctx, f):
    _abi.check(_abi.load().lbm_get_state(ctx.handle, _ptr(f, np.float32)), ctx.handle, "lbm_get_state")


def lbm_step(ctx, nsteps=1):
    _abi.check(_abi.load().lbm_step(ctx.handle, int(nsteps)), ctx.handle, "lbm_step")


def lbm_check(ctx):
    """Returns the status (LBM_OK or LBM_ERR_UNSTABLE); raises on other errors."""
    st = _abi.load().lbm_check(ctx.handle)
    if st not in (_abi.LBM_OK, _abi.LBM_ERR_UNSTABLE):
        _abi.check(st, ctx.handle, "lbm_check")
    return st


def lbm_check_guards(ctx):
    """Raises if a guard region around the population buffers was overwritten."""
    _abi.check(_abi.load().lbm_check_guards(ctx.handle), ctx.handle, "lbm_check_guards")


def lbm_selftest_guards(ctx):
    """Raises unless a changed guard byte is reported and a restored one is not."""
    _abi.check(_abi.load().lbm_selftest_guards(ctx.handle), ctx.handle, "lbm_selftest_guards")


def lbm_set_wait_limit(ctx, cycles):
    """Limit (SM clock cycles) of the tensor-core step kernels' MMA-completion waits; 0 gives up at once."""
    _abi.check(_abi.load().lbm_set_wait_limit(ctx.handle, int(cycles)), ctx.handle, "lbm_set_wait_limit")


def lbm_macroscopic(ctx, rho, u):
    _abi.check(_abi.load().lbm_macroscopic(ctx.handle, _ptr(rho, np.float32), _ptr(u, np.float32)),
               ctx.handle, "lbm_macroscopic")


def lbm_kinetic_energy(ctx, ke=None):
    """Returns the kinetic energy as a float when ke is None, else writes into ke (1 double)."""
    out = ke if ke is not None else np.zeros(1, dtype=np.float64)
    _abi.check(_abi.load().lbm_kinetic_energy(ctx.handle, _ptr(out, np.float64)), ctx.handle, "lbm_kinetic_energy")
    return float(out[0]) if ke is None else None


def lbm_energy_spectrum(ctx, E, nbins=None, ke=None):
    nbins = int(nbins if nbins is not None else E.shape[0])
    _abi.check(_abi.load().lbm_energy_spectrum(ctx.handle, _ptr(E, np.float64), nbins, _ptr(ke, np.float64)),
               ctx.handle, "lbm_energy_spectrum")


def nco_set_weights(ctx, theta):
    n = int(theta.shape[0])
    _abi.check(_abi.load().nco_set_weights(ctx.handle, _ptr(theta, np.float32), n), ctx.handle, "nco_set_weights")


def lbm_record_begin(ctx, k):
    _abi.check(_abi.load().lbm_record_begin(ctx.handle, int(k)), ctx.handle, "lbm_record_begin")


def nco_backward(ctx, dL_du=None, dL_drho=None, dL_dtheta=None, dL_df0=None):
    _abi.check(_abi.load().nco_backward(ctx.handle, _ptr(dL_du, np.float32), _ptr(dL_drho, np.float32),
                                        _ptr(dL_dtheta, np.float32), _ptr(dL_df0, np.float32)),
               ctx.handle, "nco_backward")


def nco_backward_ke(ctx, obs_step, dL_dk, dL_du=None, dL_drho=None, dL_dtheta=None, dL_df0=None):
    """obs_step: step counts since lbm_record_begin; dL_dk: the loss cotangent of k at each."""
    steps = np.ascontiguousarray(np.asarray(obs_step, dtype=np.int64).astype(np.int32))
    dk = np.ascontiguousarray(np.asarray(dL_dk, dtype=np.float64))
    if steps.shape != dk.shape or steps.ndim != 1:
        raise ValueError("obs_step and dL_dk must be 1-D and of the same length")
    _abi.check(_abi.load().nco_backward_ke(ctx.handle, int(steps.size), ctypes.c_void_p(steps.ctypes.data),
                                           ctypes.c_void_p(dk.ctypes.data), _ptr(dL_du, np.float32),
                                           _ptr(dL_drho, np.float32), _ptr(dL_dtheta, np.float32),
                                           _ptr(dL_df0, np.float32)),
               ctx.handle, "nco_backward_ke")


def lbm_force_draws(ctx, phi, psi):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    _abi.check(_abi.load().lbm_force_draws(ctx.handle, _ptr(phi, np.float64), _ptr(psi, np.float64),
                                           int(phi.shape[0])), ctx.handle, "lbm_force_draws")


def lbm_get_raw_state(ctx):
    """The stored state byte for byte (host uint8 array of lbm_raw_state_bytes)."""
    n = int(_abi.load().lbm_raw_state_bytes(ctx.handle))
    buf = np.empty(n, dtype=np.uint8)
    _abi.check(_abi.load().lbm_get_raw_state(ctx.handle, _ptr(buf, np.uint8)), ctx.handle, "lbm_get_raw_state")
    return buf


def lbm_set_raw_state(ctx, buf):
    """Restores lbm_get_raw_state's bytes into a context of the same grid and storage."""
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    if buf.size != int(_abi.load().lbm_raw_state_bytes(ctx.handle)):
        raise ValueError("lbm_set_raw_state: size does not match the context")
    _abi.check(_abi.load().lbm_set_raw_state(ctx.handle, _ptr(buf, np.uint8)), ctx.handle, "lbm_set_raw_state")


def lbm_get_force_state(ctx):
    """The forcing state of a forced context (96 fixed-point projection sums, int64)."""
    sums = np.zeros(96, dtype=np.int64)
    _abi.check(_abi.load().lbm_get_force_state(ctx.handle, _ptr(sums, np.int64)), ctx.handle, "lbm_get_force_state")
    return sums


def lbm_set_force_state(ctx, sums):
    """Restores lbm_get_force_state's sums (after lbm_set_state, to resume a forced run)."""
    sums = np.ascontiguousarray(sums, dtype=np.int64)
    if sums.shape != (96,):
        raise ValueError("lbm_set_force_state: 96 sums expected")
    _abi.check(_abi.load().lbm_set_force_state(ctx.handle, _ptr(sums, np.int64)), ctx.handle, "lbm_set_force_state")


def lbm_group_tables():
    """The library's own O_h tables: R (48,3,3), vperm, mperm, msign (48,27) int32."""
    R = np.zeros((48, 9), dtype=np.int32)
    vp = np.zeros((48, 27), dtype=np.int32)
    mp = np.zeros((48, 27), dtype=np.int32)
    ms = np.zeros((48, 27), dtype=np.int32)
    _abi.check(_abi.load().lbm_group_tables(R.ctypes.data, vp.ctypes.data, mp.ctypes.data, ms.ctypes.data))
    return R.reshape(48, 3, 3), vp, mp, ms


def lbm_tgv_reduced_table():
    """The library's reduced Taylor-Green symmetry table: A (27,3,3), k (27,3), pmap (27,27) int32."""
    A = np.zeros((27, 9), dtype=np.int32)
    k = np.zeros((27, 3), dtype=np.int32)
    pm = np.zeros((27, 27), dtype=np.int32)
    _abi.check(_abi.load().lbm_tgv_reduced_table(A.ctypes.data, k.ctypes.data, pm.ctypes.data))
    return A.reshape(27, 3, 3), k, pm


def lbm_spectrum_shells(nx, ny, nz):
    """Spectrum shell of every wave vector of an nx x ny x nz box, (nz, ny, nx) int32 in
    FFT order, from the library's device binning code."""
    out = np.zeros((int(nz), int(ny), int(nx)), dtype=np.int32)
    _abi.check(_abi.load().lbm_spectrum_shells(int(nx), int(ny), int(nz), out.ctypes.data), None,
               "lbm_spectrum_shells")
    return out


def lbm_kinetic_energy_noalloc(f, nx, ny, nz, ke, stream=None):
    """Kinetic energy of caller-held device populations into a caller-held device double,
    with no allocation in the library (see include/lbm.h). Raises LbmError on failure."""
    st = _abi.load().lbm_kinetic_energy_noalloc(_ptr(f, np.float32), int(nx), int(ny), int(nz),
                                                 _ptr(ke, np.float64),
                                                 stream if stream is not None else _current_stream())
    _abi.check(st, None, "lbm_kinetic_energy_noalloc")


def lbm_selftest_tensor_cores():
    """Run the tcgen05 GEMM self-test; returns the largest absolute error (0.0 expected)."""
    err = ctypes.c_double(0.0)
    _abi.check(_abi.load().lbm_selftest_tensor_cores(ctypes.byref(err)), None, "lbm_selftest_tensor_cores")
    return err.value


def lbm_version():
    return _abi.load().lbm_version().decode()


class LbmBatch:
    """Owner of an lbm_batch* (destroyed with the object) and views of its instances."""

    def __init__(self, handle, cfgs):
        self.handle = handle
        self.instances = [None] * len(cfgs)
        self.cfgs = cfgs

    def __len__(self):
        return len(self.cfgs)

    def __getitem__(self, i):
        return lbm_batch_get(self, i)

    def __del__(self):
        try:
            if self.handle:
                _abi.load().lbm_batch_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def lbm_batch_create(specs, stream=None):
    """lbm_batch_create: specs is a list of dicts with the keyword arguments of lbm_create
    (nx, ny, nz, nu, storage, forcing, rho_window); op, net and boundary are fixed to the
    batched form (NCO, BF16 network, periodic)."""
    lib = _abi.load()
    n = len(specs)
    arr = (_abi.lbm_config * n)()
    for i, sp in enumerate(specs):
        sp = dict(sp)
        sp.setdefault("op", "nco")
        sp.setdefault("net", "bf16")
        arr[i] = _config(**sp)
    handle = ctypes.c_void_p()
    st = lib.lbm_batch_create(n, arr, stream if stream is not None else _current_stream(), ctypes.byref(handle))
    _abi.check(st, None, "lbm_batch_create")
    return LbmBatch(handle, [arr[i] for i in range(n)])


def lbm_batch_get(batch, i):
    """The i-th instance as an LbmContext view (for lbm_init, lbm_force_draws, ...)."""
    if batch.instances[i] is None:
        h = ctypes.c_void_p()
        _abi.check(_abi.load().lbm_batch_get(batch.handle, int(i), ctypes.byref(h)), batch=batch.handle,
                   what="lbm_batch_get")
        batch.instances[i] = LbmContext(h, batch.cfgs[i], owner=batch)
    return batch.instances[i]


def lbm_batch_set_weights(batch, theta):
    n = theta.numel() if hasattr(theta, "numel") else theta.size
    _abi.check(_abi.load().lbm_batch_set_weights(batch.handle, _ptr(theta, np.float32), int(n)),
               batch=batch.handle, what="lbm_batch_set_weights")


def lbm_batch_autotune(batch):
    """Returns the chosen tile shape: 0 (pairs of group elements across two warpgroups) or
    2, 3, 4 (chunks of four elements per warpgroup, that many warpgroups per SM)."""
    choice = ctypes.c_int(0)
    _abi.check(_abi.load().lbm_batch_autotune(batch.handle, ctypes.byref(choice)), batch=batch.handle,
               what="lbm_batch_autotune")
    return choice.value


def lbm_batch_set_tile_shape(batch, shape):
    _abi.check(_abi.load().lbm_batch_set_tile_shape(batch.handle, int(shape)), batch=batch.handle,
               what="lbm_batch_set_tile_shape")


def lbm_batch_step(batch, nsteps=1, use_graph=True):
    _abi.check(_abi.load().lbm_batch_step(batch.handle, int(nsteps), int(bool(use_graph))), batch=batch.handle,
               what="lbm_batch_step")


def lbm_batch_check(batch):
    """Returns the status (LBM_OK or LBM_ERR_UNSTABLE); raises on other errors."""
    st = _abi.load().lbm_batch_check(batch.handle)
    if st not in (_abi.LBM_OK, _abi.LBM_ERR_UNSTABLE):
        _abi.check(st, batch=batch.handle, what="lbm_batch_check")
    return st


def lbm_batch_destroy(batch):
    if batch.handle:
        for v in batch.instances:
            if v is not None:
                v.handle = None
        _abi.check(_abi.load().lbm_batch_destroy(batch.handle))
        batch.handle = None
