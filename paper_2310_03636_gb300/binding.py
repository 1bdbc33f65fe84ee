"""Thin ctypes binding of libgpe.so (include/gpe.h).  Argument marshalling only: every
step of the split-step path runs in the library's CUDA kernels.  Torch is used for
device memory and streams.  There is no fallback: if the library is missing, importing
this module raises.
"""
import ctypes
import math
import os

import numpy as np
import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libgpe.so")

GPE_OK, GPE_EINVAL, GPE_ENOMEM, GPE_ECUDA, GPE_ETIMEOUT, GPE_ENONFINITE, GPE_EUNSUPPORTED = range(7)
GPE_C64, GPE_C128 = 0, 1
GPE_OBS_SPECTRA, GPE_OBS_DIAG, GPE_OBS_WINDING = 1, 2, 4
GPE_INTEGRATOR_PAPER, GPE_INTEGRATOR_ROTATION = 0, 1
STATUS_NAMES = {0: "GPE_OK", 1: "GPE_EINVAL", 2: "GPE_ENOMEM", 3: "GPE_ECUDA", 4: "GPE_ETIMEOUT",
                5: "GPE_ENONFINITE", 6: "GPE_EUNSUPPORTED"}


class gpe_traj(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("n", ctypes.c_int32 * 3), ("dx", ctypes.c_double),
                ("psi", ctypes.c_void_p)]


class gpe_params(ctypes.Structure):
    _fields_ = [("c0", ctypes.c_double), ("c1", ctypes.c_double), ("q", ctypes.c_double),
                ("dt", ctypes.c_double), ("q_knots", ctypes.POINTER(ctypes.c_double)),
                ("n_knots", ctypes.c_int32), ("t_end", ctypes.c_double)]


class GPEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is not built; run __graft_entry__.build() first")
    lib = ctypes.CDLL(_LIB_PATH)
    vp, i32, i64, u32, u64, dbl = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_double)
    pd = ctypes.POINTER(ctypes.c_double)
    sig = {
        "gpe_batch_create": ([ctypes.POINTER(gpe_traj), i32, ctypes.c_int, ctypes.POINTER(gpe_params),
                              ctypes.POINTER(vp)], ctypes.c_int),
        "gpe_batch_destroy": ([vp], ctypes.c_int),
        "tw_init_noise": ([vp, u64, pd, dbl, vp], ctypes.c_int),
        "gpe_step_batch": ([vp, i64, vp], ctypes.c_int),
        "observables_accumulate": ([vp, vp, u32, i32, vp], ctypes.c_int),
        "gpe_obs_layout": ([vp, ctypes.POINTER(i32), ctypes.POINTER(i64)], ctypes.c_int),
        "gpe_bin_counts": ([vp, ctypes.POINTER(i64)], ctypes.c_int),
        "gpe_obs_group_layout": ([vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i64)], ctypes.c_int),
        "gpe_batch_get_step": ([vp], i64),
        "gpe_batch_set_step": ([vp, i64], ctypes.c_int),
        "gpe_batch_save": ([vp, ctypes.c_char_p, vp], ctypes.c_int),
        "gpe_batch_load": ([vp, ctypes.c_char_p, vp], ctypes.c_int),
        "gpe_sync_status": ([vp, vp], ctypes.c_int),
        "gpe_profile_enable": ([vp, i32], ctypes.c_int),
        "gpe_profile_read": ([vp, pd, ctypes.POINTER(i64)], ctypes.c_int),
        "gpe_adjoint_step": ([vp, vp, vp, i64, vp, vp], ctypes.c_int),
        "gpe_adjoint_segment": ([vp, vp, vp, i64, i64, vp, vp, vp], ctypes.c_int),
        "gpe_batch_upload": ([vp, vp, vp], ctypes.c_int),
        "gpe_batch_download": ([vp, vp, vp], ctypes.c_int),
        "gpe_obs_download": ([vp, vp, i32, vp, vp], ctypes.c_int),
        "gpe_sf_band_loss": ([vp, vp, dbl, dbl, vp, vp, vp], ctypes.c_int),
        "gpe_launch_count": ([], i64),
        "gpe_batch_set_graph": ([vp, i32], ctypes.c_int),
        "gpe_batch_set_wait_limit": ([vp, i64], ctypes.c_int),
        "gpe_debug_fail_alloc": ([i64], ctypes.c_int),
        "gpe_debug_table_memory": ([i32], ctypes.c_int),
        "gpe_batch_set_integrator": ([vp, i32], ctypes.c_int),
        "gpe_batch_set_traj_base": ([vp, i64], ctypes.c_int),
        "gpe_batch_set_potential": ([vp, ctypes.POINTER(i32), vp], ctypes.c_int),
        "gpe_batch_set_autotune": ([vp, i32], ctypes.c_int),
        "gpe_batch_get_tiles": ([vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)], ctypes.c_int),
        "gpe_batch_set_tiles": ([vp, i32, i32, i32], ctypes.c_int),
        "gpe_batch_set_xpass_threads": ([vp, i32, i32], ctypes.c_int),
        "gpe_batch_get_xpass_threads": ([vp, i32, ctypes.POINTER(i32)], ctypes.c_int),
        "gpe_batch_set_lanes": ([vp, i32], ctypes.c_int),
        "gpe_batch_get_lanes": ([vp, i32, ctypes.POINTER(i32)], ctypes.c_int),
        "gpe_batch_set_mean_field": ([vp, ctypes.POINTER(i32), vp], ctypes.c_int),
        "gpe_check_sincos": ([vp, vp, i64, vp], ctypes.c_int),
        "gpe_fma_rate": ([i32, i64, ctypes.POINTER(dbl), vp], ctypes.c_int),
        "gpe_diagnostics_noalloc": ([vp, i32, i32, ctypes.POINTER(i32), dbl, ctypes.c_int, dbl, dbl, dbl, vp, vp],
                                    ctypes.c_int),
        "gpe_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


LIB = _load()


def _check(status):
    if status != GPE_OK:
        raise GPEError(status, LIB.gpe_last_error().decode())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


# ----------------------------------------------------------------- C-ABI mirrors

def gpe_batch_create(trajs, dtype, c0, c1, q, dt, q_knots=None, t_end=0.0):
    """trajs: list of (shape, dx, psi_tensor); shape slowest axis first."""
    arr = (gpe_traj * len(trajs))()
    for i, (shape, dx, psi) in enumerate(trajs):
        arr[i].ndim = len(shape)
        n = list(reversed(shape)) + [1] * (3 - len(shape))
        for a in range(3):
            arr[i].n[a] = int(n[a])
        arr[i].dx = float(dx)
        arr[i].psi = ctypes.c_void_p(psi.data_ptr())
    p = gpe_params(c0=float(c0), c1=float(c1), q=float(q), dt=float(dt))
    knots_buf = None
    if q_knots is not None:
        knots_buf = (ctypes.c_double * len(q_knots))(*[float(x) for x in q_knots])
        p.q_knots = knots_buf
        p.n_knots = len(q_knots)
        p.t_end = float(t_end)
    h = ctypes.c_void_p()
    _check(LIB.gpe_batch_create(arr, len(trajs), dtype, ctypes.byref(p), ctypes.byref(h)))
    return h


def gpe_batch_destroy(h):
    _check(LIB.gpe_batch_destroy(h))


def tw_init_noise(h, seed, mean_spinor, noise_per_mode, stream=None):
    m = (ctypes.c_double * 6)(*[float(x) for x in mean_spinor])
    _check(LIB.tw_init_noise(h, ctypes.c_uint64(int(seed)), m, float(noise_per_mode), _stream(stream)))


def gpe_step_batch(h, nsteps, stream=None):
    _check(LIB.gpe_step_batch(h, int(nsteps), _stream(stream)))


def observables_accumulate(h, acc, flags, slot, stream=None):
    assert acc.dtype == torch.float64 and acc.is_cuda and acc.is_contiguous()
    _check(LIB.observables_accumulate(h, ctypes.c_void_p(acc.data_ptr()), int(flags), int(slot), _stream(stream)))


def gpe_obs_layout(h):
    nb = ctypes.c_int32()
    sd = ctypes.c_int64()
    _check(LIB.gpe_obs_layout(h, ctypes.byref(nb), ctypes.byref(sd)))
    return nb.value, sd.value


def gpe_bin_counts(h, nbins):
    out = (ctypes.c_int64 * nbins)()
    _check(LIB.gpe_bin_counts(h, out))
    return np.array(out, dtype=np.int64)


def gpe_sync_status(h, stream=None):
    return LIB.gpe_sync_status(h, _stream(stream))


PROFILE_KINDS = ("xpass", "strided_pass", "resident1d", "noise", "observables", "adjoint")


def gpe_profile_enable(h, on=True):
    _check(LIB.gpe_profile_enable(h, 1 if on else 0))


def gpe_profile_read(h):
    ms = (ctypes.c_double * 6)()
    n = (ctypes.c_int64 * 6)()
    _check(LIB.gpe_profile_read(h, ms, n))
    return {k: (ms[i], n[i]) for i, k in enumerate(PROFILE_KINDS)}


def gpe_adjoint_step(h, psi_step_in, lam, step_index, dLdq, stream=None):
    """psi_step_in, lam: contiguous (ntraj, 3, *shape) complex CUDA tensors; dLdq: float64 CUDA."""
    for t in (psi_step_in, lam):
        assert t.is_cuda and t.is_contiguous()
    assert dLdq.dtype == torch.float64 and dLdq.is_cuda
    _check(LIB.gpe_adjoint_step(h, ctypes.c_void_p(psi_step_in.data_ptr()), ctypes.c_void_p(lam.data_ptr()),
                                int(step_index), ctypes.c_void_p(dLdq.data_ptr()), _stream(stream)))


def gpe_adjoint_segment(h, psi_ckpt, states, n0, nseg, lam, dLdq, stream=None):
    """psi_ckpt, lam: contiguous (ntraj, 3, *shape) complex CUDA tensors; states: contiguous
    CUDA tensor of at least nseg such fields; dLdq: float64 CUDA."""
    for t in (psi_ckpt, states, lam):
        assert t.is_cuda and t.is_contiguous()
    assert states.numel() >= nseg * psi_ckpt.numel() and states.dtype == psi_ckpt.dtype
    assert dLdq.dtype == torch.float64 and dLdq.is_cuda
    _check(LIB.gpe_adjoint_segment(h, ctypes.c_void_p(psi_ckpt.data_ptr()), ctypes.c_void_p(states.data_ptr()),
                                   int(n0), int(nseg), ctypes.c_void_p(lam.data_ptr()),
                                   ctypes.c_void_p(dLdq.data_ptr()), _stream(stream)))


def gpe_sf_band_loss(h, psi, kmin, kmax, loss, lam_out=None, stream=None):
    """loss: float64 CUDA tensor (>= 1 element, overwritten); lam_out: like psi or None."""
    assert psi.is_cuda and psi.is_contiguous() and loss.dtype == torch.float64 and loss.is_cuda
    lp = ctypes.c_void_p(lam_out.data_ptr()) if lam_out is not None else None
    _check(LIB.gpe_sf_band_loss(h, ctypes.c_void_p(psi.data_ptr()), float(kmin), float(kmax),
                                ctypes.c_void_p(loss.data_ptr()), lp, _stream(stream)))


def gpe_launch_count():
    return LIB.gpe_launch_count()


def gpe_diagnostics_noalloc(psi, ndim, c0, c1, q, dx, out, stream=None):
    """psi: (ntraj, 3, *shape) complex CUDA tensor; out: (ntraj * 8,) float64 CUDA tensor."""
    assert psi.is_cuda and psi.is_contiguous() and out.dtype == torch.float64 and out.is_cuda
    shape = tuple(psi.shape[2:])
    assert len(shape) == ndim
    n = (ctypes.c_int32 * 3)(*(list(reversed(shape)) + [1] * (3 - ndim)))
    dt = GPE_C64 if psi.dtype == torch.complex64 else GPE_C128
    _check(LIB.gpe_diagnostics_noalloc(ctypes.c_void_p(psi.data_ptr()), psi.shape[0], ndim, n, float(dx), dt,
                                       float(c0), float(c1), float(q), ctypes.c_void_p(out.data_ptr()),
                                       _stream(stream)))


def _grid(shape):
    shape = tuple(shape)
    return (ctypes.c_int32 * 3)(*(list(reversed(shape)) + [1] * (3 - len(shape))))


def gpe_batch_set_potential(h, shape, V):
    """V: contiguous (3, *shape) real CUDA tensor in the batch's precision, or None."""
    if V is not None:
        assert V.is_cuda and V.is_contiguous() and V.dtype in (torch.float32, torch.float64)
        assert tuple(V.shape) == (3,) + tuple(shape)
    ptr = ctypes.c_void_p(V.data_ptr()) if V is not None else None
    _check(LIB.gpe_batch_set_potential(h, _grid(shape), ptr))


def gpe_batch_set_mean_field(h, shape, field):
    """field: contiguous (3, *shape) complex128 CUDA tensor, or None."""
    if field is not None:
        assert field.is_cuda and field.is_contiguous() and field.dtype == torch.complex128
        assert tuple(field.shape) == (3,) + tuple(shape)
    ptr = ctypes.c_void_p(field.data_ptr()) if field is not None else None
    _check(LIB.gpe_batch_set_mean_field(h, _grid(shape), ptr))


def gpe_check_sincos(x, stream=None):
    """x: float32 CUDA tensor -> (n, 4) tensor: own sin, cos, library sin, cos."""
    assert x.dtype == torch.float32 and x.is_cuda and x.is_contiguous()
    out = torch.empty((x.numel(), 4), dtype=torch.float32, device=x.device)
    _check(LIB.gpe_check_sincos(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), x.numel(),
                                _stream(stream)))
    return out


def gpe_fma_rate(kind, iters, stream=None):
    """FMA throughput of the current device in flop/s (kind 0: FP32, 1: packed FP32 pairs,
    2: FP64); one timed launch of ``iters`` loop trips per thread."""
    out = ctypes.c_double(0.0)
    _check(LIB.gpe_fma_rate(int(kind), int(iters), ctypes.byref(out), _stream(stream)))
    return out.value


# ----------------------------------------------------------------- convenience

class GPEBatch:
    """A batch of trajectories whose fields live in torch device tensors.

    shapes: one spatial shape (uniform batch, one contiguous tensor of shape
    (ntraj, 3, *shape)) or a list of shapes (ragged batch, one tensor each).
    """

    def __init__(self, shape, ntraj=1, dtype="c64", c0=1.0, c1=-0.1, q=0.09, dt=0.02, dx=1.0,
                 q_knots=None, t_end=0.0, device="cuda", psi=None):
        self.dtype = GPE_C64 if dtype == "c64" else GPE_C128
        tdt = torch.complex64 if self.dtype == GPE_C64 else torch.complex128
        self.dx, self.dt, self.c0, self.c1, self.q = dx, dt, c0, c1, q
        if isinstance(shape, (list,)) and shape and isinstance(shape[0], (tuple, list)):
            self.shapes = [tuple(s) for s in shape]
            # trajectories of one shape share one allocation, back to back, so that the
            # library can use its tensor-map passes (and tune their tiles) for the group
            self._blocks = {}
            for s in dict.fromkeys(self.shapes):
                cnt = self.shapes.count(s)
                self._blocks[s] = torch.zeros((cnt, 3) + s, dtype=tdt, device=device)
            used = {s: 0 for s in self._blocks}
            self.psi = []
            for s in self.shapes:
                self.psi.append(self._blocks[s][used[s]])
                used[s] += 1
            trajs = [(s, dx, p) for s, p in zip(self.shapes, self.psi)]
            self.uniform = False
        else:
            self.shapes = [tuple(shape)] * ntraj
            if psi is None:
                psi = torch.zeros((ntraj, 3) + tuple(shape), dtype=tdt, device=device)
            assert psi.dtype == tdt and psi.is_contiguous() and psi.shape == (ntraj, 3) + tuple(shape)
            self.psi = psi
            trajs = [(tuple(shape), dx, psi[i]) for i in range(ntraj)]
            self.uniform = True
        self.ntraj = len(trajs)
        self.h = gpe_batch_create(trajs, self.dtype, c0, c1, q, dt, q_knots, t_end)

    def close(self):
        if getattr(self, "h", None):
            gpe_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_noise(self, seed, mean_spinor=(0.0, 0.0, 1.0, 0.0, 0.0, 0.0), noise_per_mode=0.5, stream=None):
        tw_init_noise(self.h, seed, mean_spinor, noise_per_mode, stream)

    def step(self, nsteps, stream=None):
        gpe_step_batch(self.h, nsteps, stream)

    def layout(self):
        return gpe_obs_layout(self.h)

    def new_accumulator(self, nslots):
        nb, sd = self.layout()
        return torch.zeros(nslots * sd, dtype=torch.float64, device=self.psi.device if self.uniform else self.psi[0].device)

    def observables(self, acc, flags=GPE_OBS_SPECTRA | GPE_OBS_DIAG, slot=0, stream=None):
        observables_accumulate(self.h, acc, flags, slot, stream)

    def group_layout(self, traj=0):
        """(nbins, spectra_offset) of trajectory traj's shape group within a slot."""
        nb = ctypes.c_int32()
        off = ctypes.c_int64()
        _check(LIB.gpe_obs_group_layout(self.h, int(traj), ctypes.byref(nb), ctypes.byref(off)))
        return nb.value, off.value

    def bin_counts(self):
        nb, _ = self.layout()
        return gpe_bin_counts(self.h, nb)

    def sync_status(self, stream=None):
        return gpe_sync_status(self.h, stream)

    @property
    def step_count(self):
        return LIB.gpe_batch_get_step(self.h)

    def set_step(self, step):
        _check(LIB.gpe_batch_set_step(self.h, int(step)))

    def save(self, path, stream=None):
        """Write a checkpoint (fields, step, configuration) to the host file ``path``."""
        _check(LIB.gpe_batch_save(self.h, os.fsencode(str(path)), _stream(stream)))

    def load(self, path, stream=None):
        """Restore fields and step from a checkpoint of a batch of this configuration."""
        _check(LIB.gpe_batch_load(self.h, os.fsencode(str(path)), _stream(stream)))

    def set_traj_base(self, base):
        _check(LIB.gpe_batch_set_traj_base(self.h, int(base)))

    def set_integrator(self, kind):
        _check(LIB.gpe_batch_set_integrator(self.h, int(kind)))

    def set_graph(self, enable=True):
        _check(LIB.gpe_batch_set_graph(self.h, 1 if enable else 0))

    def set_wait_limit(self, first_wait_polls=-1):
        """Poll limit of each pass block's first copy wait (-1: the default; 0 expires it at
        once, a test of the timeout path)."""
        _check(LIB.gpe_batch_set_wait_limit(self.h, int(first_wait_polls)))

    def set_autotune(self, enable=True):
        _check(LIB.gpe_batch_set_autotune(self.h, 1 if enable else 0))

    def set_tiles(self, cols_y, cols_z=0, traj=0):
        """Fix the strided passes' tile widths of trajectory traj's shape group (0 keeps one)."""
        _check(LIB.gpe_batch_set_tiles(self.h, int(traj), int(cols_y), int(cols_z)))

    def set_xpass_threads(self, threads, traj=0):
        """Fix the x-pass block size (128 or 256, or 192 at x extent 512; 0 = default) of
        trajectory traj's group."""
        _check(LIB.gpe_batch_set_xpass_threads(self.h, int(traj), int(threads)))

    def xpass_threads(self, traj=0):
        """Block size of the x pass in use for trajectory traj's group (0 for 1D)."""
        t = ctypes.c_int32()
        _check(LIB.gpe_batch_get_xpass_threads(self.h, int(traj), ctypes.byref(t)))
        return int(t.value)

    def upload(self, host, stream=None):
        """Copy host fields (CPU tensor holding every trajectory in batch order, back to
        back, the batch's dtype; pinned memory for an asynchronous copy) into the batch."""
        assert not host.is_cuda and host.is_contiguous()
        _check(LIB.gpe_batch_upload(self.h, ctypes.c_void_p(host.data_ptr()), _stream(stream)))

    def download(self, host, stream=None):
        """Copy the batch's fields into a host tensor laid out as for upload."""
        assert not host.is_cuda and host.is_contiguous()
        _check(LIB.gpe_batch_download(self.h, ctypes.c_void_p(host.data_ptr()), _stream(stream)))

    def download_slot(self, acc, slot, host, stream=None):
        """Copy accumulator slot ``slot`` of the device tensor acc into the host tensor host."""
        assert acc.is_cuda and acc.dtype == torch.float64 and not host.is_cuda and host.dtype == torch.float64
        _check(LIB.gpe_obs_download(self.h, ctypes.c_void_p(acc.data_ptr()), int(slot),
                                    ctypes.c_void_p(host.data_ptr()), _stream(stream)))

    def set_lanes(self, lanes=-1):
        """Trajectory lanes per 2D/3D shape group (-1: the default, 1: off, at most 64)."""
        _check(LIB.gpe_batch_set_lanes(self.h, int(lanes)))

    def lanes(self, traj=0):
        """Lanes the shape group of trajectory traj is stepped in."""
        n = ctypes.c_int32()
        _check(LIB.gpe_batch_get_lanes(self.h, int(traj), ctypes.byref(n)))
        return int(n.value)

    def tiles(self, traj=0):
        """(cols_y, cols_z, tuned) of the column passes of trajectory traj's group."""
        cols = (ctypes.c_int32 * 2)()
        tuned = ctypes.c_int32()
        _check(LIB.gpe_batch_get_tiles(self.h, int(traj), cols, ctypes.byref(tuned)))
        return int(cols[0]), int(cols[1]), bool(tuned.value)

    def set_potential(self, V, shape=None):
        """V_m(x) for the trajectories on grid ``shape`` (default: the batch's first shape).
        V: (3, *shape) tensor (moved to the device in the batch's real precision) or None.
        The batch keeps a reference while it is set."""
        shape = tuple(shape) if shape is not None else self.shapes[0]
        if V is not None:
            rdt = torch.float32 if self.dtype == GPE_C64 else torch.float64
            dev = self.psi.device if self.uniform else self.psi[0].device
            V = torch.as_tensor(V).to(device=dev, dtype=rdt).contiguous()
        gpe_batch_set_potential(self.h, shape, V)
        if not hasattr(self, "_pot"):
            self._pot = {}
        self._pot[shape] = V

    def set_mean_field(self, field, shape=None):
        """Mean field added to the mean spinor by init_noise on grid ``shape``:
        (3, *shape) complex tensor (held as complex128 on the device) or None."""
        shape = tuple(shape) if shape is not None else self.shapes[0]
        if field is not None:
            dev = self.psi.device if self.uniform else self.psi[0].device
            field = torch.as_tensor(field).to(device=dev, dtype=torch.complex128).contiguous()
        gpe_batch_set_mean_field(self.h, shape, field)
        if not hasattr(self, "_mf"):
            self._mf = {}
        self._mf[shape] = field


def unpack_slot(acc_slot, nbins, ntraj):
    """Split one accumulator slot into spectra (4, nbins) and diagnostics (ntraj, 8)."""
    a = acc_slot.detach().cpu().numpy() if torch.is_tensor(acc_slot) else np.asarray(acc_slot)
    spec = a[:4 * nbins].reshape(4, nbins) if nbins > 0 else np.zeros((4, 0))
    diag = a[4 * max(nbins, 0):4 * max(nbins, 0) + 8 * ntraj].reshape(ntraj, 8)
    return spec, diag


def unpack_winding(acc_slot, nbins, ntraj):
    """Per-trajectory winding numbers Q_w / 2 pi of one accumulator slot."""
    a = acc_slot.detach().cpu().numpy() if torch.is_tensor(acc_slot) else np.asarray(acc_slot)
    o = 4 * max(nbins, 0) + 8 * ntraj
    return a[o:o + ntraj].copy()
