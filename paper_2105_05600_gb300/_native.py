"""ctypes binding of librosefusion.so (include/rosefusion.h, include/rf_proposal.h).

Argument marshalling only: every function here has the name of the C entry
point it calls, turns torch tensors into device pointers and numpy arrays into
host pointers, and raises RfError when the library returns a status < 0.  No
tracking arithmetic happens in Python.  If the compiled library is missing
this module raises at import time; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librosefusion.so")

RF_OK, RF_ERR_ARG, RF_ERR_CUDA, RF_ERR_TIMEOUT, RF_ERR_EMPTY, RF_ERR_NOMEM = 0, -1, -2, -3, -4, -5
RF_OVERLAP, RF_NORMALIZE, RF_COMPENSATED, RF_NEAREST, RF_RHO_REF_CENTER, RF_L1, RF_RIGHT_MULT = 1, 2, 4, 8, 16, 32, 64
RF_CELL_MARGIN = 128
RF_APS_WITH_CENTRE = 256
RF_DEFAULT_FLAGS = RF_OVERLAP | RF_NORMALIZE | RF_COMPENSATED | RF_CELL_MARGIN
RF_MAX_ITERS = 64
DTYPES = {"f32": 0, "f16": 1, "i16": 2}


class RfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"librosefusion status {status}: {msg}")
        self.status = status


class rf_intrinsics(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int), ("height", ctypes.c_int), ("z_min", ctypes.c_float),
                ("z_max", ctypes.c_float)]


class rf_pose(ctypes.Structure):
    _fields_ = [("q", ctypes.c_float * 4), ("t", ctypes.c_float * 3)]


class rf_params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_float), ("beta", ctypes.c_float), ("eps", ctypes.c_float),
                ("stop_eps", ctypes.c_float), ("k_max", ctypes.c_int), ("flags", ctypes.c_int),
                ("stride", ctypes.c_int), ("reserved", ctypes.c_int)]


class rf_iter_stats(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("n_overlap", ctypes.c_int), ("n_aps", ctypes.c_int), ("argmax", ctypes.c_int),
                ("rho_ref", ctypes.c_float), ("rho_tilde", ctypes.c_float), ("rho_max", ctypes.c_float),
                ("rho_second", ctypes.c_float), ("pose", ctypes.c_float * 7), ("scale", ctypes.c_float * 6),
                ("offset", ctypes.c_float * 6), ("stop", ctypes.c_int), ("level", ctypes.c_int),
                ("n_particles", ctypes.c_int), ("corner", ctypes.c_int)]


class rf_launch_config(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int), ("work_warps", ctypes.c_int), ("group", ctypes.c_int),
                ("ms", ctypes.c_float)]


class rf_frame_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("n_points", ctypes.c_int),
                ("reserved", ctypes.c_int), ("lookups", ctypes.c_longlong), ("r1", ctypes.c_float * 6),
                ("pad", ctypes.c_float * 2), ("it", rf_iter_stats * RF_MAX_ITERS)]


class rf_track_options(ctypes.Structure):
    _fields_ = [("init_pose_dev", ctypes.c_void_p), ("scale_dev", ctypes.c_void_p), ("run_flag_dev", ctypes.c_void_p),
                ("k_max", ctypes.c_int), ("reserved", ctypes.c_int)]


class rf_proposal_params(ctypes.Structure):
    _fields_ = [("k_learned", ctypes.c_int), ("k_fallback", ctypes.c_int), ("kappa", ctypes.c_float),
                ("theta", ctypes.c_float), ("r_min", ctypes.c_float * 6), ("r_max", ctypes.c_float * 6),
                ("resume", ctypes.c_int), ("stuck", ctypes.c_int)]


class rf_learned_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("used_fallback", ctypes.c_int), ("chose_fallback", ctypes.c_int),
                ("iters_learned", ctypes.c_int), ("iters_fallback", ctypes.c_int), ("rho_learned", ctypes.c_float),
                ("rho_fallback", ctypes.c_float), ("rho_prev", ctypes.c_float), ("init_pose", ctypes.c_float * 7),
                ("r0", ctypes.c_float * 6), ("lookups", ctypes.c_longlong)]


RF_MLP_IN, RF_MLP_IN_USED, RF_MLP_HIDDEN, RF_MLP_OUT, RF_MLP_OUT_USED = 832, 774, 256, 16, 12
RF_MLP_MAX_BATCH, RF_MLP_MAX_TRAIN_BATCH = 4096, 1024
RF_MLP_EVAL_STATS = 13

EXPORTS = ["rf_last_error", "rf_version", "pst_create", "rf_volume_create", "rf_volume_destroy", "rf_volume_reset",
           "rf_volume_upload", "rf_volume_download", "rf_volume_info", "tsdf_integrate", "tsdf_integrate_dev",
           "rf_depth_to_points",
           "rf_overlap_mask", "fitness_eval", "fitness_eval_noalloc", "rf_tracker_create", "rf_tracker_destroy", "rf_tracker_get_scale",
           "rf_tracker_set_scale", "rf_tracker_set_params", "rf_tracker_set_schedule", "pfo_track_frame_async",
           "pfo_track_frame", "rf_tracker_last_status", "rf_sequence_start", "rf_sequence_step",
           "rf_tracker_debug_skip_barrier", "rf_batch_create", "rf_batch_destroy", "rf_batch_depth_slot",
           "rf_batch_pose_dev", "rf_batch_start", "rf_batch_step", "rf_batch_autotune", "rf_batch_set_config",
           "rf_batch_stats_dev", "pfo_track_frame_ex_async", "rf_mlp_num_params", "rf_mlp_create",
           "rf_mlp_destroy", "rf_mlp_set_params", "rf_mlp_get_params", "rf_mlp_forward", "rf_mlp_gradient",
           "rf_mlp_train_step", "rf_mlp_status", "rf_proposal_features", "rf_proposal_target",
           "rf_proposal_default_params", "rf_proposal_apply", "rf_learned_create", "rf_learned_destroy",
           "rf_learned_start", "rf_learned_step", "rf_l2_gather_probe", "rf_volume_counters",
           "rf_tracker_set_config", "rf_tracker_get_config", "rf_tracker_autotune", "rf_mlp_evaluate",
           "rf_mlp_calibrate_scale"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"librosefusion.so not built ({LIB_PATH}); run paper_2105_05600_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, i, f = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    sig = {
        "rf_last_error": (ctypes.c_char_p, []),
        "rf_version": (ctypes.c_char_p, []),
        "pst_create": (i, [i, ctypes.c_uint64, i, P, P]),
        "rf_volume_create": (i, [i, i, i, f, f, ctypes.POINTER(f), i, ctypes.POINTER(P)]),
        "rf_volume_destroy": (None, [P]),
        "rf_volume_reset": (i, [P, P]),
        "rf_volume_upload": (i, [P, P, P]),
        "rf_volume_download": (i, [P, P, P]),
        "rf_volume_info": (i, [P, ctypes.POINTER(i), ctypes.POINTER(f), ctypes.POINTER(f), ctypes.POINTER(f),
                               ctypes.POINTER(i)]),
        "tsdf_integrate": (i, [P, P, ctypes.POINTER(rf_intrinsics), ctypes.POINTER(rf_pose), P]),
        "tsdf_integrate_dev": (i, [P, P, ctypes.POINTER(rf_intrinsics), P, P, P]),
        "rf_depth_to_points": (i, [P, ctypes.POINTER(rf_intrinsics), i, P, P]),
        "rf_overlap_mask": (i, [P, i, P, ctypes.POINTER(rf_intrinsics), ctypes.POINTER(rf_pose),
                                ctypes.POINTER(rf_pose), f, P, P, P]),
        "fitness_eval": (i, [P, P, i, P, i, ctypes.POINTER(rf_pose), ctypes.POINTER(f), ctypes.POINTER(rf_params),
                             P, P, P, P]),
        "fitness_eval_noalloc": (i, [P, P, i, P, i, ctypes.POINTER(rf_pose), ctypes.POINTER(f),
                                     ctypes.POINTER(rf_params), P, P, P, P]),
        "rf_tracker_create": (i, [P, P, i, ctypes.POINTER(rf_params), i, i, ctypes.POINTER(P)]),
        "rf_tracker_destroy": (None, [P]),
        "rf_tracker_get_scale": (i, [P, ctypes.POINTER(f)]),
        "rf_tracker_set_scale": (i, [P, ctypes.POINTER(f)]),
        "rf_tracker_set_params": (i, [P, ctypes.POINTER(rf_params)]),
        "pfo_track_frame_async": (i, [P, P, P, ctypes.POINTER(rf_intrinsics), P, P, P, P]),
        "pfo_track_frame": (i, [P, P, P, ctypes.POINTER(rf_intrinsics), ctypes.POINTER(rf_pose),
                                ctypes.POINTER(rf_pose), ctypes.POINTER(rf_frame_stats), P]),
        "rf_tracker_last_status": (i, [P]),
        "rf_sequence_start": (i, [P, P, i, ctypes.POINTER(rf_intrinsics), ctypes.POINTER(rf_pose), P]),
        "rf_sequence_step": (i, [P, P, i, ctypes.POINTER(rf_intrinsics), ctypes.POINTER(rf_pose), P, P, P]),
        "rf_tracker_debug_skip_barrier": (i, [P, i, i]),
        "rf_tracker_set_schedule": (i, [P, i, ctypes.POINTER(i), ctypes.POINTER(i)]),
        "rf_batch_create": (i, [ctypes.POINTER(P), i, ctypes.POINTER(rf_intrinsics), ctypes.POINTER(P)]),
        "rf_batch_destroy": (None, [P]),
        "rf_batch_depth_slot": (i, [P, i, i, ctypes.POINTER(P)]),
        "rf_batch_pose_dev": (i, [P, i, i, ctypes.POINTER(P)]),
        "rf_batch_start": (i, [P, ctypes.POINTER(rf_pose), P]),
        "rf_batch_step": (i, [P, i, i, P]),
        "rf_batch_autotune": (i, [P, i, ctypes.POINTER(rf_launch_config), P]),
        "rf_batch_set_config": (i, [P, ctypes.POINTER(rf_launch_config)]),
        "rf_tracker_set_config": (i, [P, ctypes.POINTER(rf_launch_config)]),
        "rf_tracker_get_config": (i, [P, ctypes.POINTER(rf_launch_config)]),
        "rf_tracker_autotune": (i, [P, P, P, ctypes.POINTER(rf_intrinsics), P, ctypes.POINTER(rf_launch_config), P]),
        "rf_batch_stats_dev": (i, [P, ctypes.POINTER(P)]),
        "pfo_track_frame_ex_async": (i, [P, P, P, ctypes.POINTER(rf_intrinsics), P, P, P,
                                         ctypes.POINTER(rf_track_options), P]),
        "rf_mlp_num_params": (i, []),
        "rf_mlp_create": (i, [i, ctypes.POINTER(P)]),
        "rf_mlp_destroy": (None, [P]),
        "rf_mlp_set_params": (i, [P, ctypes.POINTER(f)]),
        "rf_mlp_get_params": (i, [P, ctypes.POINTER(f)]),
        "rf_mlp_forward": (i, [P, P, i, P, P]),
        "rf_mlp_gradient": (i, [P, P, P, P, i, i, P, P, P, P]),
        "rf_mlp_train_step": (i, [P, P, P, P, i, i, f, P, P]),
        "rf_mlp_status": (i, [P]),
        "rf_mlp_evaluate": (i, [P, P, P, P, i, i, P, P, P]),
        "rf_mlp_calibrate_scale": (i, [P, P, P, P, i, i, ctypes.POINTER(ctypes.c_float), P]),
        "rf_proposal_features": (i, [P, P, ctypes.POINTER(rf_intrinsics), P, P, P, P]),
        "rf_proposal_target": (i, [P, P, P, P]),
        "rf_proposal_default_params": (None, [ctypes.POINTER(rf_proposal_params)]),
        "rf_proposal_apply": (i, [P, P, P, ctypes.POINTER(rf_proposal_params), P, P, P]),
        "rf_learned_create": (i, [P, P, P, ctypes.POINTER(rf_proposal_params), i, i, ctypes.POINTER(P)]),
        "rf_learned_destroy": (None, [P]),
        "rf_learned_start": (i, [P, P, i, ctypes.POINTER(rf_intrinsics), ctypes.POINTER(rf_pose), P]),
        "rf_learned_step": (i, [P, P, i, ctypes.POINTER(rf_intrinsics), i, ctypes.POINTER(rf_pose), P, P, P]),
        "rf_l2_gather_probe": (i, [P, ctypes.c_size_t, i, i, i, P, P]),
        "rf_volume_counters": (i, [P, ctypes.POINTER(ctypes.c_longlong), i]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


# --------------------------------------------------------------------------- marshalling helpers
def _check(status):
    if status < 0:
        raise RfError(status, lib.rf_last_error().decode())
    return status


def _stream(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t, dtype=None):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def make_intrinsics(K: dict) -> rf_intrinsics:
    return rf_intrinsics(K["fx"], K["fy"], K["cx"], K["cy"], int(K["width"]), int(K["height"]), K["z_min"],
                         K["z_max"])


def make_pose(p) -> rf_pose:
    p = np.asarray(p, dtype=np.float64).reshape(7)
    return rf_pose((ctypes.c_float * 4)(*p[:4]), (ctypes.c_float * 3)(*p[4:]))


def pose_array(p: rf_pose) -> np.ndarray:
    return np.array(list(p.q) + list(p.t), dtype=np.float64)


def make_params(tau=1.0, beta=0.1, eps=1e-3, stop_eps=1e-6, k_max=20, flags=RF_DEFAULT_FLAGS, stride=1) -> rf_params:
    return rf_params(tau, beta, eps, stop_eps, int(k_max), int(flags), int(stride), 0)


def config_dict(cfg: rf_launch_config) -> dict:
    return dict(ctas_per_sm=cfg.ctas_per_sm, work_warps=cfg.work_warps, group=cfg.group, ms=cfg.ms)


def stats_dict(s: rf_frame_stats) -> dict:
    rows = []
    for k in range(min(s.iters, RF_MAX_ITERS)):
        r = s.it[k]
        rows.append(dict(k=r.k, n_overlap=r.n_overlap, n_aps=r.n_aps, argmax=r.argmax, rho_ref=r.rho_ref,
                         rho_tilde=r.rho_tilde, rho_max=r.rho_max, rho_second=r.rho_second, pose=list(r.pose),
                         scale=list(r.scale), offset=list(r.offset), stop=r.stop, level=r.level,
                         n_particles=r.n_particles, corner=r.corner))
    return dict(iters=s.iters, status=s.status, n_points=s.n_points, lookups=s.lookups, r1=list(s.r1), it=rows)


def stats_from_device(t) -> rf_frame_stats:
    """Parse a device buffer holding one rf_frame_stats (copied to the host)."""
    raw = t.cpu().numpy().tobytes()
    return rf_frame_stats.from_buffer_copy(raw[:ctypes.sizeof(rf_frame_stats)])


def new_stats_buffer(device="cuda"):
    import torch

    return torch.zeros(ctypes.sizeof(rf_frame_stats), dtype=torch.uint8, device=device)


def rf_version() -> str:
    return lib.rf_version().decode()


# --------------------------------------------------------------------------- PST
def pst_create(n: int, seed: int = 1, method: int = 0, out=None, stream=None):
    """Template of n particles in the unit 6D ball; returns a (6, n) float32 CUDA tensor."""
    import torch

    if out is None:
        out = torch.empty((6, n), dtype=torch.float32, device="cuda")
    _check(lib.pst_create(int(n), ctypes.c_uint64(int(seed)), int(method), _dptr(out, torch.float32),
                          _stream(stream)))
    return out


# --------------------------------------------------------------------------- volume
class Volume:
    """Owning wrapper of an rf_volume handle."""

    def __init__(self, dims, voxel, trunc, origin=(0.0, 0.0, 0.0), dtype="f32"):
        h = ctypes.c_void_p()
        org = (ctypes.c_float * 3)(*origin)
        dims = tuple(int(d) for d in (dims if hasattr(dims, "__len__") else (dims,) * 3))
        _check(lib.rf_volume_create(dims[0], dims[1], dims[2], float(voxel), float(trunc), org, DTYPES[dtype],
                                    ctypes.byref(h)))
        self.handle = h
        self.dims = dims
        self.voxel = float(voxel)
        self.trunc = float(trunc)
        self.origin = tuple(float(o) for o in origin)
        self.dtype = dtype

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib.rf_volume_destroy(h)
            self.handle = None

    @property
    def np_code_dtype(self):
        return {"f32": np.float32, "f16": np.float16, "i16": np.int16}[self.dtype]

    def reset(self, stream=None):
        _check(lib.rf_volume_reset(self.handle, _stream(stream)))

    def counters(self, reset=False):
        """rf_volume_counters: dict(voxels_updated, bricks_visited, bricks_repacked)."""
        out = (ctypes.c_longlong * 3)()
        _check(lib.rf_volume_counters(self.handle, out, int(bool(reset))))
        return dict(voxels_updated=out[0], bricks_visited=out[1], bricks_repacked=out[2])

    def upload(self, codes: np.ndarray, weights: np.ndarray | None = None):
        """codes: storage codes, shape (dz, dy, dx) or flat x-fastest."""
        codes = np.ascontiguousarray(codes, dtype=self.np_code_dtype)
        w = None if weights is None else np.ascontiguousarray(weights, dtype=np.uint8)
        _check(lib.rf_volume_upload(self.handle, codes.ctypes.data_as(ctypes.c_void_p),
                                    None if w is None else w.ctypes.data_as(ctypes.c_void_p)))

    def download(self):
        """(codes, weights) as (dz, dy, dx) numpy arrays."""
        dx, dy, dz = self.dims
        codes = np.empty((dz, dy, dx), dtype=self.np_code_dtype)
        w = np.empty((dz, dy, dx), dtype=np.uint8)
        _check(lib.rf_volume_download(self.handle, codes.ctypes.data_as(ctypes.c_void_p),
                                      w.ctypes.data_as(ctypes.c_void_p)))
        return codes, w


def tsdf_integrate(vol: Volume, depth, K: dict, pose, stream=None):
    import torch

    Ki = make_intrinsics(K)
    P = make_pose(pose)
    _check(lib.tsdf_integrate(vol.handle, _dptr(depth, torch.float32), ctypes.byref(Ki), ctypes.byref(P),
                              _stream(stream)))


def tsdf_integrate_dev(vol: Volume, depth, K: dict, pose_dev, status_dev=None, stream=None):
    import torch

    Ki = make_intrinsics(K)
    _check(lib.tsdf_integrate_dev(vol.handle, _dptr(depth, torch.float32), ctypes.byref(Ki),
                                  _dptr(pose_dev, torch.float32), _dptr(status_dev), _stream(stream)))


# --------------------------------------------------------------------------- points / overlap / fitness
def rf_depth_to_points(depth, K: dict, stride: int, out=None, stream=None):
    import torch

    W, H = int(K["width"]), int(K["height"])
    m = (-(-W // stride)) * (-(-H // stride))
    if out is None:
        out = torch.empty((m, 4), dtype=torch.float32, device=depth.device)
    Ki = make_intrinsics(K)
    _check(lib.rf_depth_to_points(_dptr(depth, torch.float32), ctypes.byref(Ki), int(stride),
                                  _dptr(out, torch.float32), _stream(stream)))
    return out


def rf_overlap_mask(points, prev_depth, K: dict, pose_cur, pose_prev, cell_extent=0.0, stream=None):
    """(mask uint8[m], count int32[1]); cell_extent (metres) > 0 adds the cell-footprint inset."""
    import torch

    m = points.shape[0]
    mask = torch.empty(max(m, 1), dtype=torch.uint8, device=points.device)
    count = torch.zeros(1, dtype=torch.int32, device=points.device)
    Ki = make_intrinsics(K)
    pc, pp = make_pose(pose_cur), make_pose(pose_prev)
    _check(lib.rf_overlap_mask(_dptr(points, torch.float32), int(m), _dptr(prev_depth, torch.float32),
                               ctypes.byref(Ki), ctypes.byref(pc), ctypes.byref(pp), float(cell_extent), _dptr(mask),
                               _dptr(count), _stream(stream)))
    return mask[:m], count


def fitness_eval(vol: Volume, points, pst, centre, scale, params: rf_params, stream=None):
    """(rho float32[n], sumsq float64[n], nvalid int32[n]) CUDA tensors."""
    import torch

    n = pst.shape[1]
    rho = torch.empty(n, dtype=torch.float32, device=points.device)
    S = torch.empty(n, dtype=torch.float64, device=points.device)
    nv = torch.empty(n, dtype=torch.int32, device=points.device)
    c = make_pose(centre)
    sc = (ctypes.c_float * 6)(*np.asarray(scale, dtype=np.float64).reshape(6))
    _check(lib.fitness_eval(vol.handle, _dptr(points, torch.float32), int(points.shape[0]),
                            _dptr(pst, torch.float32), int(n), ctypes.byref(c), sc, ctypes.byref(params),
                            _dptr(rho), _dptr(S), _dptr(nv), _stream(stream)))
    return rho, S, nv


def fitness_eval_noalloc(vol: Volume, points, pst, centre, scale, params: rf_params, out=None, stream=None):
    """fitness_eval without device allocation in the library (its scratch is a
    fixed static array).  `out` may pass preallocated (rho, sumsq, nvalid)."""
    import torch

    n = pst.shape[1]
    if out is None:
        out = (torch.empty(n, dtype=torch.float32, device=points.device),
               torch.empty(n, dtype=torch.float64, device=points.device),
               torch.empty(n, dtype=torch.int32, device=points.device))
    rho, S, nv = out
    c = make_pose(centre)
    sc = (ctypes.c_float * 6)(*np.asarray(scale, dtype=np.float64).reshape(6))
    _check(lib.fitness_eval_noalloc(vol.handle, _dptr(points, torch.float32), int(points.shape[0]),
                                    _dptr(pst, torch.float32), int(n), ctypes.byref(c), sc, ctypes.byref(params),
                                    _dptr(rho), _dptr(S), _dptr(nv), _stream(stream)))
    return rho, S, nv


# --------------------------------------------------------------------------- tracker
class Tracker:
    """Owning wrapper of an rf_tracker handle (keeps the volume and template alive)."""

    def __init__(self, vol: Volume, pst, params: rf_params, max_width: int, max_height: int):
        import torch

        h = ctypes.c_void_p()
        _check(lib.rf_tracker_create(vol.handle, _dptr(pst, torch.float32), int(pst.shape[1]), ctypes.byref(params),
                                     int(max_width), int(max_height), ctypes.byref(h)))
        self.handle = h
        self.vol = vol
        self.pst = pst
        self.params = params

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib.rf_tracker_destroy(h)
            self.handle = None

    def get_scale(self):
        r = (ctypes.c_float * 6)()
        _check(lib.rf_tracker_get_scale(self.handle, r))
        return np.array(list(r), dtype=np.float64)

    def set_scale(self, r):
        _check(lib.rf_tracker_set_scale(self.handle, (ctypes.c_float * 6)(*np.asarray(r, np.float64).reshape(6))))

    def set_params(self, params: rf_params):
        _check(lib.rf_tracker_set_params(self.handle, ctypes.byref(params)))
        self.params = params

    def set_config(self, ctas_per_sm=0, work_warps=3648, group=0):
        cfg = rf_launch_config(int(ctas_per_sm), int(work_warps), int(group), 0.0)
        _check(lib.rf_tracker_set_config(self.handle, ctypes.byref(cfg)))

    def get_config(self):
        cfg = rf_launch_config()
        _check(lib.rf_tracker_get_config(self.handle, ctypes.byref(cfg)))
        return config_dict(cfg)

    def autotune(self, depth, prev_depth, K: dict, prev_pose_dev, stream=None):
        """rf_tracker_autotune on one frame; returns the chosen configuration."""
        import torch

        Ki = make_intrinsics(K)
        cfg = rf_launch_config()
        _check(lib.rf_tracker_autotune(self.handle, _dptr(depth, torch.float32), _dptr(prev_depth, torch.float32),
                                       ctypes.byref(Ki), _dptr(prev_pose_dev, torch.float32), ctypes.byref(cfg),
                                       _stream(stream)))
        return config_dict(cfg)

    def last_status(self):
        return lib.rf_tracker_last_status(self.handle)

    def debug_skip_barrier(self, enable: bool, timeout_ms: int):
        _check(lib.rf_tracker_debug_skip_barrier(self.handle, int(bool(enable)), int(timeout_ms)))

    def set_schedule(self, n, stride):
        """Multi-resolution alternation: level l scores the first n[l] particles on
        the points at stride[l] (Sec. 4)."""
        L = len(n)
        _check(lib.rf_tracker_set_schedule(self.handle, L, (ctypes.c_int * L)(*[int(x) for x in n]),
                                           (ctypes.c_int * L)(*[int(x) for x in stride])))


class Batch:
    """Owning wrapper of an rf_batch: up to RF_MAX_BATCH sequences stepped together."""

    def __init__(self, trackers, Ks):
        n = len(trackers)
        hs = (ctypes.c_void_p * n)(*[t.handle.value for t in trackers])
        Karr = (rf_intrinsics * n)(*[make_intrinsics(K) for K in Ks])
        h = ctypes.c_void_p()
        _check(lib.rf_batch_create(hs, n, Karr, ctypes.byref(h)))
        self.handle = h
        self.trackers = list(trackers)
        self.Ks = [dict(K) for K in Ks]
        self.n = n

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib.rf_batch_destroy(h)
            self.handle = None

    def depth_slot(self, i, parity):
        """A torch view of the device slot that must hold frame f (f % 2 == parity) of sequence i."""
        import torch

        ptr = ctypes.c_void_p()
        _check(lib.rf_batch_depth_slot(self.handle, int(i), int(parity), ctypes.byref(ptr)))
        return _view_device(ptr.value, (self.Ks[i]["height"], self.Ks[i]["width"]), torch.float32)

    def pose_dev(self, i, parity):
        import torch

        ptr = ctypes.c_void_p()
        _check(lib.rf_batch_pose_dev(self.handle, int(i), int(parity), ctypes.byref(ptr)))
        return _view_device(ptr.value, (7,), torch.float32)

    def stats(self):
        """Host rf_frame_stats dicts of the last step, one per sequence."""
        import torch

        ptr = ctypes.c_void_p()
        _check(lib.rf_batch_stats_dev(self.handle, ctypes.byref(ptr)))
        raw = _view_device(ptr.value, (self.n * ctypes.sizeof(rf_frame_stats),), torch.uint8).cpu().numpy().tobytes()
        sz = ctypes.sizeof(rf_frame_stats)
        return [stats_dict(rf_frame_stats.from_buffer_copy(raw[i * sz:(i + 1) * sz])) for i in range(self.n)]

    def start(self, poses, stream=None):
        arr = (rf_pose * self.n)(*[make_pose(p) for p in poses])
        _check(lib.rf_batch_start(self.handle, arr, _stream(stream)))

    def step(self, parity, use_graph=False, stream=None):
        _check(lib.rf_batch_step(self.handle, int(parity), int(bool(use_graph)), _stream(stream)))

    def autotune(self, parity, stream=None):
        cfg = rf_launch_config()
        _check(lib.rf_batch_autotune(self.handle, int(parity), ctypes.byref(cfg), _stream(stream)))
        return config_dict(cfg)

    def set_config(self, ctas_per_sm=0, work_warps=3648, group=0):
        cfg = rf_launch_config(int(ctas_per_sm), int(work_warps), int(group), 0.0)
        _check(lib.rf_batch_set_config(self.handle, ctypes.byref(cfg)))


def _view_device(ptr, shape, dtype):
    """A torch tensor aliasing library-owned device memory (valid while the owner lives)."""
    import torch

    n = 1
    for s in shape:
        n *= s
    itemsize = torch.tensor([], dtype=dtype).element_size()

    class _CudaArray:
        __cuda_array_interface__ = {"shape": (n,), "typestr": {1: "|u1", 4: "<f4"}[itemsize],
                                    "data": (ptr, False), "version": 3}

    return torch.as_tensor(_CudaArray(), device="cuda").view(dtype).reshape(shape)


def pfo_track_frame(tr: Tracker, depth, prev_depth, K: dict, prev_pose, stream=None, check=True):
    """Returns (pose float64[7], stats dict, status)."""
    import torch

    Ki = make_intrinsics(K)
    pp = make_pose(prev_pose)
    out = rf_pose()
    st = rf_frame_stats()
    status = lib.pfo_track_frame(tr.handle, _dptr(depth, torch.float32), _dptr(prev_depth, torch.float32),
                                 ctypes.byref(Ki), ctypes.byref(pp), ctypes.byref(out), ctypes.byref(st),
                                 _stream(stream))
    if check and status < 0 and status != RF_ERR_EMPTY:
        _check(status)
    return pose_array(out), stats_dict(st), status


def pfo_track_frame_async(tr: Tracker, depth, prev_depth, K: dict, prev_pose_dev, out_pose_dev, stats_dev=None,
                          stream=None):
    import torch

    Ki = make_intrinsics(K)
    _check(lib.pfo_track_frame_async(tr.handle, _dptr(depth, torch.float32), _dptr(prev_depth, torch.float32),
                                     ctypes.byref(Ki), _dptr(prev_pose_dev, torch.float32),
                                     _dptr(out_pose_dev, torch.float32), _dptr(stats_dev), _stream(stream)))


def rf_sequence_start(tr: Tracker, depth, K: dict, pose, stream=None):
    """depth: CUDA tensor or (pinned) host numpy/torch array."""
    Ki = make_intrinsics(K)
    P = make_pose(pose)
    ptr, on_host = _any_ptr(depth)
    _check(lib.rf_sequence_start(tr.handle, ptr, on_host, ctypes.byref(Ki), ctypes.byref(P), _stream(stream)))


def rf_sequence_step(tr: Tracker, depth, K: dict, want_host_pose=True, out_pose_dev=None, stats_dev=None,
                     stream=None):
    """Track + fuse the next frame.  Returns (pose float64[7] or None, status)."""
    Ki = make_intrinsics(K)
    ptr, on_host = _any_ptr(depth)
    out = rf_pose() if want_host_pose else None
    status = lib.rf_sequence_step(tr.handle, ptr, on_host, ctypes.byref(Ki),
                                  ctypes.byref(out) if out is not None else None, _dptr(out_pose_dev),
                                  _dptr(stats_dev), _stream(stream))
    if status < 0 and status != RF_ERR_EMPTY:
        _check(status)
    return (pose_array(out) if out is not None else None), status


def _any_ptr(a):
    """(pointer, on_host) for a CUDA tensor, a CPU tensor or a numpy array."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"] or a.dtype != np.float32:
            raise ValueError("host depth must be a contiguous float32 array")
        return ctypes.c_void_p(a.ctypes.data), 1
    if a.is_cuda:
        return _dptr(a), 0
    if not a.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(a.data_ptr()), 1


def pfo_track_frame_ex_async(tr: Tracker, depth, prev_depth, K: dict, prev_pose_dev, out_pose_dev, stats_dev=None,
                             init_pose_dev=None, scale_dev=None, run_flag_dev=None, k_max=0, stream=None):
    """pfo_track_frame_async with a caller-supplied c_0 / r_0, run flag and iteration cap."""
    import torch

    Ki = make_intrinsics(K)
    o = rf_track_options(_dptr(init_pose_dev, torch.float32), _dptr(scale_dev, torch.float32),
                         _dptr(run_flag_dev, torch.int32), int(k_max), 0)
    _check(lib.pfo_track_frame_ex_async(tr.handle, _dptr(depth, torch.float32), _dptr(prev_depth, torch.float32),
                                        ctypes.byref(Ki), _dptr(prev_pose_dev, torch.float32),
                                        _dptr(out_pose_dev, torch.float32), _dptr(stats_dev), ctypes.byref(o),
                                        _stream(stream)))


# --------------------------------------------------------------------------- learned proposal (rf_proposal.h)
def _bf16_ptr(t):
    """Device pointer of a contiguous bfloat16 (or int16 bit-pattern) CUDA tensor."""
    import torch

    if t.dtype not in (torch.bfloat16, torch.int16):
        raise ValueError(f"expected bfloat16 bits, got {t.dtype}")
    return _dptr(t)


def rf_mlp_num_params() -> int:
    return int(lib.rf_mlp_num_params())


class MLP:
    """rf_mlp: the proposal network's parameters, Adam state and activations on the device."""

    def __init__(self, max_batch: int):
        h = ctypes.c_void_p()
        _check(lib.rf_mlp_create(int(max_batch), ctypes.byref(h)))
        self.handle = h
        self.max_batch = int(max_batch)
        self.n_params = rf_mlp_num_params()

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            lib.rf_mlp_destroy(h)
            self.handle = None

    def set_params(self, theta):
        a = np.ascontiguousarray(theta, dtype=np.float32).reshape(-1)
        if a.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {a.size}")
        _check(lib.rf_mlp_set_params(self.handle, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def get_params(self) -> np.ndarray:
        a = np.zeros(self.n_params, dtype=np.float32)
        _check(lib.rf_mlp_get_params(self.handle, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return a

    def forward(self, x, out=None, stream=None):
        """x: (B, 832) bfloat16 CUDA tensor -> (B, 16) float32."""
        import torch

        B = x.shape[0]
        if out is None:
            out = torch.empty((B, RF_MLP_OUT), dtype=torch.float32, device="cuda")
        _check(lib.rf_mlp_forward(self.handle, _bf16_ptr(x), int(B), _dptr(out, torch.float32), _stream(stream)))
        return out

    def gradient(self, x_all, y_all, batch, idx=None, stream=None):
        """(grad float32[P], loss float32[1], outputs float32[batch, 16]) of one batch."""
        import torch

        grad = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        out = torch.empty((batch, RF_MLP_OUT), dtype=torch.float32, device="cuda")
        _check(lib.rf_mlp_gradient(self.handle, _bf16_ptr(x_all), _dptr(y_all, torch.float32),
                                   _dptr(idx, torch.int32), int(x_all.shape[0]), int(batch), _dptr(grad),
                                   _dptr(loss), _dptr(out), _stream(stream)))
        return grad, loss, out

    def train_step(self, x_all, y_all, batch, lr, idx=None, loss_out=None, stream=None):
        import torch

        _check(lib.rf_mlp_train_step(self.handle, _bf16_ptr(x_all), _dptr(y_all, torch.float32),
                                     _dptr(idx, torch.int32), int(x_all.shape[0]), int(batch), float(lr),
                                     _dptr(loss_out, torch.float32), _stream(stream)))

    def evaluate(self, x_all, y_all, idx=None, n_rows=None, mu_out=None, stream=None):
        """rf_mlp_evaluate: (mu float32 (rows, 6) CUDA tensor, stats float64[13] CUDA
        tensor) over rows idx (or the first n_rows)."""
        import torch

        rows = int(idx.shape[0]) if idx is not None else int(n_rows or x_all.shape[0])
        mu = mu_out if mu_out is not None else torch.empty((rows, 6), dtype=torch.float32, device=x_all.device)
        stats = torch.empty(RF_MLP_EVAL_STATS, dtype=torch.float64, device=x_all.device)
        _check(lib.rf_mlp_evaluate(self.handle, _bf16_ptr(x_all), _dptr(y_all, torch.float32),
                                   _dptr(idx, torch.int32), int(x_all.shape[0]), rows, _dptr(mu), _dptr(stats),
                                   _stream(stream)))
        return mu, stats

    def calibrate_scale(self, x_all, y_all, idx=None, n_rows=None, stream=None):
        """rf_mlp_calibrate_scale: adds log k to the log-scale output biases; returns k."""
        import torch

        rows = int(idx.shape[0]) if idx is not None else int(n_rows or x_all.shape[0])
        k = (ctypes.c_float * 6)()
        _check(lib.rf_mlp_calibrate_scale(self.handle, _bf16_ptr(x_all), _dptr(y_all, torch.float32),
                                          _dptr(idx, torch.int32), int(x_all.shape[0]), rows, k, _stream(stream)))
        return [float(v) for v in k]

    def status(self) -> int:
        return lib.rf_mlp_status(self.handle)


def rf_proposal_features(depth, prev_depth, K: dict, pose_prev2_dev, pose_prev_dev, x_out=None, stream=None):
    """Network input of one frame pair -> bfloat16 CUDA tensor [832] (or x_out, a row of a dataset)."""
    import torch

    if x_out is None:
        x_out = torch.empty(RF_MLP_IN, dtype=torch.bfloat16, device="cuda")
    Ki = make_intrinsics(K)
    _check(lib.rf_proposal_features(_dptr(depth, torch.float32), _dptr(prev_depth, torch.float32), ctypes.byref(Ki),
                                    _dptr(pose_prev2_dev, torch.float32), _dptr(pose_prev_dev, torch.float32),
                                    _bf16_ptr(x_out), _stream(stream)))
    return x_out


def rf_proposal_target(pose_prev_dev, pose_cur_dev, y_out=None, stream=None):
    import torch

    if y_out is None:
        y_out = torch.empty(6, dtype=torch.float32, device="cuda")
    _check(lib.rf_proposal_target(_dptr(pose_prev_dev, torch.float32), _dptr(pose_cur_dev, torch.float32),
                                  _dptr(y_out, torch.float32), _stream(stream)))
    return y_out


def proposal_params(**kw) -> rf_proposal_params:
    p = rf_proposal_params()
    lib.rf_proposal_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k in ("r_min", "r_max"):
            setattr(p, k, (ctypes.c_float * 6)(*v))
        else:
            setattr(p, k, v)
    return p


def rf_proposal_apply(out_dev, x_dev, pose_prev_dev, params: rf_proposal_params, stream=None):
    """(c_0 float32[7], r_0 float32[6]) CUDA tensors from one network output and
    the input row it came from."""
    import torch

    c0 = torch.empty(7, dtype=torch.float32, device="cuda")
    r0 = torch.empty(6, dtype=torch.float32, device="cuda")
    _check(lib.rf_proposal_apply(_dptr(out_dev, torch.float32), _bf16_ptr(x_dev), _dptr(pose_prev_dev, torch.float32),
                                 ctypes.byref(params), _dptr(c0), _dptr(r0), _stream(stream)))
    return c0, r0


def learned_stats_dict(t) -> dict:
    raw = t.cpu().numpy().tobytes()[:ctypes.sizeof(rf_learned_stats)]
    s = rf_learned_stats.from_buffer_copy(raw)
    return dict(status=s.status, used_fallback=s.used_fallback, chose_fallback=s.chose_fallback,
                iters_learned=s.iters_learned, iters_fallback=s.iters_fallback, rho_learned=s.rho_learned,
                rho_fallback=s.rho_fallback, rho_prev=s.rho_prev, init_pose=list(s.init_pose), r0=list(s.r0),
                lookups=s.lookups)


def new_learned_stats_buffer(device="cuda"):
    import torch

    return torch.zeros(ctypes.sizeof(rf_learned_stats), dtype=torch.uint8, device=device)


class Learned:
    """rf_learned: proposal-driven tracking of one sequence (tracker + volume + trained network)."""

    def __init__(self, tr: Tracker, vol: Volume, net: MLP, params: rf_proposal_params, max_width: int,
                 max_height: int):
        h = ctypes.c_void_p()
        _check(lib.rf_learned_create(tr.handle, vol.handle, net.handle, ctypes.byref(params), int(max_width),
                                     int(max_height), ctypes.byref(h)))
        self.handle = h
        self._keep = (tr, vol, net)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            lib.rf_learned_destroy(h)
            self.handle = None

    def start(self, depth, K: dict, pose, stream=None):
        Ki = make_intrinsics(K)
        P = make_pose(pose)
        ptr, on_host = _any_ptr(depth)
        _check(lib.rf_learned_start(self.handle, ptr, on_host, ctypes.byref(Ki), ctypes.byref(P), _stream(stream)))

    def step(self, depth, K: dict, use_graph=False, want_host_pose=True, out_pose_dev=None, stats_dev=None,
             stream=None):
        """Track + fuse the next frame.  Returns (pose float64[7] or None, status)."""
        Ki = make_intrinsics(K)
        ptr, on_host = _any_ptr(depth)
        out = rf_pose() if want_host_pose else None
        status = lib.rf_learned_step(self.handle, ptr, on_host, ctypes.byref(Ki), int(bool(use_graph)),
                                     ctypes.byref(out) if out is not None else None, _dptr(out_pose_dev),
                                     _dptr(stats_dev), _stream(stream))
        if status < 0 and status != RF_ERR_EMPTY:
            _check(status)
        return (pose_array(out) if out is not None else None), status


def rf_l2_gather_probe(buf, loads_per_thread, ctas_per_sm, sink, mode=0, stream=None):
    """One launch of the gather microbenchmark over the CUDA tensor `buf` (mode 0:
    random 16-byte records, 1: random 128-byte lines); sink: CUDA uint32/int32
    tensor of ctas_per_sm x SMs x 256 entries."""
    _check(lib.rf_l2_gather_probe(_dptr(buf), buf.numel() * buf.element_size(), int(loads_per_thread),
                                  int(ctas_per_sm), int(mode), _dptr(sink), _stream(stream)))
