"""FP64 CPU oracle for the ROSEFusion PFO/PST tracking path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s cpu_baseline / reference leg may import this package.  It
shares no code with the CUDA library in ``paper_2105_05600_gb300``; the C
source ``rf_oracle.c`` is the implementation, this module only marshals numpy
arrays.  Every function cites the paper passage it follows (ROSEFusion,
Zhang et al., ACM TOG 40(4) 2021):

    quat_to_rot / quat_mul ........ Sec. 3.3 (state = quaternion + translation)
    compose_offset / particle_pose  Sec. 3.3 MovePST / RescalePST, Algorithm 1
    unproject ..................... Sec. 3.1 Eq. unproj; Sec. 4 stride downsampling
    overlap ....................... Sec. 4 Eq. validness
    tsdf_sample / fitness ......... Sec. 3.1 Eq. likelihood, Sec. 4 Eq. normallh
    pst_update .................... Sec. 3.3 Eq. ebs, rsdir, rsinter, momentum; Eq. wafit
    pfo_step ...................... one iteration of Algorithm 1 (state in, state out)
    pfo_frame / pfo_frame_sched ... Algorithm 1 + Sec. 4 initialisation / stop rules / corner cases
    fitness_particles ............. Eq. normallh for a range of template particles
    tsdf_integrate ................ Sec. 3 overview (Curless-Levoy volumetric fusion)
    pst_uniform / philox .......... Sec. 4 "PST pre-sampling" (uniform unit 6D ball)
    ate / te ...................... Sec. 5.1 ATE, Eq. te
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "librf_oracle.so")
_SRC = os.path.join(_HERE, "rf_oracle.c")

OVERLAP, NORMALIZE, COMPENSATED, NEAREST, RHO_REF_CENTER, L1, RIGHT_MULT, CELL_MARGIN = 1, 2, 4, 8, 16, 32, 64, 128
APS_WITH_CENTRE = 256
DEFAULT_FLAGS = OVERLAP | NORMALIZE | COMPENSATED | CELL_MARGIN
TRACE_STRIDE = 40
STATE_LEN = 16
TIE_PX, TIE_RHO = 1e-3, 1e-5  # decision margins the trace counts (columns 35, 36)
# trace columns (see rf_oracle.c)
T_K, T_NO, T_NAPS, T_RHO_REF, T_RHO_TILDE, T_RHO_MAX, T_ARGMAX = 0, 1, 2, 3, 4, 5, 6
T_POSE, T_SCALE, T_DBAR = slice(7, 14), slice(14, 20), slice(20, 26)
T_MIN_GAP, T_MIN_MARGIN, T_STOP, T_RHO_2ND, T_LEVEL, T_NL = 26, 27, 28, 29, 30, 31
T_CORNER, T_VALID, T_EMPTY_RUN, T_FRAGILE_PX, T_TIES, T_SENS, T_STEP, T_SENS2 = 32, 33, 34, 35, 36, 37, 38, 39
QMODE = {"f64": 0, "f32": 1, "f16": 2, "i16": 3}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile rf_oracle.c into a shared library with gcc (plain -O2, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D = ctypes.POINTER(ctypes.c_double)
            F = ctypes.POINTER(ctypes.c_float)
            I = ctypes.POINTER(ctypes.c_int)
            U32 = ctypes.POINTER(ctypes.c_uint32)
            d, i = ctypes.c_double, ctypes.c_int
            lib.or_quat_mul.argtypes = [D, D, D]
            lib.or_quat_to_rot.argtypes = [D, D]
            lib.or_compose_offset.argtypes = [D, D, i, D]
            lib.or_particle_pose.argtypes = [D, D, D, i, D]
            lib.or_unproject.argtypes = [F, i, i, d, d, d, d, d, d, i, D]
            lib.or_unproject.restype = i
            lib.or_overlap.argtypes = [D, i, F, i, i, d, d, d, d, d, d, D, D, d, I, D]
            lib.or_overlap.restype = i
            lib.or_tsdf_sample.argtypes = [D, I, d, D, D, i, D]
            lib.or_tsdf_sample.restype = i
            lib.or_fitness.argtypes = [D, I, d, D, D, I, i, D, d, i, D, I, I, D]
            lib.or_pst_update.argtypes = [i, D, D, d, D, d, d, D, D, D]
            lib.or_pst_update.restype = i
            lib.or_pfo_frame.argtypes = [D, I, d, D, D, i, F, i, i, d, d, d, d, d, d, D, D, D, F, i,
                                         d, d, d, d, i, i, D, D, D, I]
            lib.or_pfo_frame.restype = i
            lib.or_pfo_frame_mt.argtypes = [D, I, d, D, D, i, F, i, i, d, d, d, d, d, d, D, D, D, F, i,
                                            d, d, d, d, i, i, i, D, D, D, I]
            lib.or_pfo_frame_mt.restype = i
            lib.or_pfo_step.argtypes = [D, I, d, D, D, i, i, F, i, i, d, d, d, d, d, d, D, F, i, d, d, d, d, i, i,
                                        i, i, D, D]
            lib.or_pfo_step.restype = i
            lib.or_fitness_particles.argtypes = [D, I, d, D, D, I, i, D, D, F, i, i, i, d, i, i, D, I, D]
            lib.or_tsdf_integrate_mt.argtypes = [D, I, I, d, D, d, i, i, F, i, i, d, d, d, d, d, d, D, i]
            lib.or_quantize.argtypes = [d, i]
            lib.or_quantize.restype = d
            lib.or_tsdf_integrate.argtypes = [D, I, I, d, D, d, i, i, F, i, i, d, d, d, d, d, d, D]
            lib.or_philox4x32_10.argtypes = [U32, U32, U32]
            lib.or_pst_uniform.argtypes = [i, ctypes.c_uint64, F]
            lib.or_pst_uniform.restype = i
            lib.or_ate.argtypes = [D, D, i, D, D]
            lib.or_te.argtypes = [D, D]
            lib.or_te.restype = d
            lib.or_grid_search.argtypes = [D, I, d, D, D, I, i, D, D, i, d, i, D]
            lib.or_grid_search.restype = d
            lib.or_fitness_fragile.argtypes = [D, I, d, D, D, I, i, D, d, i, d, D, I, I, D, I]
            lib.or_pfo_frame_sched.argtypes = [D, I, d, D, i, I, ctypes.POINTER(D), I, F, i, i, d, d, d, d, d, d, D,
                                               D, D, F, i, d, d, d, d, i, i, D, D, D, I]
            lib.or_pfo_frame_sched.restype = i
            lib.or_pfo_frame_sched_mt.argtypes = [D, I, d, D, i, I, ctypes.POINTER(D), I, F, i, i, d, d, d, d, d, d,
                                                  D, D, D, F, i, d, d, d, d, i, i, i, D, D, D, I]
            lib.or_pfo_frame_sched_mt.restype = i
            lib.or_tsdf_integrate_ambiguity.argtypes = [I, d, D, d, F, i, i, d, d, d, d, d, d, D, d, I]
            _lib = lib
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


# --------------------------------------------------------------------------- geometry
def quat_mul(a, b):
    """Hamilton product (Sec. 3.3)."""
    lib = _load()
    a, pa = _d(a)
    b, pb = _d(b)
    o, po = _d(np.zeros(4))
    lib.or_quat_mul(pa, pb, po)
    return o


def quat_to_rot(q):
    """Rotation matrix of a unit quaternion (w, x, y, z)."""
    lib = _load()
    q, pq = _d(q)
    R, pR = _d(np.zeros(9))
    lib.or_quat_to_rot(pq, pR)
    return R.reshape(3, 3)


def compose_offset(c, delta, flags=DEFAULT_FLAGS):
    """c (+) delta: MovePST reading (Sec. 3.3)."""
    lib = _load()
    c, pc = _d(c)
    dl, pd = _d(delta)
    o, po = _d(np.zeros(7))
    lib.or_compose_offset(pc, pd, int(flags), po)
    return o


def particle_pose(c, r, omega6, flags=DEFAULT_FLAGS):
    """Particle pose c (+) (r . omega) (Sec. 3.3, Sec. 4 GPU implementation)."""
    lib = _load()
    c, pc = _d(c)
    r, pr = _d(r)
    om, po_ = _d(omega6)
    o, po = _d(np.zeros(7))
    lib.or_particle_pose(pc, pr, po_, int(flags), po)
    return o


def unproject(depth, K, stride):
    """Strided unprojection (Eq. unproj).  K = dict(fx, fy, cx, cy, z_min, z_max).
    Returns (M, 4) float64 array of (x, y, z, valid)."""
    lib = _load()
    depth, pdp = _f(depth)
    H, W = depth.shape
    nw, nh = -(-W // stride), -(-H // stride)
    pts, pp = _d(np.zeros((nh * nw, 4)))
    m = lib.or_unproject(pdp, W, H, K["fx"], K["fy"], K["cx"], K["cy"], K["z_min"], K["z_max"], int(stride), pp)
    assert m == nh * nw
    return pts


def overlap(pts, prev_depth, K, pose_cur, pose_prev, cell_m=0.0):
    """Eq. validness mask and rounding margins for every point; cell_m > 0 also
    keeps the re-projection fx cell_m / z' pixels inside frame t-1's image."""
    lib = _load()
    pts, pp = _d(pts)
    prev_depth, pdp = _f(prev_depth)
    H, W = prev_depth.shape
    M = pts.shape[0]
    pc, ppc = _d(pose_cur)
    pv, ppv = _d(pose_prev)
    mask, pm = _i(np.zeros(M, np.int32))
    margin, pmg = _d(np.zeros(M))
    n = lib.or_overlap(pp, M, pdp, W, H, K["fx"], K["fy"], K["cx"], K["cy"], K["z_min"], K["z_max"], ppc, ppv,
                       float(cell_m), pm, pmg)
    return mask, margin, n


class Volume:
    """Dense FP64 TSDF (x fastest, NaN = unobserved) with integer weights."""

    def __init__(self, dims, voxel, origin, trunc, w_max=255, qmode="f64"):
        self.dims = np.array(dims, dtype=np.int32)
        self.voxel = float(voxel)
        self.origin = np.array(origin, dtype=np.float64)
        self.trunc = float(trunc)
        self.w_max = int(w_max)
        self.qmode = QMODE[qmode] if isinstance(qmode, str) else int(qmode)
        n = int(np.prod(self.dims))
        self.F = np.full(n, np.nan, dtype=np.float64)
        self.W = np.zeros(n, dtype=np.int32)

    def grid(self):
        """F as a (z, y, x) view."""
        d = self.dims
        return self.F.reshape(d[2], d[1], d[0])

    def integrate(self, depth, K, pose, threads=1):
        """Volumetric fusion of one depth frame at pose (Sec. 3 overview); threads
        splits the voxel slices (same result for any count)."""
        lib = _load()
        depth, pdp = _f(depth)
        H, W = depth.shape
        pose, pp = _d(pose)
        _, pdim = _i(self.dims)
        _, por = _d(self.origin)
        args = (self.F.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                self.W.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), pdim, self.voxel, por, self.trunc, self.w_max,
                self.qmode, pdp, W, H, K["fx"], K["fy"], K["cx"], K["cy"], K["z_min"], K["z_max"], pp)
        if threads == 1:
            lib.or_tsdf_integrate(*args)
        else:
            lib.or_tsdf_integrate_mt(*args, int(threads))

    def sample(self, p, flags=0):
        lib = _load()
        p, pp = _d(p)
        _, pdim = _i(self.dims)
        _, por = _d(self.origin)
        out = ctypes.c_double(0.0)
        ok = lib.or_tsdf_sample(self.F.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), pdim, self.voxel, por, pp,
                                int(flags), ctypes.byref(out))
        return (out.value if ok else None)

    def fitness(self, pts, in_set, pose, tau=1.0, flags=DEFAULT_FLAGS):
        """(S, n_valid, |O|, rho) of one pose (Eq. normallh)."""
        lib = _load()
        pts, pp = _d(pts)
        in_set, pin = _i(in_set)
        pose, ppose = _d(pose)
        _, pdim = _i(self.dims)
        _, por = _d(self.origin)
        S, rho = ctypes.c_double(), ctypes.c_double()
        n, nO = ctypes.c_int(), ctypes.c_int()
        lib.or_fitness(self.F.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), pdim, self.voxel, por, pp, pin,
                       pts.shape[0], ppose, float(tau), int(flags), ctypes.byref(S), ctypes.byref(n),
                       ctypes.byref(nO), ctypes.byref(rho))
        return S.value, n.value, nO.value, rho.value

    def fitness_fragile(self, pts, in_set, pose, tau=1.0, flags=DEFAULT_FLAGS, delta_g=1e-3):
        """(S, n_valid, |O|, rho, n_fragile): n_fragile counts points whose sample
        validity (or nearest voxel) flips within +-delta_g voxels."""
        lib = _load()
        pts, pp = _d(pts)
        in_set, pin = _i(in_set)
        pose, ppose = _d(pose)
        _, pdim = _i(self.dims)
        _, por = _d(self.origin)
        S, rho = ctypes.c_double(), ctypes.c_double()
        n, nO, fr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        lib.or_fitness_fragile(self.F.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), pdim, self.voxel, por, pp,
                               pin, pts.shape[0], ppose, float(tau), int(flags), float(delta_g), ctypes.byref(S),
                               ctypes.byref(n), ctypes.byref(nO), ctypes.byref(rho), ctypes.byref(fr))
        return S.value, n.value, nO.value, rho.value, fr.value

    def integrate_ambiguity(self, depth, K, pose, tol=1e-4):
        """int32 map (same layout as F) of voxels whose fusion decisions are near a threshold."""
        lib = _load()
        depth, pdp = _f(depth)
        H, W = depth.shape
        pose, pp = _d(pose)
        _, pdim = _i(self.dims)
        _, por = _d(self.origin)
        amb, pa = _i(np.zeros(self.F.shape[0], np.int32))
        lib.or_tsdf_integrate_ambiguity(pdim, self.voxel, por, self.trunc, pdp, W, H, K["fx"], K["fy"], K["cx"],
                                        K["cy"], K["z_min"], K["z_max"], pp, float(tol), pa)
        return amb

    def grid_search(self, pts, in_set, c, half, steps, tau=1.0, flags=DEFAULT_FLAGS):
        """Best (rho, pose) over a steps^6 grid of offsets about c (brute force)."""
        lib = _load()
        pts, pp = _d(pts)
        in_set, pin = _i(in_set)
        c, pc = _d(c)
        half, ph = _d(half)
        _, pdim = _i(self.dims)
        _, por = _d(self.origin)
        best, pb = _d(np.zeros(7))
        rho = lib.or_grid_search(self.F.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), pdim, self.voxel, por, pp,
                                 pin, pts.shape[0], pc, ph, int(steps), float(tau), int(flags), pb)
        return rho, best

    def pfo_frame_sched(self, level_pts, level_n, prev_depth, K, pose_prev, c0, r0, omega, params, threads=1):
        """Algorithm 1 with multi-resolution alternation (Sec. 4): level l uses the
        first level_n[l] template rows and the point set level_pts[l].  Same
        return value as pfo_frame."""
        lib = _load()
        L = len(level_pts)
        arrs = [np.ascontiguousarray(p, dtype=np.float64) for p in level_pts]
        ptrs = (ctypes.POINTER(ctypes.c_double) * L)(*[a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in arrs])
        ln, pln = _i(np.asarray(level_n, np.int32))
        lm, plm = _i(np.array([a.shape[0] for a in arrs], np.int32))
        prev_depth, pdp = _f(prev_depth)
        H, W = prev_depth.shape
        pose_prev, ppv = _d(pose_prev)
        c0, pc0 = _d(c0)
        r0, pr0 = _d(r0)
        omega, pom = _f(omega)
        N = omega.shape[1]
        k_max = int(params["k_max"])
        _, pdim = _i(self.dims)
        _, por = _d(self.origin)
        pose, ppo = _d(np.zeros(7))
        r1, pr1 = _d(np.zeros(6))
        trace, ptr = _d(np.zeros((k_max, TRACE_STRIDE)))
        iters = ctypes.c_int(0)
        args = [self.F.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), pdim, self.voxel, por, L, pln, ptrs, plm, pdp,
                W, H, K["fx"], K["fy"], K["cx"], K["cy"], K["z_min"], K["z_max"], ppv, pc0, pr0, pom, N,
                float(params["tau"]), float(params["beta"]), float(params["eps"]), float(params["stop_eps"]), k_max,
                int(params["flags"])]
        if threads == 1:
            st = lib.or_pfo_frame_sched(*args, ppo, pr1, ptr, ctypes.byref(iters))
        else:
            st = lib.or_pfo_frame_sched_mt(*args, int(threads), ppo, pr1, ptr, ctypes.byref(iters))
        return dict(status=st, pose=pose, r1=r1, iters=iters.value, trace=trace[:iters.value])

    def pfo_frame(self, pts, prev_depth, K, pose_prev, c0, r0, omega, params, threads=1):
        """Algorithm 1 for one frame.  params: dict(tau, beta, eps, stop_eps, k_max, flags).
        Returns dict(status, pose, r1, iters, trace[iters, TRACE_STRIDE]); threads
        splits the per-particle fitness loop (same result for any count)."""
        lib = _load()
        pts, pp = _d(pts)
        prev_depth, pdp = _f(prev_depth)
        H, W = prev_depth.shape
        pose_prev, ppv = _d(pose_prev)
        c0, pc0 = _d(c0)
        r0, pr0 = _d(r0)
        omega, pom = _f(omega)
        N = omega.shape[1]
        k_max = int(params["k_max"])
        _, pdim = _i(self.dims)
        _, por = _d(self.origin)
        pose, ppo = _d(np.zeros(7))
        r1, pr1 = _d(np.zeros(6))
        trace, ptr = _d(np.zeros((k_max, TRACE_STRIDE)))
        iters = ctypes.c_int(0)
        args = [self.F.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), pdim, self.voxel, por, pp, pts.shape[0], pdp,
                W, H, K["fx"], K["fy"], K["cx"], K["cy"], K["z_min"], K["z_max"], ppv, pc0, pr0, pom, N,
                float(params["tau"]), float(params["beta"]), float(params["eps"]), float(params["stop_eps"]), k_max,
                int(params["flags"])]
        if threads == 1:
            st = lib.or_pfo_frame(*args, ppo, pr1, ptr, ctypes.byref(iters))
        else:
            st = lib.or_pfo_frame_mt(*args, int(threads), ppo, pr1, ptr, ctypes.byref(iters))
        return dict(status=st, pose=pose, r1=r1, iters=iters.value, trace=trace[:iters.value])

    def pfo_step(self, pts, n_level, prev_depth, K, pose_prev, omega, params, state, centre_ref=False, threads=1):
        """One iteration of Algorithm 1 (see or_pfo_step) on the first n_level
        template particles.  state = dict(c, r, rho_carry, empty_run, k) is the
        state before the iteration.  Returns (stop code, new state dict, trace row)."""
        lib = _load()
        pts, pp = _d(pts)
        prev_depth, pdp = _f(prev_depth)
        H, W = prev_depth.shape
        pose_prev, ppv = _d(pose_prev)
        omega, pom = _f(omega)
        N = omega.shape[1]
        _, pdim = _i(self.dims)
        _, por = _d(self.origin)
        st = np.zeros(STATE_LEN)
        st[0:7] = state["c"]
        st[7:13] = state["r"]
        st[13] = state.get("rho_carry", 0.0)
        st[14] = state.get("empty_run", 0)
        st[15] = state["k"]
        st, pst = _d(st)
        row, prow = _d(np.zeros(TRACE_STRIDE))
        stop = lib.or_pfo_step(self.F.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), pdim, self.voxel, por, pp,
                               pts.shape[0], int(n_level), pdp, W, H, K["fx"], K["fy"], K["cx"], K["cy"], K["z_min"],
                               K["z_max"], ppv, pom, N, float(params["tau"]), float(params["beta"]),
                               float(params["eps"]), float(params["stop_eps"]), int(params["k_max"]),
                               int(params["flags"]), int(bool(centre_ref)), int(threads), pst, prow)
        new = dict(c=st[0:7].copy(), r=st[7:13].copy(), rho_carry=float(st[13]), empty_run=int(st[14]),
                   k=int(st[15]))
        return stop, new, row

    def fitness_particles(self, pts, mask, c, r, omega, i_begin, i_end, tau=1.0, flags=DEFAULT_FLAGS, threads=1):
        """(rho, n_valid) of template particles [i_begin, i_end) about centre c with
        axes r over the points with mask != 0 (Eq. normallh)."""
        lib = _load()
        pts, pp = _d(pts)
        mask, pm = _i(mask)
        c, pc = _d(c)
        r, pr = _d(r)
        omega, pom = _f(omega)
        N = omega.shape[1]
        _, pdim = _i(self.dims)
        _, por = _d(self.origin)
        rho, prho = _d(np.zeros(N))
        nval, pnv = _i(np.zeros(N, np.int32))
        delta, pdl = _d(np.zeros(6 * N))
        lib.or_fitness_particles(self.F.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), pdim, self.voxel, por, pp,
                                 pm, pts.shape[0], pc, pr, pom, N, int(i_begin), int(i_end), float(tau), int(flags),
                                 int(threads), prho, pnv, pdl)
        return rho[i_begin:i_end].copy(), nval[i_begin:i_end].copy()


def pst_update(rho, delta, rho_ref, r_prev, beta=0.1, eps=1e-3):
    """APS + Eq. ebs/wafit/rsdir/rsinter/momentum.  Returns (n_aps, delta_bar, rho_tilde, r)."""
    lib = _load()
    rho, prho = _d(rho)
    delta, pdl = _d(delta)
    r_prev, prp = _d(r_prev)
    dbar, pdb = _d(np.zeros(6))
    rout, pro = _d(np.zeros(6))
    rt = ctypes.c_double()
    n = lib.or_pst_update(rho.shape[0], prho, pdl, float(rho_ref), prp, float(beta), float(eps), pdb,
                          ctypes.byref(rt), pro)
    return n, dbar, rt.value, rout


def quantize(F, qmode):
    return _load().or_quantize(float(F), QMODE[qmode] if isinstance(qmode, str) else int(qmode))


def philox4x32_10(ctr, key):
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib.or_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def pst_uniform(n, seed):
    """Uniform PST in the unit 6D ball (Sec. 4), 6 x n float32, row 0 = origin."""
    lib = _load()
    out, po = _f(np.zeros((6, n), np.float32))
    st = lib.or_pst_uniform(int(n), ctypes.c_uint64(int(seed)), po)
    assert st == 0
    return out


def ate(est, gt):
    """(mean, rmse) translational error after rigid alignment (Sec. 5.1)."""
    lib = _load()
    est, pe = _d(est)
    gt, pg = _d(gt)
    m, r = ctypes.c_double(), ctypes.c_double()
    lib.or_ate(pe, pg, est.shape[0], ctypes.byref(m), ctypes.byref(r))
    return m.value, r.value


def te(est, gt):
    """Eq. te for one frame."""
    lib = _load()
    est, pe = _d(est)
    gt, pg = _d(gt)
    return lib.or_te(pe, pg)
