"""Thin Python binding of the C ABI in include/asm.h (ctypes).

Argument marshalling only: every step of the sampling path runs in the CUDA
library libasm_gb300.so.  PyTorch supplies the device workspace and the
stream.  There is no CPU fallback: if the library or a GPU is missing, the
calls raise.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

from . import build as _build

ASM_OK = 0
ASM_FP64 = 0
ASM_MIXED = 1
ASM_SAMPLE_CONTINUE = 1
ASM_SAMPLE_TIMING = 2
ASM_SAMPLE_MOMENTS = 4
ASM_SAMPLE_REFRESH_FP64 = 8
ASM_SAMPLE_STEP_TRACE = 16
ASM_FLAG_TEST_STALL = 0x80000000   # asm_desc flag: failure-path tests only
ASM_ERR_TIMEOUT = -10
ASM_SNAPSHOT_EVERY = 8
BIN_SWEEPS = 64      # binning: level-0 bin length in sweeps
BIN_LEVELS = 8       # binning: doubling levels

_dp = ct.POINTER(ct.c_double)
_ip = ct.POINTER(ct.c_int)


class asm_desc(ct.Structure):
    _fields_ = [("M", ct.c_int), ("N", ct.c_int),
                ("K", _dp), ("G", _dp), ("C", _dp), ("w", _dp),
                ("n_levels", ct.c_int), ("level_nblocks", _ip), ("block_start", _ip),
                ("Kt", _dp), ("gt", _dp), ("d", _dp), ("V", _dp), ("U", _dp),
                ("flags", ct.c_uint32), ("P", ct.c_int), ("dK_dtheta", _dp), ("dw_dtheta", _dp),
                ("prior_shape", _dp)]


class asm_stats(ct.Structure):
    _fields_ = [("chains", ct.c_int64), ("sweeps_done", ct.c_int64), ("kept_sweeps", ct.c_int64),
                ("precision", ct.c_int64), ("degenerate_moves", ct.c_int64),
                ("zero_mode_moves", ct.c_int64), ("tail_capped", ct.c_int64),
                ("nonfinite_moves", ct.c_int64), ("max_resync_drift", ct.c_double),
                ("sweep_launches", ct.c_int64), ("other_launches", ct.c_int64),
                ("timed_launches", ct.c_int64), ("sweep_kernel_ms", ct.c_double),
                ("timeouts", ct.c_int64), ("graph_replays", ct.c_int64), ("tc_refreshes", ct.c_int64),
                ("team_lanes", ct.c_int32),
                ("consumers_per_cta", ct.c_int32), ("ctas", ct.c_int32), ("work_items", ct.c_int32),
                ("min_blocks", ct.c_int32), ("reserved_", ct.c_int32), ("prior_rejections", ct.c_int64)]


EXPORTS = ["asm_setup", "asm_workspace_bytes", "asm_sample", "asm_average", "asm_chain_state",
           "asm_status", "asm_destroy", "asm_error_string", "asm_sample_noalloc", "asm_set_stream_ids",
           "asm_checkpoint", "asm_restore", "asm_backward", "asm_setup_batch", "asm_problem_count",
           "asm_average_at", "asm_tune", "asm_partition_hierarchy", "asm_mc_error", "asm_measure_ceiling",
           "asm_step_trace"]
# instruction mixes of asm_measure_ceiling
CEILING_KINDS = {"pass_f32": 0, "pass_f32_smem": 1, "ffma": 2, "fmnmx": 3, "imnmx": 4, "pass_f64": 5,
                 "pass_f64_smem": 6, "dfma": 7, "dmnmx": 8, "i64mnmx": 9}
ASM_NOALLOC_SCRATCH_BYTES = 64 << 20

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libasm_gb300.so (building it in-tree first if asked)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {path}")
        _build.build()
    L = ct.CDLL(path)
    L.asm_setup.argtypes = [ct.POINTER(asm_desc), ct.POINTER(ct.c_void_p)]
    L.asm_setup.restype = ct.c_int
    L.asm_workspace_bytes.argtypes = [ct.c_void_p, ct.c_int, ct.c_int]
    L.asm_workspace_bytes.restype = ct.c_size_t
    L.asm_sample.argtypes = [ct.c_void_p, ct.c_int, ct.c_long, ct.c_long, ct.c_uint64, ct.c_int,
                             ct.c_uint32, ct.c_void_p, ct.c_size_t, ct.c_void_p]
    L.asm_sample.restype = ct.c_int
    L.asm_average.argtypes = [ct.c_void_p, _dp, _dp, _dp, _dp]
    L.asm_average.restype = ct.c_int
    L.asm_chain_state.argtypes = [ct.c_void_p, _dp, _dp]
    L.asm_chain_state.restype = ct.c_int
    L.asm_status.argtypes = [ct.c_void_p, ct.POINTER(asm_stats)]
    L.asm_status.restype = ct.c_int
    L.asm_destroy.argtypes = [ct.c_void_p]
    L.asm_destroy.restype = None
    L.asm_error_string.argtypes = [ct.c_int]
    L.asm_error_string.restype = ct.c_char_p
    L.asm_sample_noalloc.argtypes = [ct.c_void_p, ct.c_int, ct.c_long, ct.c_long, ct.c_uint64, ct.c_int,
                                     ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]
    L.asm_sample_noalloc.restype = ct.c_int
    L.asm_set_stream_ids.argtypes = [ct.c_void_p, ct.c_uint64, ct.c_uint64]
    L.asm_set_stream_ids.restype = ct.c_int
    L.asm_checkpoint.argtypes = [ct.c_void_p, ct.c_void_p, ct.POINTER(ct.c_size_t)]
    L.asm_checkpoint.restype = ct.c_int
    L.asm_restore.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_size_t, ct.c_void_p, ct.c_size_t, ct.c_void_p]
    L.asm_restore.restype = ct.c_int
    L.asm_backward.argtypes = [ct.c_void_p, _dp, _dp, _dp]
    L.asm_backward.restype = ct.c_int
    L.asm_setup_batch.argtypes = [ct.c_int, ct.POINTER(asm_desc), ct.POINTER(ct.c_void_p)]
    L.asm_setup_batch.restype = ct.c_int
    L.asm_problem_count.argtypes = [ct.c_void_p]
    L.asm_problem_count.restype = ct.c_int
    L.asm_average_at.argtypes = [ct.c_void_p, ct.c_int, _dp, _dp, _dp, _dp]
    L.asm_average_at.restype = ct.c_int
    L.asm_tune.argtypes = [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p, ct.c_size_t, ct.c_void_p,
                           ct.POINTER(ct.c_int), ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)]
    L.asm_tune.restype = ct.c_int
    L.asm_partition_hierarchy.argtypes = [ct.c_int, _ip, _ip, _ip, _ip]
    L.asm_partition_hierarchy.restype = ct.c_int
    L.asm_mc_error.argtypes = [ct.c_void_p, ct.c_int, _dp, _dp, _dp, _ip]
    L.asm_mc_error.restype = ct.c_int
    L.asm_measure_ceiling.argtypes = [ct.c_int, ct.c_double, _dp, _dp, _dp]
    L.asm_measure_ceiling.restype = ct.c_int
    L.asm_step_trace.argtypes = [ct.c_void_p, ct.c_int, _dp, ct.c_int, _ip]
    L.asm_step_trace.restype = ct.c_int
    _lib = L
    return L


def partition_hierarchy(N):
    """asm_partition_hierarchy: the levels (arrays of block starts) of the
    blocked-modes hierarchy on N grid points, from the whole grid down to one
    point per block.  Host-side, needs no GPU."""
    L = load()
    nl, tot = ct.c_int(0), ct.c_int(0)
    nb = np.zeros(64, dtype=np.int32)
    _check(L.asm_partition_hierarchy(int(N), ct.byref(nl), nb.ctypes.data_as(_ip), None, ct.byref(tot)),
           "asm_partition_hierarchy")
    bs = np.zeros(max(tot.value, 1), dtype=np.int32)
    _check(L.asm_partition_hierarchy(int(N), ct.byref(nl), nb.ctypes.data_as(_ip), bs.ctypes.data_as(_ip),
                                     ct.byref(tot)), "asm_partition_hierarchy")
    out, o = [], 0
    for l in range(nl.value):
        out.append(bs[o:o + nb[l]].copy())
        o += nb[l]
    return out


def measure_ceiling(kind, target_ms=30.0):
    """asm_measure_ceiling: measured rate of one instruction mix on the current
    GPU (elements/s for the pass kinds, instructions/s otherwise), with the SM
    clock seen during the launch (MHz) and the launch time (ms)."""
    _require_cuda()
    rate, mhz, ms = ct.c_double(0), ct.c_double(0), ct.c_double(0)
    _check(load().asm_measure_ceiling(CEILING_KINDS[kind], float(target_ms), ct.byref(rate), ct.byref(mhz),
                                      ct.byref(ms)), "asm_measure_ceiling")
    return {"rate": rate.value, "sm_mhz": mhz.value, "ms": ms.value}


class ASMError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {load().asm_error_string(code).decode()} ({code})")


def _check(code, where):
    if code != ASM_OK:
        raise ASMError(code, where)


def _dptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _require_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the average-spectrum sampler runs on a CUDA GPU only (no CPU fallback)")
    return torch


def _make_desc(K, G, C, levels, w=None, factors=None, dK_dtheta=None, dw_dtheta=None, prior_shape=None,
               flags=0):
    """asm_desc of one problem plus the arrays it points into (kept alive by
    the caller until asm_setup returns)."""
    keep = []
    K = np.ascontiguousarray(K, dtype=np.float64)
    M, N = K.shape
    G = np.ascontiguousarray(G, dtype=np.float64)
    C = np.ascontiguousarray(C, dtype=np.float64)
    w = np.ones(N) if w is None else np.ascontiguousarray(w, dtype=np.float64)
    levels = [np.asarray(l, dtype=np.int32) for l in levels]
    nb = np.array([len(l) for l in levels], dtype=np.int32)
    bs = np.concatenate(levels).astype(np.int32)
    d = asm_desc()
    d.M, d.N = M, N
    d.K, d.G, d.C, d.w = _dptr(K), _dptr(G), _dptr(C), _dptr(w)
    d.n_levels = len(levels)
    d.level_nblocks = nb.ctypes.data_as(_ip)
    d.block_start = bs.ctypes.data_as(_ip)
    d.flags = int(flags)
    keep += [K, G, C, w, nb, bs]
    if factors is not None:
        arrs = [np.ascontiguousarray(getattr(factors, k), dtype=np.float64) for k in ("Kt", "gt", "d", "V", "U")]
        keep += arrs
        d.Kt, d.gt, d.d, d.V, d.U = (_dptr(a) for a in arrs)
    P = 0
    if dK_dtheta is not None:
        dK = np.ascontiguousarray(dK_dtheta, dtype=np.float64)
        dw = np.ascontiguousarray(dw_dtheta, dtype=np.float64)
        P = dK.shape[0]
        assert dK.shape == (P, M, N) and dw.shape == (P, N)
        keep += [dK, dw]
        d.P, d.dK_dtheta, d.dw_dtheta = P, _dptr(dK), _dptr(dw)
    if prior_shape is not None:
        a = np.ascontiguousarray(prior_shape, dtype=np.float64)
        assert a.shape == (N,)
        keep.append(a)
        d.prior_shape = _dptr(a)
    return d, keep, (M, N, w, levels, P)


class _Handle:
    """Workspace, sampling, tuning and counters shared by single problems and
    batches."""

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.asm_destroy(self._h)
            self._h = None

    def workspace_bytes(self, chains, precision=ASM_MIXED):
        return int(load().asm_workspace_bytes(self._h, chains, precision))

    def _workspace(self, chains, precision, workspace=None):
        torch = _require_cuda()
        need = self.workspace_bytes(chains, precision)
        if need == 0:
            raise ASMError(-7, "asm_workspace_bytes")
        if workspace is None:
            if self._ws is None or self._ws.numel() < need or self._ws.device != torch.device("cuda", torch.cuda.current_device()):
                self._ws = torch.empty(need, dtype=torch.uint8, device="cuda")
            workspace = self._ws
        else:
            self._ws = workspace
        return torch, workspace

    def sample(self, chains, burn_in, sweeps, seed, precision=ASM_MIXED, cont=False, stream=None,
               workspace=None, timing=False, moments=False, refresh_fp64=False, step_trace=False):
        """asm_sample on a torch workspace (allocated here unless given) and the
        current torch stream (or `stream`)."""
        torch, workspace = self._workspace(chains, precision, workspace)
        s = stream if stream is not None else torch.cuda.current_stream()
        flags = ((ASM_SAMPLE_CONTINUE if cont else 0) | (ASM_SAMPLE_TIMING if timing else 0) |
                 (ASM_SAMPLE_MOMENTS if moments else 0) | (ASM_SAMPLE_REFRESH_FP64 if refresh_fp64 else 0) |
                 (ASM_SAMPLE_STEP_TRACE if step_trace else 0))
        _check(load().asm_sample(self._h, chains, burn_in, sweeps, ct.c_uint64(seed), precision, flags,
                                 ct.c_void_p(workspace.data_ptr()), workspace.numel(),
                                 ct.c_void_p(s.cuda_stream)), "asm_sample")
        self.chains = chains

    def tune(self, chains, precision=ASM_MIXED, stream=None, workspace=None):
        """asm_tune: picks the fastest launch shape (lanes per chain, chain warps
        per CTA, register budget) for `chains` chains; returns
        (team_lanes, consumers, min_blocks)."""
        torch, workspace = self._workspace(chains, precision, workspace)
        s = stream if stream is not None else torch.cuda.current_stream()
        team, cons, mb = ct.c_int(0), ct.c_int(0), ct.c_int(0)
        _check(load().asm_tune(self._h, chains, precision, ct.c_void_p(workspace.data_ptr()), workspace.numel(),
                               ct.c_void_p(s.cuda_stream), ct.byref(team), ct.byref(cons), ct.byref(mb)),
               "asm_tune")
        return team.value, cons.value, mb.value

    def set_stream_ids(self, problem_id=0, chain_offset=0):
        _check(load().asm_set_stream_ids(self._h, ct.c_uint64(problem_id), ct.c_uint64(chain_offset)),
               "asm_set_stream_ids")

    def mc_error(self, k=0):
        """asm_mc_error: binned Monte Carlo error of <fbar> of problem k:
        ess, sem_fbar (N each), sigma2_levels (8 x N), bins_per_chain (8)."""
        N = self.shapes[k][1] if hasattr(self, "shapes") else self.N
        ess, sem = np.zeros(N), np.zeros(N)
        lv = np.zeros((BIN_LEVELS, N))
        bins = np.zeros(BIN_LEVELS, dtype=np.int32)
        _check(load().asm_mc_error(self._h, k, _dptr(ess), _dptr(sem), _dptr(lv), bins.ctypes.data_as(_ip)),
               "asm_mc_error")
        return {"ess": ess, "sem_fbar": sem, "sigma2_levels": lv, "bins_per_chain": bins}

    def step_trace(self, k=0, max_sweeps=4096):
        """asm_step_trace: mean over the chains of |f(s+1) - f(s)| / |f(s)| per sweep s
        (sweeps sampled with step_trace=True)."""
        out = np.zeros(max_sweeps)
        n = ct.c_int(0)
        _check(load().asm_step_trace(self._h, k, _dptr(out), max_sweeps, ct.byref(n)), "asm_step_trace")
        return out[:n.value]

    def status(self):
        st = asm_stats()
        _check(load().asm_status(self._h, ct.byref(st)), "asm_status")
        return {k: getattr(st, k) for k, _ in asm_stats._fields_}


def _average(h, k, N, w):
    mean_A, sem_A, ess, mean_f = (np.zeros(N) for _ in range(4))
    _check(load().asm_average_at(h, k, _dptr(mean_A), _dptr(sem_A), _dptr(ess), _dptr(mean_f)),
           "asm_average_at")
    return {"mean_A": mean_A, "sem_A": sem_A, "ess": ess, "mean_fbar": mean_f, "sem_fbar": sem_A * w}


class Batch(_Handle):
    """Independent problems sampled together (asm_setup_batch): every problem's
    chains run in the same persistent launches.  `problems` is a sequence of
    dicts with the keyword arguments of Problem (K, G, C, levels, w, factors)."""

    def __init__(self, problems):
        L = load()
        descs, keeps, self.shapes = [], [], []
        for pr in problems:
            d, keep, (M, N, w, levels, _) = _make_desc(**pr)
            descs.append(d)
            keeps.append(keep)
            self.shapes.append((M, N, w))
        arr = (asm_desc * len(descs))(*descs)
        h = ct.c_void_p()
        _check(L.asm_setup_batch(len(descs), arr, ct.byref(h)), "asm_setup_batch")
        self._h = h
        self._ws = None
        self.chains = 0
        assert L.asm_problem_count(h) == len(descs)

    def __len__(self):
        return len(self.shapes)

    def average(self, k):
        M, N, w = self.shapes[k]
        return _average(self._h, k, N, w)


class Problem(_Handle):
    """A set-up problem: owns the library handle and a torch workspace.

    K (M x N, acting on fbar), G (M), C (M x M) and the levels (list of arrays
    of block starts) follow Sec. II and IV of the paper; w are the Riemann
    weights (A = fbar / w).  `factors` (optional) is an object with Kt, gt, d,
    V, U arrays in the layout of asm_desc to use given singular vectors."""

    def __init__(self, K, G, C, levels, w=None, factors=None, dK_dtheta=None, dw_dtheta=None, prior_shape=None,
                 flags=0):
        L = load()
        d, self._keep, (self.M, self.N, self.w, self.levels, self.P) = _make_desc(
            K, G, C, levels, w, factors, dK_dtheta, dw_dtheta, prior_shape, flags)
        h = ct.c_void_p()
        _check(L.asm_setup(ct.byref(d), ct.byref(h)), "asm_setup")
        self._h = h
        self._ws = None
        self.chains = 0

    def sample_noalloc(self, chains, burn_in, sweeps, seed, precision, out_mean, out_sem2, out_m2,
                       stream=None):
        """asm_sample_noalloc: the library allocates nothing; the outputs are the
        caller's device tensors (N float64 each), written asynchronously."""
        torch = _require_cuda()
        for t in (out_mean, out_sem2, out_m2):
            if t.dtype != torch.float64 or not t.is_cuda or t.numel() < self.N or not t.is_contiguous():
                raise ValueError("outputs must be contiguous float64 CUDA tensors of N elements")
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(load().asm_sample_noalloc(self._h, chains, burn_in, sweeps, ct.c_uint64(seed), precision,
                                         ct.c_void_p(out_mean.data_ptr()), ct.c_void_p(out_sem2.data_ptr()),
                                         ct.c_void_p(out_m2.data_ptr()), ct.c_void_p(s.cuda_stream)),
               "asm_sample_noalloc")
        self.chains = chains

    def average(self):
        return _average(self._h, 0, self.N, self.w)

    def backward(self, v, want_G=True, want_theta=None):
        """asm_backward: vector-Jacobian products of <A> for the cotangent v (N)."""
        v = np.ascontiguousarray(v, dtype=np.float64)
        want_theta = self.P > 0 if want_theta is None else want_theta
        gG = np.zeros(self.M) if want_G else None
        gt = np.zeros(self.P) if want_theta else None
        _check(load().asm_backward(self._h, _dptr(v), _dptr(gG), _dptr(gt)), "asm_backward")
        return gG, gt

    def chain_state(self):
        f = np.zeros((self.chains, self.N))
        chi2 = np.zeros(self.chains)
        _check(load().asm_chain_state(self._h, _dptr(f), _dptr(chi2)), "asm_chain_state")
        return f, chi2

    def checkpoint(self) -> bytes:
        n = ct.c_size_t(0)
        _check(load().asm_checkpoint(self._h, None, ct.byref(n)), "asm_checkpoint")
        buf = ct.create_string_buffer(n.value)
        _check(load().asm_checkpoint(self._h, buf, ct.byref(n)), "asm_checkpoint")
        return buf.raw[:n.value]

    def restore(self, blob: bytes, chains, precision=ASM_MIXED, stream=None):
        torch = _require_cuda()
        need = self.workspace_bytes(chains, precision)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        s = stream if stream is not None else torch.cuda.current_stream()
        buf = ct.create_string_buffer(blob, len(blob))
        _check(load().asm_restore(self._h, buf, len(blob), ct.c_void_p(self._ws.data_ptr()), self._ws.numel(),
                                  ct.c_void_p(s.cuda_stream)), "asm_restore")
        self.chains = chains
