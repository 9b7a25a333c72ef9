"""ctypes wrapper of the plain FP64 CPU oracle (asm_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package smoke check and by
the CPU-baseline leg of bench.py.  The product path (the CUDA library and its
binding) never imports this module.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "asm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libasm_oracle.so")

_dp = ct.POINTER(ct.c_double)
_ip = ct.POINTER(ct.c_int)
_lp = ct.POINTER(ct.c_long)
_u64p = ct.POINTER(ct.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP over chains, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ct.CDLL(build())
        L.ora_philox4x64_10.argtypes = [_u64p, _u64p, _u64p]
        for name in ("ora_norm_cdf", "ora_norm_quantile", "ora_erfcx", "ora_log_q"):
            getattr(L, name).argtypes = [ct.c_double]
            getattr(L, name).restype = ct.c_double
        L.ora_truncnorm.argtypes = [ct.c_double] * 5
        L.ora_truncnorm.restype = ct.c_double
        L.ora_truncnorm_robert.argtypes = [ct.c_double, ct.c_double, ct.c_uint64, ct.c_uint64, ct.c_int, _dp]
        L.ora_truncnorm_robert.restype = ct.c_long
        L.ora_cholesky.argtypes = [ct.c_int, _dp, _dp]
        L.ora_cholesky.restype = ct.c_int
        L.ora_jacobi_svd.argtypes = [ct.c_int, ct.c_int, _dp, _dp, _dp, _dp]
        L.ora_jacobi_svd.restype = ct.c_int
        L.ora_setup.argtypes = [ct.c_int, ct.c_int, _dp, _dp, _dp, ct.c_int, _ip, _ip, _ip]
        L.ora_setup.restype = ct.c_void_p
        L.ora_setup_ex.argtypes = [ct.c_int, ct.c_int, _dp, _dp, _dp, ct.c_int, _ip, _ip, ct.c_int, _ip]
        L.ora_setup_ex.restype = ct.c_void_p
        L.ora_free.argtypes = [ct.c_void_p]
        L.ora_sizes.argtypes = [ct.c_void_p, _lp, _lp, _lp]
        L.ora_export.argtypes = [ct.c_void_p, _dp, _dp, _dp, _dp, _dp]
        L.ora_initial_f.argtypes = [ct.c_void_p, _dp]
        L.ora_conditional.argtypes = [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, _dp, _dp, _dp, _dp, _dp]
        L.ora_conditional.restype = ct.c_int
        L.ora_chi2.argtypes = [ct.c_void_p, _dp]
        L.ora_chi2.restype = ct.c_double
        L.ora_run.argtypes = [ct.c_void_p, ct.c_int, ct.c_long, ct.c_long, ct.c_uint64, ct.c_uint64,
                              ct.c_int, _dp, _dp, _dp, _dp, _dp, ct.c_int, _lp]
        L.ora_run.restype = ct.c_int
        L.ora_run_from.argtypes = [ct.c_void_p, ct.c_int, _dp, ct.c_long, ct.c_long, ct.c_long,
                                   ct.c_uint64, ct.c_uint64, ct.c_int, _dp, _dp, _dp, _dp, _dp,
                                   ct.c_int, _lp]
        L.ora_run_from.restype = ct.c_int
        L.ora_run_ids.argtypes = [ct.c_void_p, ct.c_int, _dp, ct.c_long, ct.c_long, ct.c_long,
                                  ct.c_uint64, ct.c_uint64, ct.c_uint64, ct.c_int, _dp, _dp, _dp, _dp, _dp,
                                  ct.c_int, _lp]
        L.ora_run_ids.restype = ct.c_int
        L.ora_set_jitter.argtypes = [ct.c_void_p, ct.c_int, ct.c_int]
        L.ora_set_prior.argtypes = [ct.c_void_p, _dp]
        L.ora_set_prior.restype = ct.c_int
        _lib = L
    return _lib


def _d(a):
    return None if a is None else a.ctypes.data_as(_dp)


def philox4x64_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint64)
    k = np.asarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().ora_philox4x64_10(c.ctypes.data_as(_u64p), k.ctypes.data_as(_u64p), out.ctypes.data_as(_u64p))
    return out


def norm_cdf(z):
    return lib().ora_norm_cdf(float(z))


def norm_quantile(p):
    return lib().ora_norm_quantile(float(p))


def erfcx(x):
    return lib().ora_erfcx(float(x))


def log_q(x):
    return lib().ora_log_q(float(x))


def truncnorm(mu, sigma, lo, hi, u):
    return lib().ora_truncnorm(float(mu), float(sigma), float(lo), float(hi), float(u))


def truncnorm_robert(a, b, n, seed=1, stream=0):
    """n draws of N(0,1) on [a, b] by Robert's (1995) rejection sampler and
    the number of proposals it made."""
    out = np.zeros(n)
    tries = lib().ora_truncnorm_robert(float(a), float(b), ct.c_uint64(seed), ct.c_uint64(stream), n, _d(out))
    return out, tries


def cholesky(C):
    C = np.ascontiguousarray(C, dtype=np.float64)
    L = np.zeros_like(C)
    rc = lib().ora_cholesky(C.shape[0], _d(C), _d(L))
    if rc != 0:
        raise ValueError("not SPD")
    return L


def jacobi_svd(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    m, n = A.shape
    s = np.zeros(n)
    U = np.zeros((m, n))
    V = np.zeros((n, n))
    rc = lib().ora_jacobi_svd(m, n, _d(A), _d(s), _d(U), _d(V))
    if rc < 0:
        raise RuntimeError(f"Jacobi SVD failed ({rc})")
    return s, U, V


@dataclass
class Decomposition:
    """Whitened kernel/data and the per-block factors, in the layout the CUDA
    library accepts as a given decomposition."""
    Kt: np.ndarray
    gt: np.ndarray
    d: np.ndarray
    V: np.ndarray
    U: np.ndarray


class OracleProblem:
    ERRORS = {-1: "shape", -2: "not SPD", -3: "non-finite", -4: "improper zero mode"}

    def __init__(self, K, G, C, levels, prior_shape=None, flat_exp=40):
        K = np.ascontiguousarray(K, dtype=np.float64)
        G = np.ascontiguousarray(G, dtype=np.float64)
        C = np.ascontiguousarray(C, dtype=np.float64)
        self.M, self.N = K.shape
        self.levels = [np.asarray(l, dtype=np.int32) for l in levels]
        nb = np.array([len(l) for l in self.levels], dtype=np.int32)
        bs = np.concatenate(self.levels).astype(np.int32)
        err = ct.c_int(0)
        self._h = lib().ora_setup_ex(self.M, self.N, _d(K), _d(G), _d(C), len(self.levels),
                                     nb.ctypes.data_as(_ip), bs.ctypes.data_as(_ip), int(flat_exp), ct.byref(err))
        if not self._h:
            raise ValueError(f"oracle setup failed: {self.ERRORS.get(err.value, err.value)}")
        self.err = err.value
        if prior_shape is not None:
            a = np.ascontiguousarray(prior_shape, dtype=np.float64)
            if a.shape != (self.N,) or lib().ora_set_prior(self._h, _d(a)) != 0:
                raise ValueError("prior shape must be N values >= 1")

    def __del__(self):
        if getattr(self, "_h", None):
            lib().ora_free(self._h)
            self._h = None

    def set_jitter(self, on=True, unit_exp=52, pattern=0):
        """Rounding-sensitivity probe: every move's conditional mean and interval
        ends moved by one rounding at unit roundoff 2^-unit_exp before its draw,
        the directions taken from bits of the move's Philox word chosen by
        `pattern` (0..15) (tests only)."""
        lib().ora_set_jitter(self._h, int(unit_exp) if on else 0, int(pattern))

    def blocks(self):
        """(level, block, start, n) for every block in level order."""
        out = []
        for l, starts in enumerate(self.levels):
            for b, s in enumerate(starts):
                e = starts[b + 1] if b + 1 < len(starts) else self.N
                out.append((l, b, int(s), int(e - s)))
        return out

    def decomposition(self) -> Decomposition:
        nd, nv, nu = ct.c_long(), ct.c_long(), ct.c_long()
        lib().ora_sizes(self._h, ct.byref(nd), ct.byref(nv), ct.byref(nu))
        Kt = np.zeros((self.M, self.N))
        gt = np.zeros(self.M)
        d = np.zeros(nd.value)
        V = np.zeros(nv.value)
        U = np.zeros(nu.value)
        lib().ora_export(self._h, _d(Kt), _d(gt), _d(d), _d(V), _d(U))
        return Decomposition(Kt, gt, d, V, U)

    def initial_f(self):
        f = np.zeros(self.N)
        lib().ora_initial_f(self._h, _d(f))
        return f

    def chi2(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        return lib().ora_chi2(self._h, _d(f))

    def conditional(self, level, block, j, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        mu, sg, lo, hi = ct.c_double(), ct.c_double(), ct.c_double(), ct.c_double()
        rc = lib().ora_conditional(self._h, level, block, j, _d(f), ct.byref(mu), ct.byref(sg),
                                   ct.byref(lo), ct.byref(hi))
        if rc != 0:
            raise IndexError("bad level/block/mode")
        return mu.value, sg.value, lo.value, hi.value

    def run(self, chains, burn_in, sweeps, seed, problem_id=0, threads=0, trace_chains=0,
            f_start=None, sweep0=0, chain_offset=0):
        """Returns a dict with f_final, S1, S2 (chains x N), chi2 (chains),
        kept (sweeps), stats and, if asked, trace (trace_chains x sweeps_total x N)."""
        N = self.N
        f_final = np.zeros((chains, N))
        S1 = np.zeros((chains, N))
        S2 = np.zeros((chains, N))
        chi2 = np.zeros(chains)
        total = burn_in + sweeps
        trace = np.zeros((trace_chains, total, N)) if trace_chains else None
        stats = np.zeros(4, dtype=np.int64)
        if f_start is None:
            f_start = self.initial_f()
        fs = np.ascontiguousarray(np.broadcast_to(f_start, (chains, N)), dtype=np.float64)
        rc = lib().ora_run_ids(self._h, chains, _d(fs), sweep0, burn_in, sweeps, ct.c_uint64(seed),
                               ct.c_uint64(problem_id), ct.c_uint64(chain_offset), threads, _d(f_final),
                               _d(S1), _d(S2), _d(chi2), _d(trace), trace_chains, stats.ctypes.data_as(_lp))
        if rc != 0:
            raise RuntimeError("oracle run failed")
        return {"f_final": f_final, "S1": S1, "S2": S2, "chi2": chi2, "kept": sweeps,
                "stats": stats, "trace": trace}


def summarize(S1, S2, kept, w=None):
    """Mean of fbar over all chains and sweeps, its standard error from the
    spread of the independent chain means, and the effective sample size
    (posterior variance over squared standard error)."""
    S1 = np.asarray(S1, dtype=np.float64)
    S2 = np.asarray(S2, dtype=np.float64)
    C = S1.shape[0]
    cm = S1 / kept
    mean = cm.mean(axis=0)
    var = (S2.sum(axis=0) / (C * kept)) - mean ** 2
    sem = cm.std(axis=0, ddof=1) / np.sqrt(C) if C > 1 else np.full_like(mean, np.nan)
    ess = np.where(sem > 0, np.maximum(var, 0.0) / np.maximum(sem, 1e-300) ** 2, np.nan)
    out = {"mean_fbar": mean, "sem_fbar": sem, "var_fbar": var, "ess": ess}
    if w is not None:
        out["mean_A"] = mean / w
        out["sem_A"] = sem / w
    return out


BIN_SWEEPS = 64      # sweeps per level-0 bin (aligned to absolute sweep indices)
BIN_LEVELS = 8       # doubling levels: bins of 64, 128, ..., 8192 sweeps


def binning(trace, sweep0, burn_in, b0=BIN_SWEEPS, levels=BIN_LEVELS):
    """Monte Carlo error of the mean of fbar by binning (Flyvbjerg and Petersen,
    J. Chem. Phys. 91, 461 (1989)): the kept sweeps of every chain are cut into
    bins of b0 sweeps aligned to multiples of b0 in the absolute sweep index
    (only bins lying wholly after the burn-in count), neighbouring bins are
    merged pairwise level by level, and at level k the squared error of the
    grand mean is the variance of the level-k bin means over all chains'
    bins divided by their number.

    trace: chains x sweeps x N states after each sweep, the first one being
    absolute sweep `sweep0`; burn_in: absolute index of the first kept sweep.
    Returns (sigma2 per level, levels x N; bins per chain per level)."""
    trace = np.asarray(trace, dtype=np.float64)
    C, T, N = trace.shape
    first = -(-max(burn_in, sweep0) // b0) * b0          # first bin start inside the kept range
    nb0 = (sweep0 + T - first) // b0 if sweep0 + T > first else 0
    sig2 = np.full((levels, N), np.nan)
    counts = np.zeros(levels, dtype=np.int64)
    if nb0 <= 0:
        return sig2, counts
    x = trace[:, first - sweep0: first - sweep0 + nb0 * b0, :].reshape(C, nb0, b0, N).mean(axis=2)
    for k in range(levels):
        m = x.shape[1]
        counts[k] = m
        if m >= 1:
            means = x.reshape(C * m, N)
            n = means.shape[0]
            if n > 1:
                sig2[k] = means.var(axis=0, ddof=1) / n
        if m < 2:
            break
        x = 0.5 * (x[:, 0:2 * (m // 2):2, :] + x[:, 1:2 * (m // 2):2, :])
    return sig2, counts


def mc_error(trace, sweep0, burn_in, S1, S2, kept):
    """The error estimate the library reports: sigma^2 = the largest binning
    level with at least two bins per chain, or the squared spread of the chain
    means if that is larger; ESS = posterior variance / sigma^2."""
    sig2, counts = binning(trace, sweep0, burn_in)
    s = summarize(S1, S2, kept)
    best = np.array(s["sem_fbar"]) ** 2
    for k in range(len(counts)):
        if counts[k] >= 2:
            best = np.fmax(best, sig2[k])
    ess = np.maximum(s["var_fbar"], 0.0) / np.maximum(best, 1e-300)
    return {"sigma2": best, "ess": ess, "sigma2_levels": sig2, "bins_per_chain": counts}
