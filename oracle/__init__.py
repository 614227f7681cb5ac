"""Plain CPU oracle for the skew-symmetric LABS search (arXiv 2011.00068).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` use it to check and time the GPU library.  The library never
imports it, and it shares no code with the library.

The arithmetic lives in ``labs_oracle.c`` (plain C, built here with gcc on first
use); this module only marshals numpy arrays through ctypes.  Every function cites
the passage of the paper it follows:

* ``ck`` / ``isl`` / ``psl`` / ``merit`` -- Eq. 1, Eq. 2, PSL (Section 1), Eq. 3.
* ``skew_expand`` / ``is_skew`` -- Eq. 4 in the 0-based reading s[c+j] = (-1)^j s[c-j],
  c = n-1, L = 2n-1.
* ``hex_decode`` / ``hex_encode`` -- the encoding rule printed below Table 1.
* ``neighbor_delta`` -- Algorithm 1's neighbourhood (flip each free variable),
  by the general two-position change of every C_k.
* ``philox4x32_10`` / ``random_start`` -- Philox4x32-10 (Salmon et al., SC'11) and
  the random start of Algorithm 1.
* ``walk`` -- Algorithm 1 in the self-avoiding-walk form with restarts (lssOrel).
* ``bestfirst`` -- Algorithm 1 as printed: best-first search with a fixed-size
  priority queue of evaluated neighbours (impxLast, Section 3).
* ``enumerate_skew`` -- exhaustive search over skew-symmetric sequences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "labs_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liblabs_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile labs_oracle.c into a shared object (gcc, portable flags)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    fresh = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
    if fresh and not force:
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-shared", "-fPIC", "-pthread",
           "-Wall", "-Werror", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class WalkCfg(ctypes.Structure):
    _fields_ = [("tabu_log2", ctypes.c_int32), ("probe_cap", ctypes.c_int32),
                ("patience", ctypes.c_int32), ("target_num", ctypes.c_int32),
                ("target_den", ctypes.c_int32)]


class WalkResult(ctypes.Structure):
    _fields_ = [("final_isl", ctypes.c_int32), ("best_isl", ctypes.c_int32),
                ("best_step", ctypes.c_int64), ("target_step", ctypes.c_int64),
                ("restarts", ctypes.c_int32), ("overflows", ctypes.c_int32),
                ("final_psl", ctypes.c_int32), ("best_psl", ctypes.c_int32), ("cache_hits", ctypes.c_int64)]


WALK_RESULT_FIELDS = [f[0] for f in WalkResult._fields_]
TRACE_RESTART = 0x10000


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
            L.lo_ck.argtypes = [P, i32, i32]; L.lo_ck.restype = i64
            L.lo_isl.argtypes = [P, i32]; L.lo_isl.restype = i64
            L.lo_psl.argtypes = [P, i32]; L.lo_psl.restype = i64
            L.lo_merit.argtypes = [i32, i64]; L.lo_merit.restype = ctypes.c_double
            L.lo_skew_expand.argtypes = [P, i32, P]; L.lo_skew_expand.restype = ctypes.c_int
            L.lo_is_skew.argtypes = [P, i32]; L.lo_is_skew.restype = ctypes.c_int
            L.lo_hex_decode.argtypes = [ctypes.c_char_p, i32, P]; L.lo_hex_decode.restype = ctypes.c_int
            L.lo_hex_encode.argtypes = [P, i32, ctypes.c_char_p]; L.lo_hex_encode.restype = ctypes.c_int
            L.lo_neighbor_delta.argtypes = [P, i32, P]; L.lo_neighbor_delta.restype = ctypes.c_int
            L.lo_philox4x32_10.argtypes = [P, P, P]; L.lo_philox4x32_10.restype = None
            L.lo_random_start.argtypes = [u64, ctypes.c_uint32, ctypes.c_uint32, i32, P]
            L.lo_random_start.restype = None
            L.lo_zobrist_key.argtypes = [i32, i32]; L.lo_zobrist_key.restype = u64
            L.lo_fingerprint.argtypes = [P, i32]; L.lo_fingerprint.restype = u64
            L.lo_walk.argtypes = [i32, u64, i64, i64, i64, ctypes.POINTER(WalkCfg), P, P, P, P, P, i32]
            L.lo_walk.restype = ctypes.c_int
            L.lo_walk_psl.argtypes = L.lo_walk.argtypes
            L.lo_walk_psl.restype = ctypes.c_int
            L.lo_enumerate.argtypes = [i32, P, P, P, P, i32]; L.lo_enumerate.restype = ctypes.c_int
            L.lo_bestfirst.argtypes = [i32, u64, i64, i64, i64, ctypes.POINTER(WalkCfg), i32, P, P, P, P, P, i32]
            L.lo_bestfirst.restype = ctypes.c_int
            L.lo_bestfirst_cached.argtypes = L.lo_bestfirst.argtypes
            L.lo_bestfirst_cached.restype = ctypes.c_int
            L.lo_walk_replay.argtypes = [i32, u64, i64, i64, ctypes.POINTER(WalkCfg), i32, i32, P, P, i32, i32, P, P,
                                         P, P, P, P, P]
            L.lo_walk_replay.restype = ctypes.c_int
            _lib = L
    return _lib


def _i8(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.int8)
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def ck(s, k: int) -> int:
    """Eq. 1: aperiodic autocorrelation C_k of a +-1 sequence."""
    s = _i8(s)
    return int(lib().lo_ck(_ptr(s), s.size, k))


def isl(s) -> int:
    """Eq. 2: ISL = sum_{k=1}^{L-1} C_k^2."""
    s = _i8(s)
    return int(lib().lo_isl(_ptr(s), s.size))


def psl(s) -> int:
    """Section 1: PSL = max_k |C_k|, k = 1..L-1."""
    s = _i8(s)
    return int(lib().lo_psl(_ptr(s), s.size))


def merit(L: int, isl_value: int) -> float:
    """Eq. 3: F = L^2 / (2 ISL)."""
    return float(lib().lo_merit(L, isl_value))


def skew_expand(x, L: int) -> np.ndarray:
    """Eq. 4: the n = (L+1)/2 free variables x -> the full skew-symmetric sequence."""
    x = _i8(x)
    n = (L + 1) // 2
    if x.size != n:
        raise ValueError("need n = (L+1)/2 free variables")
    s = np.empty(L, dtype=np.int8)
    if lib().lo_skew_expand(_ptr(x), L, _ptr(s)) != 0:
        raise ValueError("L must be odd")
    return s


def is_skew(s) -> bool:
    """Eq. 4 check (and +-1 values)."""
    s = _i8(s)
    return bool(lib().lo_is_skew(_ptr(s), s.size))


def hex_decode(hexstr: str, L: int) -> np.ndarray:
    """Table 1 encoding: hex -> bits, drop leading zero bits, 0 -> +1, 1 -> -1."""
    s = np.empty(L, dtype=np.int8)
    if lib().lo_hex_decode(hexstr.encode(), L, _ptr(s)) != 0:
        raise ValueError("bad hex string for L=%d" % L)
    return s


def hex_encode(s) -> str:
    """Inverse of hex_decode, ceil(L/4) upper-case digits."""
    s = _i8(s)
    out = ctypes.create_string_buffer((s.size + 3) // 4 + 1)
    if lib().lo_hex_encode(_ptr(s), s.size, out) != 0:
        raise ValueError("not a +-1 sequence")
    return out.value.decode()


def neighbor_delta(s) -> np.ndarray:
    """dISL_i for flipping free variable i = 0..n-1 (and its mirror), int64 [n]."""
    s = _i8(s)
    L = s.size
    d = np.empty((L + 1) // 2, dtype=np.int64)
    rc = lib().lo_neighbor_delta(_ptr(s), L, _ptr(d))
    if rc == -1:
        raise ValueError("sequence is not skew-symmetric")
    if rc != 0:
        raise RuntimeError("odd-lag autocorrelation change is nonzero")
    return d


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block function (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, dtype=np.uint32)
    lib().lo_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def random_start(seed: int, walker: int, restart: int, L: int) -> np.ndarray:
    """Free variables of the start (restart index `restart`) of walker `walker`."""
    x = np.empty((L + 1) // 2, dtype=np.int8)
    lib().lo_random_start(seed, walker, restart, L, _ptr(x))
    return x


def zobrist_key(L: int, i: int) -> int:
    return int(lib().lo_zobrist_key(L, i))


def fingerprint(s) -> int:
    s = _i8(s)
    return int(lib().lo_fingerprint(_ptr(s), s.size))


def walk(L: int, seed: int, walkers: int, steps: int, *, first_walker: int = 0,
         tabu_log2: int = 16, probe_cap: int = 32, patience: int = 0,
         target: tuple[int, int] = (17, 2), trace: bool = False, nthreads: int = 0,
         objective: str = "isl") -> dict:
    """Algorithm 1, self-avoiding-walk form, for walkers first_walker.. (+walkers).
    objective "isl" minimises ISL (Eq. 2); "psl" minimises PSL (Section 1) with ties
    broken by ISL, every neighbour measured from its recomputed C_k.

    Returns a dict of numpy arrays: the WalkResult fields per walker, ``best_seq`` and
    ``final_seq`` [walkers, L], and with ``trace`` the per-step ``trace_code`` and
    ``trace_isl`` [walkers, steps]."""
    if objective not in ("isl", "psl"):
        raise ValueError("objective is 'isl' or 'psl'")
    cfg = WalkCfg(tabu_log2, probe_cap, patience, target[0], target[1])
    res = (WalkResult * max(walkers, 1))()
    best = np.zeros((walkers, L), dtype=np.int8)
    final = np.zeros((walkers, L), dtype=np.int8)
    if trace:
        tc = np.zeros((walkers, steps), dtype=np.int32)
        ti = np.zeros((walkers, steps), dtype=np.int32)
        tcp, tip = _ptr(tc), _ptr(ti)
    else:
        tc = ti = None
        tcp = tip = None
    fn = lib().lo_walk_psl if objective == "psl" else lib().lo_walk
    rc = fn(L, seed, first_walker, walkers, steps, ctypes.byref(cfg),
            ctypes.cast(res, ctypes.c_void_p), _ptr(best), _ptr(final), tcp, tip, nthreads)
    if rc != 0:
        raise RuntimeError("oracle walk failed: %d" % rc)
    out = {f: np.array([getattr(res[w], f) for w in range(walkers)]) for f in WALK_RESULT_FIELDS}
    out["best_seq"] = best
    out["final_seq"] = final
    if trace:
        out["trace_code"] = tc
        out["trace_isl"] = ti
    return out


def bestfirst(L: int, seed: int, walkers: int, steps: int, *, pq_size: int = 32, first_walker: int = 0,
              tabu_log2: int = 16, probe_cap: int = 32, target: tuple[int, int] = (17, 2), trace: bool = False,
              nthreads: int = 0, second_hash: bool = False) -> dict:
    """Algorithm 1 as printed (best-first search with a priority queue of pq_size
    entries), for walkers first_walker.. (+walkers); outputs as walk().  Trace codes:
    the low 16 bits of each new S's fingerprint, TRACE_RESTART set after an HT overflow,
    -1 when the queue ran empty.  second_hash adds xLastovka's second table of evaluated
    neighbours (those it holds are skipped; ``cache_hits`` counts them)."""
    cfg = WalkCfg(tabu_log2, probe_cap, 0, target[0], target[1])
    res = (WalkResult * max(walkers, 1))()
    best = np.zeros((walkers, L), dtype=np.int8)
    final = np.zeros((walkers, L), dtype=np.int8)
    if trace:
        tc = np.zeros((walkers, steps), dtype=np.int32)
        ti = np.zeros((walkers, steps), dtype=np.int32)
        tcp, tip = _ptr(tc), _ptr(ti)
    else:
        tc = ti = None
        tcp = tip = None
    fn = lib().lo_bestfirst_cached if second_hash else lib().lo_bestfirst
    rc = fn(L, seed, first_walker, walkers, steps, ctypes.byref(cfg), pq_size,
            ctypes.cast(res, ctypes.c_void_p), _ptr(best), _ptr(final), tcp, tip, nthreads)
    if rc != 0:
        raise RuntimeError("oracle best-first search failed: %d" % rc)
    out = {f: np.array([getattr(res[w], f) for w in range(walkers)]) for f in WALK_RESULT_FIELDS}
    out["best_seq"] = best
    out["final_seq"] = final
    if trace:
        out["trace_code"] = tc
        out["trace_isl"] = ti
    return out


def enumerate_skew(L: int, nthreads: int = 0) -> tuple[int, int, int, np.ndarray]:
    """All skew-symmetric sequences with centre +1: (min ISL, #minimisers, lowest
    minimising assignment, its sequence)."""
    m = ctypes.c_int64()
    cnt = ctypes.c_uint64()
    first = ctypes.c_uint64()
    seq = np.zeros(L, dtype=np.int8)
    rc = lib().lo_enumerate(L, ctypes.byref(m), ctypes.byref(cnt), ctypes.byref(first), _ptr(seq),
                            nthreads)
    if rc != 0:
        raise ValueError("enumeration needs odd 3 <= L <= 79")
    return int(m.value), int(cnt.value), int(first.value), seq


def walk_replay(L: int, seed: int, walker: int, steps: int, *, tau: int, score_steps, scores, restart_idx,
                restart_bits, tabu_log2: int = 16, probe_cap: int = 32, patience: int = 0,
                target: tuple[int, int] = (17, 2)) -> dict:
    """One walker of the learned mode, replayed from the choices a GPU run recorded:
    scores [k][>= n] used at steps score_steps[k], restart states restart_bits [k][8] used
    at restart indices restart_idx[k]."""
    cfg = WalkCfg(tabu_log2, probe_cap, patience, target[0], target[1])
    res = WalkResult()
    ss = np.ascontiguousarray(score_steps, dtype=np.int64)
    sc = np.ascontiguousarray(scores, dtype=np.float32)
    if sc.ndim == 1:
        sc = sc.reshape(len(ss), -1)
    ri = np.ascontiguousarray(restart_idx, dtype=np.int64)
    rb = np.ascontiguousarray(restart_bits, dtype=np.uint32).reshape(-1)
    best = np.zeros(L, dtype=np.int8)
    final = np.zeros(L, dtype=np.int8)
    tc = np.zeros(steps, dtype=np.int32)
    ti = np.zeros(steps, dtype=np.int32)
    stride = sc.shape[1] if sc.size else 1
    rc = lib().lo_walk_replay(L, seed, walker, steps, ctypes.byref(cfg), tau, len(ss), _ptr(ss), _ptr(sc), stride,
                              len(ri), _ptr(ri), _ptr(rb), ctypes.byref(res), _ptr(best), _ptr(final), _ptr(tc),
                              _ptr(ti))
    if rc != 0:
        raise RuntimeError("oracle replay failed: %d" % rc)
    out = {f: getattr(res, f) for f in WALK_RESULT_FIELDS}
    out.update(best_seq=best, final_seq=final, trace_code=tc, trace_isl=ti)
    return out
