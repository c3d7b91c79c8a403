"""Thin ctypes binding of liblp (include/lp.h): argument marshalling only.

Every step of the fixpoint runs in liblp's CUDA kernels; this module never computes a model.
Buffers may be torch tensors (CUDA or CPU), numpy arrays, or anything exposing ``data_ptr()``;
bit vectors are 64-bit words (torch.int64 / numpy uint64) in the layout of lp.h.
"""
import ctypes
import os

import numpy as np

from . import _build

OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_NO_FIXPOINT, ERR_TOO_MANY_GUESSES, ERR_TIMEOUT = range(7)
STATUS_NAMES = ["LP_OK", "LP_ERR_INVALID", "LP_ERR_OOM", "LP_ERR_CUDA", "LP_ERR_NO_FIXPOINT",
                "LP_ERR_TOO_MANY_GUESSES", "LP_ERR_TIMEOUT"]
LP_ROWS, LP_TIMING = 1, 2
LP_COMPILE_HOST_ONLY = 1
LP_COMPILE_ON_HOST = 2
LP_COMPILE_ON_DEVICE = 4
LP_BATCH_FULL_SWEEP = 1
LP_BATCH_FROM_M0 = 2


class LPError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class _Info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "n_atoms", "n_rules", "n_prime", "nnz", "n_barred", "n_aux", "k", "n_fact_rows", "n_and_rows",
        "n_or_rows", "device_bytes", "upload_bytes")] + [("compile_ms", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32), ("kernel_ms", ctypes.c_float),
                ("launches", ctypes.c_int64), ("tiles", ctypes.c_int64), ("tile_words", ctypes.c_int64),
                ("max_tile_iters", ctypes.c_int64), ("sum_tile_iters", ctypes.c_int64),
                ("frontier_rows", ctypes.c_int64), ("frontier_entries", ctypes.c_int64),
                ("frontier_list", ctypes.c_int64), ("frontier_deps", ctypes.c_int64)]


EXPORTS = ["lp_compile", "lp_program_info", "lp_least_model", "lp_stable_models", "lp_last_solve_stats",
           "lp_export_matrix", "lp_free", "lp_last_error", "lp_launch_count", "lp_least_model_static",
           "lp_relaxed_workspace", "lp_relaxed_forward", "lp_relaxed_backward", "lp_compile_batch", "lp_batch_info",
           "lp_batch_program_info", "lp_batch_stable_models", "lp_batch_free", "lp_get_schedule", "lp_set_schedule",
           "lp_autotune", "lp_stable_search", "lp_check_grid_barrier", "lp_check_matrix", "lp_debug_fail_alloc",
           "lp_debug_internal", "lp_batch_last_stats"]

LP_TUNE_LEAST = 1
LP_TUNE_STABLE = 2
SCHEDULE_FIELDS = ("fixpoint_kernel", "fixpoint_blocks_per_sm", "fixpoint_row_split", "fixpoint_chunk_batch",
                   "fixpoint_row_map", "stable_tile_words", "stable_blocks_per_sm", "stable_row_split",
                   "stable_frontier", "fixpoint_stage")


class _Schedule(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int32) for f in SCHEDULE_FIELDS]


class _TuneRecord(ctypes.Structure):
    _fields_ = [("schedule", _Schedule), ("solve", ctypes.c_int32), ("ms", ctypes.c_float)]

# Version of the schedule fields and their meaning (row maps, kernels); part of the key of
# autotune_cached, so a cache written by another build is not applied.
SCHEDULE_FORMAT = 3

_lib = None


def _device_key():
    """Name and SM count of the current CUDA device: a tuned schedule belongs to one device."""
    try:
        import torch
        if torch.cuda.is_available():
            prop = torch.cuda.get_device_properties(torch.cuda.current_device())
            return f"{prop.name}/{prop.multi_processor_count}SM"
    except Exception:  # pragma: no cover
        pass
    return "nodevice"


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load liblp.so (fails loudly if it was not built; there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"liblp is not built ({path} missing): run __graft_entry__.build()")
        _build.build()
    L = ctypes.CDLL(path)
    P, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    L.lp_compile.argtypes = [i32, i64, P, P, P, P, u32, P, ctypes.POINTER(P)]
    L.lp_program_info.argtypes = [P, ctypes.POINTER(_Info)]
    L.lp_least_model.argtypes = [P, P, P, i32, u32, ctypes.POINTER(i32), P]
    L.lp_stable_models.argtypes = [P, P, i64, P, P, i64, ctypes.POINTER(i64), i32, P]
    L.lp_last_solve_stats.argtypes = [P, ctypes.POINTER(_Stats), P]
    L.lp_export_matrix.argtypes = [P, P, P, P, P, P]
    L.lp_relaxed_workspace.argtypes = [P, i32, i32, i32, ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.lp_relaxed_forward.argtypes = [P, P, P, i32, i32, ctypes.c_float, i32, P, P, P]
    L.lp_relaxed_backward.argtypes = [P, P, P, i32, i32, ctypes.c_float, i32, P, P, P, P, P]
    for name in ("lp_relaxed_workspace", "lp_relaxed_forward", "lp_relaxed_backward"):
        getattr(L, name).restype = ctypes.c_int
    L.lp_compile_batch.argtypes = [i32, P, P, P, P, P, P, u32, P, ctypes.POINTER(P)]
    L.lp_batch_info.argtypes = [P] + [ctypes.POINTER(i64)] * 5
    L.lp_batch_program_info.argtypes = [P, i32, ctypes.POINTER(_Info), ctypes.POINTER(i64)]
    L.lp_batch_stable_models.argtypes = [P, P, P, P, i32, P]
    for name in ("lp_compile_batch", "lp_batch_info", "lp_batch_program_info", "lp_batch_stable_models"):
        getattr(L, name).restype = ctypes.c_int
    L.lp_batch_last_stats.argtypes = [P, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64), P]
    L.lp_batch_last_stats.restype = ctypes.c_int
    L.lp_batch_free.argtypes = [P]
    L.lp_batch_free.restype = None
    L.lp_get_schedule.argtypes = [P, ctypes.POINTER(_Schedule)]
    L.lp_set_schedule.argtypes = [P, ctypes.POINTER(_Schedule)]
    L.lp_autotune.argtypes = [P, u32, i32, ctypes.POINTER(_TuneRecord), i32, ctypes.POINTER(i32), P]
    L.lp_stable_search.argtypes = [P, i32, i32, ctypes.c_uint64, P, i64, ctypes.POINTER(i64), P]
    L.lp_check_grid_barrier.argtypes = [i32, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float), P]
    L.lp_check_matrix.argtypes = [P, ctypes.POINTER(i64), P]
    L.lp_debug_fail_alloc.argtypes = [i64]
    L.lp_debug_fail_alloc.restype = None
    L.lp_debug_internal.argtypes = [P, i32, P, ctypes.POINTER(i64), P]
    for name in ("lp_get_schedule", "lp_set_schedule", "lp_autotune", "lp_stable_search", "lp_check_grid_barrier",
                 "lp_check_matrix", "lp_debug_internal"):
        getattr(L, name).restype = ctypes.c_int
    L.lp_least_model_static.argtypes = [i32, P, P, P, P, P, i32, ctypes.POINTER(i32), P]
    L.lp_least_model_static.restype = ctypes.c_int
    L.lp_free.argtypes = [P]
    L.lp_free.restype = None
    L.lp_last_error.restype = ctypes.c_char_p
    L.lp_launch_count.restype = ctypes.c_int64
    for name in ("lp_compile", "lp_program_info", "lp_least_model", "lp_stable_models", "lp_last_solve_stats",
                 "lp_export_matrix"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status):
    if status != OK:
        raise LPError(status, load().lp_last_error().decode())


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if hasattr(x, "is_contiguous") and not x.is_contiguous():
            raise ValueError("tensor must be contiguous (liblp reads and writes buffers as dense arrays)")
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def least_model_static(n_rows, row_ptr, col, threshold, v0, out, max_iters=1 << 30, sync=True, stream=None):
    """lp_least_model_static: Algorithm 1 on caller-held device buffers, no allocation.
    Returns the iteration count when sync."""
    it = ctypes.c_int32(-1)
    _check(load().lp_least_model_static(int(n_rows), _ptr(row_ptr), _ptr(col), _ptr(threshold), _ptr(v0), _ptr(out),
                                        int(max_iters), ctypes.byref(it) if sync else None, _stream(stream)))
    return it.value if sync else None


def check_grid_barrier(blocks, absent, limit_us, stream=None):
    """lp_check_grid_barrier: (status, ms) of one bounded grid barrier with `absent` blocks missing."""
    st, ms = ctypes.c_int32(), ctypes.c_float()
    _check(load().lp_check_grid_barrier(int(blocks), int(absent), int(limit_us), ctypes.byref(st), ctypes.byref(ms),
                                        _stream(stream)))
    return st.value, ms.value


def debug_fail_alloc(after: int) -> None:
    """lp_debug_fail_alloc: the allocation after `after` more successful ones fails (once); -1 = off."""
    load().lp_debug_fail_alloc(int(after))


def launch_count() -> int:
    return int(load().lp_launch_count())


def words(n_bits: int) -> int:
    return max(1, (n_bits + 63) // 64)


class Program:
    """A compiled program (owns the liblp handle)."""

    def __init__(self, n_atoms, head, body_off, body_atom, body_neg=None, stream=None, host_only=False,
                 on_host=False, on_device=False):
        """host_only: the host compiler alone, no device memory; on_host: the host compiler, then
        the matrix uploaded; on_device: the rules uploaded and standardized on the device (the
        default, except for programs of at most 16,384 rules plus body literals, which one host
        thread standardizes)."""
        L = load()
        self._keep = [np.ascontiguousarray(head, dtype=np.int32), np.ascontiguousarray(body_off, dtype=np.int64),
                      np.ascontiguousarray(body_atom, dtype=np.int32),
                      None if body_neg is None else np.ascontiguousarray(body_neg, dtype=np.uint8)]
        h, off, atom, neg = self._keep
        self._h = ctypes.c_void_p()
        flags = LP_COMPILE_HOST_ONLY if host_only else (LP_COMPILE_ON_HOST if on_host else 0)
        if on_device:
            flags |= LP_COMPILE_ON_DEVICE
        _check(L.lp_compile(int(n_atoms), len(h), _ptr(h), _ptr(off), _ptr(atom), _ptr(neg), flags,
                            None if host_only else _stream(stream),
                            ctypes.byref(self._h)))
        self._keep = None
        self.info = self._info()

    @classmethod
    def from_program(cls, prog, stream=None, host_only=False, on_host=False, on_device=False):
        return cls(prog.n_atoms, prog.head, prog.body_off, prog.body_atom, getattr(prog, "body_neg", None), stream,
                   host_only, on_host, on_device)

    INTERNAL = {"row_ptr": (0, np.int32), "col": (1, np.int32), "perm": (2, np.int32), "any_mask": (3, np.uint32),
                "row_tag": (4, np.int32), "fact_row": (5, np.int32), "fact_owner": (6, np.int32),
                "fact_mask": (7, np.uint64), "neg_row": (8, np.int32), "bar_row": (9, np.int32)}

    def debug_internal(self, name, stream=None):
        """An internal device array of the handle (lp_debug_internal) as a numpy array."""
        which, dt = self.INTERNAL[name]
        L = load()
        nbytes = ctypes.c_int64()
        _check(L.lp_debug_internal(self._h, which, None, ctypes.byref(nbytes), _stream(stream)))
        out = np.zeros(nbytes.value // np.dtype(dt).itemsize, dtype=dt)
        if nbytes.value:
            _check(L.lp_debug_internal(self._h, which, out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nbytes),
                                       _stream(stream)))
        return out

    def _info(self):
        i = _Info()
        _check(load().lp_program_info(self._h, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in _Info._fields_}

    def refresh_info(self):
        self.info = self._info()
        return self.info

    def least_model(self, out, init=None, max_iters=1 << 30, rows=False, timing=False, sync=True, stream=None):
        """Algorithm 1. ``out``: ceil(n/64) words (ceil(n'/64) with rows=True). Returns the
        iteration count when sync, else None (status then via last_stats)."""
        flags = (LP_ROWS if rows else 0) | (LP_TIMING if timing else 0)
        it = ctypes.c_int32(-1)
        _check(load().lp_least_model(self._h, _ptr(init), _ptr(out), int(max_iters), flags,
                                     ctypes.byref(it) if sync else None, _stream(stream)))
        return it.value if sync else None

    def stable_models(self, stable_mask, guesses=None, n_guesses=None, models=None, max_models=0,
                      max_iters=1 << 30, sync=True, stream=None):
        """Algorithms 2 + 3. Returns the number of stable guesses when sync."""
        if guesses is None and n_guesses is None:
            n_guesses = 1 << self.info["k"]
        if n_guesses is None:
            n_guesses = len(guesses)
        ns = ctypes.c_int64(-1)
        _check(load().lp_stable_models(self._h, _ptr(guesses), int(n_guesses), _ptr(stable_mask), _ptr(models),
                                       int(max_models), ctypes.byref(ns) if sync else None, int(max_iters),
                                       _stream(stream)))
        return ns.value if sync else None

    def relaxed_workspace(self, batch, steps, ckpt_every):
        """(checkpoint floats, scratch floats) for the relaxed path."""
        c, s_ = ctypes.c_int64(), ctypes.c_int64()
        _check(load().lp_relaxed_workspace(self._h, int(batch), int(steps), int(ckpt_every), ctypes.byref(c),
                                           ctypes.byref(s_)))
        return c.value, s_.value

    def relaxed_forward(self, weights, v0, batch, steps, tau, ckpt_every, ckpt, vT, stream=None):
        _check(load().lp_relaxed_forward(self._h, _ptr(weights), _ptr(v0), int(batch), int(steps), float(tau),
                                         int(ckpt_every), _ptr(ckpt), _ptr(vT), _stream(stream)))

    def relaxed_backward(self, weights, gT, batch, steps, tau, ckpt_every, ckpt, scratch, dweights, dv0,
                         stream=None):
        _check(load().lp_relaxed_backward(self._h, _ptr(weights), _ptr(gT), int(batch), int(steps), float(tau),
                                          int(ckpt_every), _ptr(ckpt), _ptr(scratch), _ptr(dweights), _ptr(dv0),
                                          _stream(stream)))

    @property
    def schedule(self):
        """The handle's schedule (lp_get_schedule) as a dict."""
        sc = _Schedule()
        _check(load().lp_get_schedule(self._h, ctypes.byref(sc)))
        return {f: getattr(sc, f) for f in SCHEDULE_FIELDS}

    def set_schedule(self, **fields):
        """Change some fields of the schedule (lp_set_schedule)."""
        cur = self.schedule
        cur.update(fields)
        sc = _Schedule(**cur)
        _check(load().lp_set_schedule(self._h, ctypes.byref(sc)))

    def autotune(self, what=LP_TUNE_LEAST | LP_TUNE_STABLE, reps=3, stream=None):
        """Time the candidate schedules (lp_autotune); returns [{schedule..., "solve", "ms"}] in run order."""
        recs = (_TuneRecord * 64)()
        n = ctypes.c_int32()
        _check(load().lp_autotune(self._h, int(what), int(reps), recs, 64, ctypes.byref(n), _stream(stream)))
        out = []
        for r in recs[:min(n.value, 64)]:
            d = {f: getattr(r.schedule, f) for f in SCHEDULE_FIELDS}
            d["solve"] = "least" if r.solve == LP_TUNE_LEAST else "stable"
            d["ms"] = r.ms
            out.append(d)
        return out

    def schedule_cache_key(self, what=LP_TUNE_LEAST | LP_TUNE_STABLE):
        """Key of autotune_cached: the device (name, SM count), the schedule format of this build
        and the program's sizes."""
        i = self.info
        return (f"{_device_key()},format={SCHEDULE_FORMAT},n'={i['n_prime']},nnz={i['nnz']},k={i['k']},"
                f"or={i['n_or_rows']},what={int(what)}")

    def autotune_cached(self, cache_path, what=LP_TUNE_LEAST | LP_TUNE_STABLE, reps=3, stream=None):
        """lp_autotune once per program shape: the chosen schedule is stored in a JSON file under a
        key of the program's sizes and reused on later calls (a schedule only changes the mapping
        onto the GPU, never the result, so two programs of the same sizes may share one). Returns
        True if the schedule came from the file, False if it was tuned now."""
        import json
        key = self.schedule_cache_key(what)
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            try:
                self.set_schedule(**{f: int(v) for f, v in cache[key].items() if f in SCHEDULE_FIELDS})
                return True
            except LPError:  # a schedule this build rejects: tune again
                pass
        self.autotune(what, reps, stream)
        cache[key] = self.schedule
        tmp = f"{cache_path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
        return False

    def stable_search(self, population=1024, rounds=16, seed=1, max_found=1 << 16, stream=None):
        """Sampled guesses + local search (lp_stable_search); returns the distinct stable guesses
        found (uint64 numpy array, ascending) and their total count."""
        out = np.zeros(max(int(max_found), 1), dtype=np.uint64)
        n = ctypes.c_int64()
        _check(load().lp_stable_search(self._h, int(population), int(rounds), ctypes.c_uint64(seed), _ptr(out),
                                       int(max_found), ctypes.byref(n), _stream(stream)))
        return out[:min(n.value, int(max_found))], n.value

    def check_matrix(self, stream=None) -> int:
        """lp_check_matrix: number of violated invariants of the compiled matrix (0 expected)."""
        n = ctypes.c_int64()
        _check(load().lp_check_matrix(self._h, ctypes.byref(n), _stream(stream)))
        return n.value

    def last_stats(self, stream=None):
        s = _Stats()
        _check(load().lp_last_solve_stats(self._h, ctypes.byref(s), _stream(stream)))
        return {f: getattr(s, f) for f, _ in _Stats._fields_}

    def export_matrix(self, stream=None):
        n, nnz = self.info["n_prime"], self.info["nnz"]
        row_ptr = np.zeros(n + 1, dtype=np.int64)
        col = np.zeros(max(nnz, 1), dtype=np.int64)
        thr = np.zeros(max(n, 1), dtype=np.int32)
        kind = np.zeros(max(n, 1), dtype=np.int8)
        _check(load().lp_export_matrix(self._h, _ptr(row_ptr), _ptr(col), _ptr(thr), _ptr(kind), _stream(stream)))
        return {"row_ptr": row_ptr, "col": col[:nnz], "threshold": thr[:n], "kind": kind[:n]}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lp_free(self._h)
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


class Batch:
    """Many independent normal programs compiled for one launch (lp_compile_batch)."""

    def __init__(self, programs, stream=None, full_sweep=False, from_m0=False):
        """full_sweep: every program evaluates every row in every iteration (LP_BATCH_FULL_SWEEP);
        by default programs with k <= 8 run the frontier schedule from F (the fixpoint from the
        fact rows with the guessed rows zero); from_m0: the frontier from M_0 (LP_BATCH_FROM_M0:
        Algorithm 2's iterates and iteration counts)."""
        L = load()
        n = len(programs)
        n_atoms = np.array([p.n_atoms for p in programs], dtype=np.int32)
        rule_off = np.zeros(n + 1, dtype=np.int64)
        rule_off[1:] = np.cumsum([len(p.head) for p in programs])
        head = np.concatenate([np.asarray(p.head, np.int32) for p in programs]) if n else np.zeros(0, np.int32)
        lit_off = np.concatenate([[0], np.cumsum([len(p.body_atom) for p in programs])]).astype(np.int64)
        body_off = np.zeros(int(rule_off[-1]) + 1, dtype=np.int64)
        for i, p in enumerate(programs):
            body_off[rule_off[i]:rule_off[i + 1] + 1] = np.asarray(p.body_off, np.int64) + lit_off[i]
        atom = np.concatenate([np.asarray(p.body_atom, np.int32) for p in programs]) if n else np.zeros(0, np.int32)
        neg = None
        if any(getattr(p, "body_neg", None) is not None for p in programs):
            neg = np.concatenate([np.asarray(p.body_neg, np.uint8) if getattr(p, "body_neg", None) is not None
                                  else np.zeros(len(p.body_atom), np.uint8) for p in programs])
        self._h = ctypes.c_void_p()
        _check(L.lp_compile_batch(n, _ptr(n_atoms), _ptr(rule_off), _ptr(head), _ptr(body_off), _ptr(atom), _ptr(neg),
                                  (LP_BATCH_FULL_SWEEP if full_sweep else 0) | (LP_BATCH_FROM_M0 if from_m0 else 0),
                                  _stream(stream), ctypes.byref(self._h)))
        vals = [ctypes.c_int64() for _ in range(5)]
        _check(L.lp_batch_info(self._h, *[ctypes.byref(v) for v in vals]))
        self.n_programs, self.total_rows, self.total_nnz, self.total_mask_words, self.device_bytes = [v.value for v in vals]
        self.k, self.mask_offset, self.info = [], [], []
        for i in range(n):
            inf, off = _Info(), ctypes.c_int64()
            _check(L.lp_batch_program_info(self._h, i, ctypes.byref(inf), ctypes.byref(off)))
            d = {f: getattr(inf, f) for f, _ in _Info._fields_}
            self.info.append(d)
            self.k.append(d["k"])
            self.mask_offset.append(off.value)

    def stable_models(self, stable_mask, n_stable=None, iters=None, max_iters=1 << 30, stream=None):
        _check(load().lp_batch_stable_models(self._h, _ptr(stable_mask), _ptr(n_stable), _ptr(iters), int(max_iters),
                                             _stream(stream)))

    def last_stats(self, stream=None):
        """Rows and entries the last solve evaluated under the frontier schedule."""
        rows, ents, byts = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().lp_batch_last_stats(self._h, ctypes.byref(rows), ctypes.byref(ents), ctypes.byref(byts),
                                          _stream(stream)))
        return {"rows_evaluated": rows.value, "entries_evaluated": ents.value, "bytes_touched": byts.value}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lp_batch_free(self._h)
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
