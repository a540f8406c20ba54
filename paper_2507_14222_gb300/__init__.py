"""Python binding of the GB300 IG library (include/ig.h).

Argument marshalling only: every step of Interpretable Generalization --
encoding (Section 3.1, Eq. 5), candidate generation (Eq. 1), coherence
(Eq. 3 / Eq. 6), supports and scores (Eq. 2), evidence (Eq. 4) and labels
(Regulations 1-3) -- runs in the library's CUDA kernels.  PyTorch provides
device memory and the current stream.  The functions take either CUDA
tensors (work is enqueued on the current stream) or numpy arrays (host
buffers: the library copies in and out itself).

Packed words are carried in torch.int64 / numpy.uint64 arrays: the library
reads and writes the same 64 bits either way.

There is no fallback: if the compiled library is missing or no GPU is usable,
every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import buildlib as _build

NORMAL = 0
ATTACK = 1

IG_OK = 0
_ERRORS = {-1: "IG_E_INVAL", -2: "IG_E_NOMEM", -3: "IG_E_CUDA",
           -4: "IG_E_TIMEOUT", -5: "IG_E_OVERFLOW", -6: "IG_E_INTERNAL",
           -7: "IG_E_IO"}
PROF_STAGES = 20


class IGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class ig_params(ctypes.Structure):
    _fields_ = [("r", ctypes.c_double), ("reg3_enabled", ctypes.c_int32),
                ("subset_kernel", ctypes.c_int32), ("index_max_q", ctypes.c_int32),
                ("index_flip_factor", ctypes.c_int32)]


def make_params(r=None, subset_kernel=0, index_max_q=0, index_flip_factor=0) -> ig_params:
    return ig_params(float(r) if r is not None else 0.0, 1 if r is not None else 0,
                     int(subset_kernel), int(index_max_q), int(index_flip_factor))


class ig_model_info_t(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("reg3_enabled", ctypes.c_int32),
                ("n_train", ctypes.c_int64 * 2),
                ("n_candidates", ctypes.c_int64 * 2),
                ("n_patterns", ctypes.c_int64 * 2),
                ("n_pairs", ctypes.c_int64 * 2),
                ("reg3_mu", ctypes.c_double), ("reg3_sigma", ctypes.c_double),
                ("reg3_r", ctypes.c_double),
                ("reg3_threshold", ctypes.c_double),
                ("coherence_tests", ctypes.c_int64 * 2),
                ("coherence_tests_tc", ctypes.c_int64 * 2),
                ("coherence_tests_idx", ctypes.c_int64 * 2),
                ("support_tests", ctypes.c_int64 * 2),
                ("subset_kernel", ctypes.c_int32), ("reserved", ctypes.c_int32)]


# Every symbol of include/ig.h with its ctypes signature.
_P, _I64, _I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
SIGNATURES = {
    "ig_encode": (ctypes.c_int, [_P, _I64, _I32, _P, _P, _I32, _P]),
    "ig_fit": (ctypes.c_int, [_P, _P, _I64, _I32, _P, _P, _P]),
    "ig_model_info": (ctypes.c_int, [_P, _P]),
    "ig_model_patterns": (ctypes.c_int, [_P, _I32, _P, _P, _P]),
    "ig_model_copy_patterns": (ctypes.c_int, [_P, _I32, _P, _P, _P, _P]),
    "ig_score": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P, _P]),
    "ig_model_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "ig_model_load": (ctypes.c_int, [ctypes.c_char_p, _P]),
    "ig_model_free": (None, [_P]),
    "ig_last_error": (ctypes.c_char_p, []),
    "ig_prof_enable": (ctypes.c_int, [_I32]),
    "ig_prof_select": (ctypes.c_int, [ctypes.c_uint32]),
    "ig_prof_reset": (ctypes.c_int, []),
    "ig_prof_read": (ctypes.c_int, [_P, _P]),
    "ig_prof_stage_name": (ctypes.c_char_p, [_I32]),
    "ig_launch_count": (ctypes.c_int64, []),
    "ig_prof_read_work": (ctypes.c_int, [_P]),
    "ig_prof_timeline": (ctypes.c_int, [_P, _P, _P, _P, _I64, _P]),
    "ig_score_noalloc": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P, _P]),
    "ig_fit_batched": (ctypes.c_int, [_P, _I32, _P, _I32, _P, _P]),
    "ig_score_batched": (ctypes.c_int, [_P, _I32, _I32, _P]),
    "ig_probe": (ctypes.c_int, [_I32, _I32, _P, _P, _P]),
    "ig_model_from_patterns": (ctypes.c_int, [_I32, _P, _P, _P, _P, _P]),
    "ig_server_create": (ctypes.c_int, [_P, _P, _P]),
    "ig_server_submit": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P, _P]),
    "ig_server_wait": (ctypes.c_int, [_P, ctypes.c_uint64, _P]),
    "ig_server_stats": (ctypes.c_int, [_P, _P, _P]),
    "ig_server_destroy": (None, [_P]),
    "ig_discretize": (ctypes.c_int, [_P, _I64, _P, _I64, _I32, _P, _I32, _P, _P]),
    "ig_filter_contradictions": (ctypes.c_int, [_P, _P, _I64, _I32, _I32, _P, _P]),
    "ig_evaluate": (ctypes.c_int, [_P, _P, _P, _P, _I64, _P]),
    "ig_reg3_sweep": (ctypes.c_int, [_P, _P, _P, _I64, ctypes.c_double, ctypes.c_double,
                                     _P, _I32, _P]),
}
SCORE_NOALLOC_MAX_ROWS = 262144

_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Loads libig_gb300.so (built by build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(
            f"IG CUDA library not built ({path} missing): run "
            "paper_2507_14222_gb300.buildlib.build() first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def build(force: bool = False) -> str:
    return _build.build(force=force)


def _check(rc: int):
    if rc != IG_OK:
        raise IGError(rc, load().ig_last_error().decode(errors="replace"))


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(x):
    """Data pointer of a contiguous torch tensor or numpy array."""
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(x.ctypes.data)


def _rows_shape(rows):
    if rows.ndim != 2:
        raise ValueError("rows must be [n, K]")
    return int(rows.shape[0]), int(rows.shape[1])


# Element types a tensor may have where the library reads 8-byte words,
# 2-byte codes, 1-byte labels and 4-byte supports (names missing from the
# installed torch are skipped).
_WORD_TYPES = ("int64", "uint64")
_CODE_TYPES = ("int16", "uint16")
_LABEL_TYPES = ("uint8", "int8", "bool")
_SUPPORT_TYPES = ("int32", "uint32")


def _torch_type_ok(x, names) -> bool:
    import torch
    return any(getattr(torch, name, None) == x.dtype for name in names)


def _check_words(rows, what="rows"):
    """[n, K] packed rows: the library reads n x K 8-byte words, so a tensor
    of another element size is rejected before anything is launched."""
    n, K = _rows_shape(rows)
    if _is_torch(rows) and not _torch_type_ok(rows, _WORD_TYPES):
        raise ValueError(f"{what} must hold 64-bit words (torch.int64 / numpy.uint64)")
    return n, K


def _check_vector(x, n: int, names, what: str):
    """A [n] array the library reads n elements of."""
    if x.ndim != 1 or int(x.shape[0]) != n:
        raise ValueError(f"{what} must have shape [{n}], not {tuple(x.shape)}")
    if _is_torch(x) and not _torch_type_ok(x, names):
        raise ValueError(f"{what}: element type {x.dtype} is not one of {', '.join(names)}")


def ig_encode(codes, cards, stream=None):
    """One-hot packing (Section 3.1, Eq. 5) of codes[n, F] with cards[F].

    codes: CUDA tensor (uint16/int16) or numpy uint16 array.  Returns the
    packed rows as a CUDA int64 tensor or a numpy uint64 array, matching the
    input's kind.
    """
    lib = load()
    cards = np.ascontiguousarray(np.asarray(cards, dtype=np.uint16))
    if codes.ndim != 2:
        raise ValueError("codes must be [n, F]")
    if _is_torch(codes) and not _torch_type_ok(codes, _CODE_TYPES):
        raise ValueError("codes must hold 16-bit codes (torch.int16 / numpy.uint16)")
    n, F = int(codes.shape[0]), int(codes.shape[1])
    if cards.ndim != 1 or int(cards.shape[0]) != F:
        raise ValueError(f"cards must have shape [{F}]")
    K = (int(cards.astype(np.int64).sum()) + 63) // 64
    if _is_torch(codes):
        import torch
        out = torch.empty((n, K), dtype=torch.int64, device=codes.device)
    else:
        codes = np.ascontiguousarray(codes, dtype=np.uint16)
        out = np.empty((n, K), dtype=np.uint64)
    _check(lib.ig_encode(_ptr(codes), n, F, _ptr(cards), _ptr(out), K,
                         _stream(stream) if _is_torch(codes) else None))
    return out


class Model:
    """A fitted IG model (coherent dictionaries P+ / P-) owned by the library."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = ig_model_info_t()
        _check(load().ig_model_info(self._h, ctypes.byref(inf)))
        return {"K": inf.K, "reg3_enabled": bool(inf.reg3_enabled),
                "n_train": tuple(inf.n_train),
                "n_candidates": tuple(inf.n_candidates),
                "n_patterns": tuple(inf.n_patterns),
                "n_pairs": tuple(inf.n_pairs),
                "reg3": (inf.reg3_mu, inf.reg3_sigma, inf.reg3_r,
                         inf.reg3_threshold),
                "coherence_tests": tuple(inf.coherence_tests),
                "coherence_tests_tc": tuple(inf.coherence_tests_tc),
                "coherence_tests_idx": tuple(inf.coherence_tests_idx),
                "support_tests": tuple(inf.support_tests),
                "subset_kernel": inf.subset_kernel}

    def patterns(self, cls: int, device: str | None = None):
        """(words uint64[P, K], support uint32[P], score uint64[P]) of class cls.

        With device=None the arrays come back as numpy arrays (host copies);
        otherwise as tensors on that CUDA device.
        """
        inf = self.info()
        P, K = inf["n_patterns"][cls], inf["K"]
        if device is None:
            w = np.empty((P, K), np.uint64)
            f = np.empty(P, np.uint32)
            s = np.empty(P, np.uint64)
            stream = None
        else:
            import torch
            w = torch.empty((P, K), dtype=torch.int64, device=device)
            f = torch.empty(P, dtype=torch.int32, device=device)
            s = torch.empty(P, dtype=torch.int64, device=device)
            stream = _stream(None)
        _check(load().ig_model_copy_patterns(self._h, cls, _ptr(w), _ptr(f),
                                             _ptr(s), stream))
        return w, f, s

    def save(self, path: str):
        _check(load().ig_model_save(self._h, path.encode()))

    def free(self):
        if self._h:
            load().ig_model_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def ig_fit(rows, labels, r: float | None = None, subset_kernel: int = 0,
           stream=None, index_max_q: int = 0, index_flip_factor: int = 0) -> Model:
    """IG training (Section 3.1: Eq. 1, Eq. 3, Eq. 2; Regulation 3 if r given).

    rows: [n, K] packed records (CUDA int64 tensor or numpy uint64 array);
    labels: [n] uint8, 1 = attack, 0 = normal.
    """
    lib = load()
    n, K = _check_words(rows)
    if not _is_torch(rows):
        rows = np.ascontiguousarray(rows, dtype=np.uint64)
    if not _is_torch(labels):
        labels = np.ascontiguousarray(labels, dtype=np.uint8)
    _check_vector(labels, n, _LABEL_TYPES, "labels")
    prm = make_params(r, subset_kernel, index_max_q, index_flip_factor)
    h = ctypes.c_void_p()
    _check(lib.ig_fit(_ptr(rows), _ptr(labels), n, K, ctypes.byref(prm),
                      ctypes.byref(h), _stream(stream) if _is_torch(rows) else None))
    return Model(h)


class ig_problem(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_void_p), ("labels", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("K", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("params", ctypes.c_void_p)]


def ig_fit_batched(problems, r: float | None = None, subset_kernel: int = 0,
                   lanes: int = 0, stream=None, per_problem_params=None) -> list:
    """Fits independent problems [(rows, labels), ...] concurrently.

    Each problem is fitted exactly as ig_fit would; returns one Model per
    problem, in order.  Arrays may be CUDA tensors or numpy arrays.
    per_problem_params: optional list of ig_params (or None entries) that
    override the batch parameters problem by problem.
    """
    lib = load()
    keep = []
    arr = (ig_problem * max(1, len(problems)))()
    any_torch = False
    for i, (rows, labels) in enumerate(problems):
        n, K = _check_words(rows, f"problem {i}: rows")
        if _is_torch(rows):
            any_torch = True
        else:
            rows = np.ascontiguousarray(rows, dtype=np.uint64)
        if not _is_torch(labels):
            labels = np.ascontiguousarray(labels, dtype=np.uint8)
        _check_vector(labels, n, _LABEL_TYPES, f"problem {i}: labels")
        keep.append((rows, labels))
        pp = per_problem_params[i] if per_problem_params else None
        if pp is not None:
            keep.append(pp)
        arr[i] = ig_problem(_ptr(rows), _ptr(labels), n, K, 0,
                            ctypes.cast(ctypes.pointer(pp), ctypes.c_void_p) if pp is not None
                            else None)
    prm = make_params(r, subset_kernel)
    outs = (ctypes.c_void_p * max(1, len(problems)))()
    _check(lib.ig_fit_batched(arr, len(problems), ctypes.byref(prm), int(lanes), outs,
                              _stream(stream) if any_torch else None))
    return [Model(ctypes.c_void_p(outs[i])) for i in range(len(problems))]


class ig_score_job(ctypes.Structure):
    _fields_ = [("model", ctypes.c_void_p), ("rows", ctypes.c_void_p), ("m", ctypes.c_int64),
                ("A_out", ctypes.c_void_p), ("N_out", ctypes.c_void_p),
                ("label_out", ctypes.c_void_p)]


def ig_score_batched(jobs, lanes: int = 0, stream=None) -> list:
    """Scores independent batches [(model, rows), ...] concurrently, each
    exactly as ig_score would; returns [(A, N, labels), ...] in order."""
    lib = load()
    arr = (ig_score_job * max(1, len(jobs)))()
    keep, outs = [], []
    any_torch = False
    for i, (model, rows) in enumerate(jobs):
        m, _ = _check_score_rows(model, rows)
        if _is_torch(rows):
            import torch
            any_torch = True
            A = torch.empty(m, dtype=torch.int64, device=rows.device)
            N = torch.empty(m, dtype=torch.int64, device=rows.device)
            lab = torch.empty(m, dtype=torch.uint8, device=rows.device)
        else:
            rows = np.ascontiguousarray(rows, dtype=np.uint64)
            A = np.empty(m, np.int64)
            N = np.empty(m, np.int64)
            lab = np.empty(m, np.uint8)
        keep.append(rows)
        outs.append((A, N, lab))
        arr[i] = ig_score_job(model.handle, _ptr(rows), m, _ptr(A), _ptr(N), _ptr(lab))
    _check(lib.ig_score_batched(arr, len(jobs), int(lanes),
                                _stream(stream) if any_torch else None))
    return outs


def _check_score_rows(model: Model, rows):
    """Scoring reads m x K 8-byte words with K from the model: reject rows of
    another width or element size before anything is launched."""
    m, K = _check_words(rows)
    if not _is_torch(rows) and np.asarray(rows).dtype.itemsize != 8:
        raise ValueError("rows must hold 64-bit words (torch.int64 / numpy.uint64)")
    mk = model.info()["K"]
    if K != mk:
        raise ValueError(f"rows have {K} words per record but the model has K = {mk}")
    return m, K


def ig_score(model: Model, rows, stream=None):
    """IG inference (Eq. 4, Regulations 1-3): returns (A, N, labels)."""
    lib = load()
    m, K = _check_score_rows(model, rows)
    if _is_torch(rows):
        import torch
        A = torch.empty(m, dtype=torch.int64, device=rows.device)
        N = torch.empty(m, dtype=torch.int64, device=rows.device)
        lab = torch.empty(m, dtype=torch.uint8, device=rows.device)
        stream = _stream(stream)
    else:
        rows = np.ascontiguousarray(rows, dtype=np.uint64)
        A = np.empty(m, np.int64)
        N = np.empty(m, np.int64)
        lab = np.empty(m, np.uint8)
        stream = None
    _check(lib.ig_score(model.handle, _ptr(rows), m, _ptr(A), _ptr(N), _ptr(lab),
                        stream))
    return A, N, lab


def ig_score_noalloc(model: Model, rows, stream=None):
    """ig_score without any device allocation inside the library.

    For callers that cannot let the library allocate device memory (a
    latency-bound scoring loop, or a process whose device memory is already
    reserved by another allocator).  rows must be a CUDA tensor with at most
    SCORE_NOALLOC_MAX_ROWS rows; the outputs are allocated here by PyTorch,
    the caller's allocator.  Returns (A, N, labels) like ig_score.
    """
    import torch
    if not _is_torch(rows) or not rows.is_cuda:
        raise ValueError("ig_score_noalloc takes CUDA tensors only")
    m, _ = _check_score_rows(model, rows)
    A = torch.empty(m, dtype=torch.int64, device=rows.device)
    N = torch.empty(m, dtype=torch.int64, device=rows.device)
    lab = torch.empty(m, dtype=torch.uint8, device=rows.device)
    _check(load().ig_score_noalloc(model.handle, _ptr(rows), m, _ptr(A), _ptr(N),
                                   _ptr(lab), _stream(stream)))
    return A, N, lab


def ig_model_from_patterns(words_normal, support_normal, words_attack, support_attack,
                           stream=None) -> Model:
    """A model holding given pattern sets (class 0 normal, 1 attack).

    words_*: [P, K] packed patterns (numpy uint64 or CUDA int64 tensors, any
    order, distinct, non-empty); support_*: [P] supports.  Scores follow
    Eq. 2.
    """
    lib = load()
    ws, fs = [], []
    any_torch = False
    for c, (w, f) in enumerate(((words_normal, support_normal), (words_attack, support_attack))):
        if _is_torch(w):
            any_torch = True
        else:
            w = np.ascontiguousarray(w, dtype=np.uint64)
        P, _ = _check_words(w, f"class {c}: words")
        if not _is_torch(f):
            f = np.ascontiguousarray(f, dtype=np.uint32)
        _check_vector(f, P, _SUPPORT_TYPES, f"class {c}: support")
        ws.append(w)
        fs.append(f)
    if int(ws[0].shape[1]) != int(ws[1].shape[1]):
        raise ValueError("both classes' words must have the same K")
    K = int(ws[0].shape[1])
    wp = (ctypes.c_void_p * 2)(*[_ptr(w).value for w in ws])
    fp = (ctypes.c_void_p * 2)(*[_ptr(f).value for f in fs])
    n = (ctypes.c_int64 * 2)(int(ws[0].shape[0]), int(ws[1].shape[0]))
    h = ctypes.c_void_p()
    _check(lib.ig_model_from_patterns(K, wp, fp, n, ctypes.byref(h),
                                      _stream(stream) if any_torch else None))
    return Model(h)


class ig_server_config(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("max_batch_flows", ctypes.c_int64), ("memory_budget_bytes", ctypes.c_int64)]


class Server:
    """Continuous-batching scoring server over a model (see include/ig.h).

    submit() queues host (numpy) flows and returns a handle; wait() blocks
    until the request's (A, N, labels) are filled and returns its latency in
    milliseconds.
    """

    def __init__(self, model: Model, slots: int = 0, max_batch_flows: int = 0,
                 memory_budget_bytes: int = 0):
        self.model = model
        cfg = ig_server_config(int(slots), 0, int(max_batch_flows), int(memory_budget_bytes))
        h = ctypes.c_void_p()
        _check(load().ig_server_create(model.handle, ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._K = int(model.info()["K"])
        self._pending = {}

    def submit(self, rows) -> int:
        rows = np.ascontiguousarray(rows, dtype=np.uint64)
        if rows.ndim != 2 or int(rows.shape[1]) != self._K:   # the server reads m x K words
            raise ValueError(f"rows must be [m, {self._K}] (the model's K), not {rows.shape}")
        m = int(rows.shape[0])
        A = np.empty(m, np.int64)
        N = np.empty(m, np.int64)
        lab = np.empty(m, np.uint8)
        t = ctypes.c_uint64()
        _check(load().ig_server_submit(self._h, _ptr(rows), m, _ptr(A), _ptr(N), _ptr(lab),
                                       ctypes.byref(t)))
        self._pending[t.value] = (rows, A, N, lab)
        return t.value

    def wait(self, ticket: int):
        """-> (A, N, labels, latency_ms)."""
        lat = ctypes.c_double()
        rc = load().ig_server_wait(self._h, ctypes.c_uint64(ticket), ctypes.byref(lat))
        rows, A, N, lab = self._pending.pop(ticket)
        _check(rc)
        return A, N, lab, lat.value

    def stats(self):
        b, f = ctypes.c_int64(), ctypes.c_int64()
        _check(load().ig_server_stats(self._h, ctypes.byref(b), ctypes.byref(f)))
        return b.value, f.value

    def close(self):
        if self._h:
            load().ig_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ig_model_load(path: str) -> Model:
    h = ctypes.c_void_p()
    _check(load().ig_model_load(path.encode(), ctypes.byref(h)))
    return Model(h)


def prof_enable(on: bool = True):
    _check(load().ig_prof_enable(1 if on else 0))


def prof_select(stages=None):
    """Time only the named stages (all when None) while profiling is on."""
    if stages is None:
        mask = 0xFFFFFFFF
    else:
        lib = load()
        names = {lib.ig_prof_stage_name(i).decode(): i for i in range(PROF_STAGES)}
        mask = 0
        for name in stages:
            mask |= 1 << names[name]
    _check(load().ig_prof_select(mask))


def prof_reset():
    _check(load().ig_prof_reset())


def prof_read() -> dict:
    """{stage name: (total ms, timed launches, executed tests)} since reset."""
    lib = load()
    ms = (ctypes.c_double * PROF_STAGES)()
    n = (ctypes.c_int64 * PROF_STAGES)()
    w = (ctypes.c_int64 * PROF_STAGES)()
    _check(lib.ig_prof_read(ms, n))
    _check(lib.ig_prof_read_work(w))
    return {lib.ig_prof_stage_name(i).decode(): (ms[i], n[i], w[i])
            for i in range(PROF_STAGES)}


def prof_timeline() -> list:
    """Stage spans since the last prof_reset(): [(stage name, stream id,
    begin ms, end ms)], in the order they were recorded."""
    lib = load()
    n = ctypes.c_int64()
    _check(lib.ig_prof_timeline(None, None, None, None, 0, ctypes.byref(n)))
    k = n.value
    st = np.zeros(max(k, 1), np.int32)
    sid = np.zeros(max(k, 1), np.uint64)
    t0 = np.zeros(max(k, 1), np.float64)
    t1 = np.zeros(max(k, 1), np.float64)
    _check(lib.ig_prof_timeline(_ptr(st), _ptr(sid), _ptr(t0), _ptr(t1), k, ctypes.byref(n)))
    return [(lib.ig_prof_stage_name(int(st[i])).decode(), int(sid[i]), float(t0[i]), float(t1[i]))
            for i in range(k)]


PROBES = {"lop3": 0, "l2_read": 1, "l2_random": 2, "mma_f8_smem": 3, "mma_f8_tmem": 4}


def probe(name: str, arg: int = 0) -> dict:
    """One throughput probe of the current GPU (ig_probe): {"rate": per second,
    "ms": timed launch, "cycles": SM clocks of the slowest CTA (MMA probes)}."""
    rate, ms, cyc = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().ig_probe(PROBES[name], int(arg), ctypes.byref(rate), ctypes.byref(ms),
                           ctypes.byref(cyc)))
    return {"rate": rate.value, "ms": ms.value, "cycles": cyc.value}


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    return int(load().ig_launch_count())


# Short aliases.
encode, fit, score, model_load = ig_encode, ig_fit, ig_score, ig_model_load


# ---- host helpers (include/ig_helpers.h): host arrays only ------------------

class ig_metrics_t(ctypes.Structure):
    _fields_ = [("tp", ctypes.c_int64), ("fp", ctypes.c_int64),
                ("tn", ctypes.c_int64), ("fn", ctypes.c_int64),
                ("accuracy", ctypes.c_double), ("precision", ctypes.c_double),
                ("recall", ctypes.c_double), ("f1", ctypes.c_double),
                ("auc", ctypes.c_double)]


def _host(x, dtype):
    """A C-contiguous numpy copy (or view) of x on the host."""
    if _is_torch(x):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(x), dtype=dtype)


def _metrics_dict(m: ig_metrics_t) -> dict:
    return {k: getattr(m, k) for k, _ in ig_metrics_t._fields_}


def ig_discretize(fit_values, categorical, p: int, values=None):
    """Section 3.1 discretiser: (codes uint16[n, F], cards uint16[F]).

    fit_values: float[n_fit, F] (NaN = missing) -- statistics and vocabulary;
    values: rows to code (default: fit_values); categorical: bool[F]."""
    fit = _host(fit_values, np.float64)
    vals = fit if values is None else _host(values, np.float64)
    if fit.ndim != 2 or vals.ndim != 2 or vals.shape[1] != fit.shape[1]:
        raise ValueError("fit_values and values must be [n, F] with the same F")
    F = fit.shape[1]
    cat = _host(categorical, np.uint8)
    if cat.shape != (F,):
        raise ValueError("categorical must have one entry per column")
    codes = np.empty(vals.shape, np.uint16)
    cards = np.empty(F, np.uint16)
    _check(load().ig_discretize(_ptr(fit), fit.shape[0], _ptr(vals), vals.shape[0], F,
                                _ptr(cat), int(p), _ptr(codes), _ptr(cards)))
    return codes, cards


def ig_filter_contradictions(rows, labels, mode: int = 0):
    """Anti-contradiction filter: bool[n] mask of the records kept."""
    r = _host(rows, np.uint64)
    lab = _host(labels, np.uint8)
    if r.ndim != 2 or lab.shape != (r.shape[0],):
        raise ValueError("rows must be [n, K] and labels [n]")
    keep = np.empty(r.shape[0], np.uint8)
    _check(load().ig_filter_contradictions(_ptr(r), _ptr(lab), r.shape[0], r.shape[1],
                                           int(mode), _ptr(keep), None))
    return keep.astype(bool)


def ig_evaluate(y_true, y_pred, A=None, N=None) -> dict:
    """Accuracy, precision, recall, F1 and (with A, N) the AUC of A - N."""
    yt = _host(y_true, np.uint8)
    yp = _host(y_pred, np.uint8)
    if yp.shape != yt.shape or yt.ndim != 1:
        raise ValueError("y_true and y_pred must be 1-D of one length")
    a = n_ = None
    if (A is None) != (N is None):
        raise ValueError("give both A and N, or neither")
    if A is not None:
        a, n_ = _host(A, np.int64), _host(N, np.int64)
        if a.shape != yt.shape or n_.shape != yt.shape:
            raise ValueError("A and N must have one entry per record")
    out = ig_metrics_t()
    _check(load().ig_evaluate(_ptr(yt), _ptr(yp), _ptr(a) if a is not None else None,
                              _ptr(n_) if n_ is not None else None, yt.shape[0],
                              ctypes.byref(out)))
    return _metrics_dict(out)


def ig_reg3_sweep(A, N, y_true, mu: float, sigma: float, rs) -> list:
    """Metrics of Regulations 1-3 for each r in rs (one dict per r)."""
    a, n_, yt = _host(A, np.int64), _host(N, np.int64), _host(y_true, np.uint8)
    if not (a.shape == n_.shape == yt.shape) or yt.ndim != 1:
        raise ValueError("A, N and y_true must be 1-D of one length")
    r = _host(rs, np.float64).reshape(-1)
    out = (ig_metrics_t * max(1, r.shape[0]))()
    _check(load().ig_reg3_sweep(_ptr(a), _ptr(n_), _ptr(yt), yt.shape[0], float(mu),
                                float(sigma), _ptr(r), r.shape[0], out))
    return [dict(_metrics_dict(out[k]), r=float(r[k])) for k in range(r.shape[0])]
