"""Python binding of montgb, the GB300 Montgomery-type modular arithmetic library.

Argument marshalling only: every function forwards to the C ABI declared in
``include/montgb.h`` (same names, same arguments) through ctypes.  Device
buffers may be given as CUDA ``torch.Tensor`` objects or as raw integer
addresses; streams as ``torch.cuda.Stream`` objects, raw ``cudaStream_t``
integers, or ``None`` for torch's current stream.  Every non-zero status is
raised as ``MontError``.

The library must have been built (``paper_2402_00675_gb300.build.build()``);
importing a function whose library is missing raises immediately -- there is
no fallback implementation.
"""

from __future__ import annotations

import ctypes
import os

from .build import LIB_PATH, build  # noqa: F401

MONT_OK = 0
MONT_EINVAL = 1
MONT_ENOMEM = 2
MONT_ECUDA = 3
MONT_ETIMEOUT = 4
MONT_EOVERFLOW = 5

MONT_REDC = 0
MONT_SIGNED = 1
MONT_PLANTARD = 2
MONT_SIGNED_PLANTARD = 3
MONT_SIGNED_PLANTARD2 = 4
SIGNED_VARIANTS = (MONT_SIGNED, MONT_SIGNED_PLANTARD, MONT_SIGNED_PLANTARD2)
PLANTARD_VARIANTS = (MONT_PLANTARD, MONT_SIGNED_PLANTARD, MONT_SIGNED_PLANTARD2)
MONT_MAX_LIMBS = 64

MONT_CONST_N = 0
MONT_CONST_NINV = 1
MONT_CONST_NPRIME = 2
MONT_CONST_R_MOD_N = 3
MONT_CONST_R2_MOD_N = 4
MONT_CONST_DOMAIN_R2 = 5

MONT_DOMAIN_DEFAULT = 0
MONT_DOMAIN_REDC = 1
MONT_DOMAIN_EXPLICIT = 2
MONT_RANGE_DEFAULT = 0
MONT_RANGE_UNSIGNED = 1
MONT_RANGE_WIDE = 2
MONT_RANGE_CENTRED = 3
MONT_RANGE_EXPLICIT = 4
MONT_SWEEP_INCLUDE_OUT_OF_SPEC = 1
MONT_SWEEP_MAX_LOG2R = 16
MONT_SWEEP_MAX_N = 32767


class MontBounds(ctypes.Structure):
    _fields_ = [("domain_rule", ctypes.c_int), ("range_rule", ctypes.c_int),
                ("t_lo", ctypes.c_int64), ("t_hi", ctypes.c_int64),
                ("r_lo", ctypes.c_int64), ("r_hi", ctypes.c_int64)]


class MontCex(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("T", ctypes.c_int64),
                ("r", ctypes.c_int64), ("expected", ctypes.c_int64)]


MONT_TUNE_MODE_MUL = 0
MONT_TUNE_MODE_TO_DOMAIN = 1
MONT_TUNE_MODE_FROM_DOMAIN = 2
MONT_TUNE_MODE_REDC = 3
MONT_TUNE_MODE_BATCHED = -1
MONT_TUNE_ELEMENTWISE = 1
MONT_TUNE_BATCHED = 2


class MontLaunchShape(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("unroll", ctypes.c_int), ("vec_bytes", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int), ("tile_iters", ctypes.c_int),
                ("team", ctypes.c_int)]


MONT_JOB_MODMUL = 0
MONT_JOB_SWEEP = 1

MONT_PIPE_SLOTS = 3
MONT_PIPE_MAX_OPS = 256
MONT_PIPE_MIN_CHUNK = 256
MONT_OP_MUL = 0
MONT_OP_REDC = 1
MONT_OP_TO_DOMAIN = 2
MONT_OP_FROM_DOMAIN = 3


class MontHostOp(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("op", ctypes.c_int), ("a", ctypes.c_void_p),
                ("b", ctypes.c_void_p), ("out", ctypes.c_void_p), ("n", ctypes.c_size_t)]


class MontJob(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("ctx", ctypes.c_void_p), ("a", ctypes.c_void_p),
                ("b", ctypes.c_void_p), ("out", ctypes.c_void_p), ("n", ctypes.c_size_t),
                ("variant", ctypes.c_int), ("log2R", ctypes.c_int), ("alpha", ctypes.c_int),
                ("N_lo", ctypes.c_uint32), ("N_hi", ctypes.c_uint32),
                ("claimed", ctypes.POINTER(MontBounds)), ("flags", ctypes.c_int),
                ("per_N_counts", ctypes.POINTER(ctypes.c_uint64)),
                ("per_N_checked", ctypes.POINTER(ctypes.c_uint64)),
                ("cex", ctypes.POINTER(MontCex)), ("cex_cap", ctypes.c_size_t),
                ("n_cex_total", ctypes.POINTER(ctypes.c_size_t)), ("timeout_ms", ctypes.c_int)]


class MontJobResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double)]


class MontError(RuntimeError):
    """A non-zero status from the C ABI."""

    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {mont_strerror(status)} (status {status})"
        if status == MONT_ECUDA:
            msg += f", cudaError {mont_last_cuda_error()}"
        super().__init__(msg)


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded shared library (loads it on first use; raises if absent)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"montgb library not built ({LIB_PATH} missing): run "
                "paper_2402_00675_gb300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        _declare(L)
        _lib = L
    return _lib


_c = ctypes
_vp = _c.c_void_p
_sz = _c.c_size_t
_int = _c.c_int
_u32p = _c.POINTER(_c.c_uint32)


def _declare(L):
    sig = {
        "mont_ctx_create": (_int, [_c.POINTER(_vp), _u32p, _int, _int, _int, _int]),
        "mont_ctx_destroy": (_int, [_vp]),
        "mont_ctx_constant": (_int, [_vp, _int, _u32p, _int, _c.POINTER(_int)]),
        "mont_ctx_query": (_int, [_vp] + [_c.POINTER(_int)] * 6),
        "mont_mul": (_int, [_vp, _vp, _vp, _vp, _sz, _vp]),
        "mont_redc": (_int, [_vp, _vp, _vp, _sz, _vp]),
        "mont_to_domain": (_int, [_vp, _vp, _vp, _sz, _vp]),
        "mont_from_domain": (_int, [_vp, _vp, _vp, _sz, _vp]),
        "mont_verify_sweep": (_int, [_int, _int, _int, _c.c_uint32, _c.c_uint32,
                                     _c.POINTER(MontBounds), _int,
                                     _c.POINTER(_c.c_uint64), _c.POINTER(_c.c_uint64),
                                     _c.POINTER(MontCex), _sz, _c.POINTER(_sz), _vp]),
        "mont_mul_batched": (_int, [_c.POINTER(_vp), _c.POINTER(_vp), _c.POINTER(_vp),
                                    _c.POINTER(_vp), _c.POINTER(_sz), _int, _vp]),
        "mont_batch_create": (_int, [_c.POINTER(_vp), _c.POINTER(_vp), _c.POINTER(_vp),
                                     _c.POINTER(_vp), _c.POINTER(_vp), _c.POINTER(_sz), _int]),
        "mont_batch_launch": (_int, [_vp, _vp]),
        "mont_batch_update": (_int, [_vp, _c.POINTER(_vp), _c.POINTER(_vp), _c.POINTER(_vp)]),
        "mont_batch_destroy": (_int, [_vp]),
        "mont_tune_set": (_int, [_int, _int, _int, _c.POINTER(MontLaunchShape)]),
        "mont_tune_get": (_int, [_int, _int, _int, _c.POINTER(MontLaunchShape)]),
        "mont_autotune": (_int, [_vp, _sz, _int, _vp]),
        "mont_tune_save": (_int, [_c.c_char_p]),
        "mont_tune_load": (_int, [_c.c_char_p]),
        "mont_verify_sweep_noalloc": (_int, [_int, _int, _int, _c.c_uint32, _c.c_uint32,
                                             _c.POINTER(MontBounds), _int,
                                             _c.POINTER(_c.c_uint64), _c.POINTER(_c.c_uint64),
                                             _c.POINTER(MontCex), _sz, _c.POINTER(_sz), _vp]),
        "mont_server_create": (_int, [_c.POINTER(_vp), _sz, _int, _int]),
        "mont_server_submit": (_int, [_vp, _c.POINTER(MontJob), _c.POINTER(_c.c_uint64)]),
        "mont_server_wait": (_int, [_vp, _c.c_uint64, _int, _c.POINTER(MontJobResult)]),
        "mont_server_job_busy": (_int, [_vp, _c.c_uint64, _c.POINTER(_int)]),
        "mont_server_query": (_int, [_vp, _c.POINTER(_sz), _c.POINTER(_sz), _c.POINTER(_sz),
                                     _c.POINTER(_c.c_double)]),
        "mont_server_destroy": (_int, [_vp]),
        "mont_probe_int_rate": (_int, [_int, _int, _vp, _c.POINTER(_c.c_double)]),
        "mont_const_prepare": (_int, [_vp, _vp, _vp, _sz, _vp]),
        "mont_mul_pre": (_int, [_vp, _vp, _vp, _vp, _sz, _vp]),
        "mont_ntt_create": (_int, [_c.POINTER(_vp), _vp, _int, _u32p]),
        "mont_ntt_forward": (_int, [_vp, _vp, _vp, _sz, _vp]),
        "mont_ntt_inverse": (_int, [_vp, _vp, _vp, _sz, _vp]),
        "mont_ntt_destroy": (_int, [_vp]),
        "mont_dot_lazy": (_int, [_vp, _vp, _vp, _vp, _sz, _c.c_uint32, _vp]),
        "mont_rns_create": (_int, [_c.POINTER(_vp), _c.POINTER(_c.c_uint64), _int]),
        "mont_rns_query": (_int, [_vp, _c.POINTER(_int), _c.POINTER(_int)]),
        "mont_rns_to_residues": (_int, [_vp, _vp, _vp, _sz, _vp]),
        "mont_rns_from_residues": (_int, [_vp, _vp, _vp, _sz, _vp]),
        "mont_rns_destroy": (_int, [_vp]),
        "mont_pipe_create": (_int, [_c.POINTER(_vp), _sz]),
        "mont_pipe_run": (_int, [_vp, _c.POINTER(MontHostOp), _int, _vp]),
        "mont_pipe_plan": (_int, [_vp, _c.POINTER(MontHostOp), _int, _c.POINTER(_sz),
                                  _c.POINTER(_int)]),
        "mont_pipe_destroy": (_int, [_vp]),
        "mont_strerror": (_c.c_char_p, [_int]),
        "mont_last_cuda_error": (_int, []),
        "mont_sync": (_int, [_vp]),
        "mont_version": (_int, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _check(status: int, where: str) -> None:
    if status != MONT_OK:
        raise MontError(status, where)


def _ptr(x):
    """Device address of a tensor (must be CUDA and contiguous) or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor (device pointer argument)")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return x.data_ptr()
    raise TypeError(f"cannot take a device pointer of {type(x).__name__}")


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _nbytes(x):
    return x.numel() * x.element_size() if hasattr(x, "numel") else None


def _limbs(x: int, k: int):
    if x < 0 or x >> (32 * k):
        raise ValueError("value does not fit in the limbs")
    return (ctypes.c_uint32 * k)(*[(x >> (32 * i)) & 0xFFFFFFFF for i in range(k)])


class Ctx:
    """An owned ``mont_ctx_t`` handle with the parameters it was made from."""

    def __init__(self, handle, N, log2R, variant, alpha, n_limbs):
        self.handle = handle
        self.N = N
        self.log2R = log2R
        self.variant = variant
        self.alpha = alpha
        self.n_limbs = n_limbs
        self.width = 32 * n_limbs
        self.elem_bytes = 4 * n_limbs

    def close(self):
        if self.handle:
            lib().mont_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        if not self.handle:
            raise ValueError("ctx already destroyed")
        return self.handle


def mont_ctx_create(N: int, log2R: int, variant: int, alpha: int = 0,
                    n_limbs: int | None = None) -> Ctx:
    """Precompute the constants of modulus N (see ``mont_ctx_create`` in montgb.h).

    ``n_limbs`` defaults to 1 for log2R of 32 (REDC family) or 64 (Plantard
    family), 2 for 64/128, and log2R/32 for multi-limb REDC."""
    if n_limbs is None:
        n_limbs = log2R // 64 if variant in PLANTARD_VARIANTS else log2R // 32
        n_limbs = max(n_limbs, 1)
    h = ctypes.c_void_p()
    _check(lib().mont_ctx_create(ctypes.byref(h), _limbs(N, n_limbs), n_limbs, log2R,
                                 variant, alpha), "mont_ctx_create")
    return Ctx(h.value, N, log2R, variant, alpha, n_limbs)


def mont_ctx_destroy(ctx: Ctx) -> None:
    ctx.close()


def mont_ctx_constant(ctx: Ctx, which: int) -> int:
    buf = (ctypes.c_uint32 * (2 * MONT_MAX_LIMBS + 8))()
    n = ctypes.c_int()
    _check(lib().mont_ctx_constant(ctx, which, buf, len(buf), ctypes.byref(n)),
           "mont_ctx_constant")
    return sum(int(buf[i]) << (32 * i) for i in range(n.value))


def mont_ctx_query(ctx: Ctx) -> dict:
    vals = [ctypes.c_int() for _ in range(6)]
    _check(lib().mont_ctx_query(ctx, *[ctypes.byref(v) for v in vals]), "mont_ctx_query")
    keys = ("width_bits", "n_limbs", "elem_bytes", "variant", "log2R", "alpha")
    return {k: v.value for k, v in zip(keys, vals)}


def _count(ctx: Ctx, out, n, scale=1):
    if n is not None:
        return int(n)
    nb = _nbytes(out)
    if nb is None:
        raise ValueError("n is required when out is a raw pointer")
    return nb // (ctx.elem_bytes * scale)


def mont_mul(ctx: Ctx, a, b, out, n: int | None = None, stream=None) -> None:
    """out[i] = a[i] b[i] R^{-1} (or -a b R^{-1} for the Plantard family), on the device."""
    _check(lib().mont_mul(ctx, _ptr(a), _ptr(b), _ptr(out), _count(ctx, out, n),
                          _stream(stream)), "mont_mul")


def mont_redc(ctx: Ctx, T, out, n: int | None = None, stream=None) -> None:
    """out[i] = reduce(T[i]) for double-width T, on the device."""
    _check(lib().mont_redc(ctx, _ptr(T), _ptr(out), _count(ctx, out, n), _stream(stream)),
           "mont_redc")


def mont_to_domain(ctx: Ctx, x, out, n: int | None = None, stream=None) -> None:
    _check(lib().mont_to_domain(ctx, _ptr(x), _ptr(out), _count(ctx, out, n), _stream(stream)),
           "mont_to_domain")


def mont_from_domain(ctx: Ctx, y, out, n: int | None = None, stream=None) -> None:
    _check(lib().mont_from_domain(ctx, _ptr(y), _ptr(out), _count(ctx, out, n),
                                  _stream(stream)), "mont_from_domain")


def _batch_arrays(ctxs, a, b, out, lens):
    count = len(ctxs)
    if not (len(a) == len(b) == len(out) == count):
        raise ValueError("ctxs, a, b, out must have the same length")
    if lens is None:
        lens = [_count(c, o, None) for c, o in zip(ctxs, out)]
    P = ctypes.c_void_p * max(count, 1)
    return (count, P(*[c.handle for c in ctxs]), P(*[_ptr(x) for x in a]),
            P(*[_ptr(x) for x in b]), P(*[_ptr(x) for x in out]),
            (ctypes.c_size_t * max(count, 1))(*[int(n) for n in lens]))


def mont_mul_batched(ctxs, a, b, out, lens=None, stream=None) -> None:
    """One persistent launch over many (modulus, vector) pairs; see montgb.h."""
    count, C, A, B, O, Ls = _batch_arrays(ctxs, a, b, out, lens)
    _check(lib().mont_mul_batched(C, A, B, O, Ls, count, _stream(stream)), "mont_mul_batched")


class Batch:
    """A mont_batch_t plan: the batch's launches recorded in a CUDA graph."""

    def __init__(self, ctxs, a, b, out, lens=None):
        count, C, A, B, O, Ls = _batch_arrays(ctxs, a, b, out, lens)
        h = ctypes.c_void_p()
        _check(lib().mont_batch_create(ctypes.byref(h), C, A, B, O, Ls, count),
               "mont_batch_create")
        self.handle = h.value
        self.count = count

    def launch(self, stream=None) -> None:
        _check(lib().mont_batch_launch(self.handle, _stream(stream)), "mont_batch_launch")

    def update(self, a, b, out) -> None:
        P = ctypes.c_void_p * max(self.count, 1)
        _check(lib().mont_batch_update(self.handle, P(*[_ptr(x) for x in a]),
                                       P(*[_ptr(x) for x in b]), P(*[_ptr(x) for x in out])),
               "mont_batch_update")

    def close(self):
        if self.handle:
            lib().mont_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mont_batch_create(ctxs, a, b, out, lens=None) -> Batch:
    return Batch(ctxs, a, b, out, lens)


def mont_batch_launch(batch: Batch, stream=None) -> None:
    batch.launch(stream)


def mont_batch_update(batch: Batch, a, b, out) -> None:
    batch.update(a, b, out)


def mont_batch_destroy(batch: Batch) -> None:
    batch.close()


class SweepResult:
    """Host-side result of mont_verify_sweep."""

    def __init__(self, moduli, counts, checked, examples, total, overflow):
        self.moduli = moduli            # the odd N of the range, in order
        self.counts = counts            # N -> counterexamples (0 for skipped N)
        self.checked = checked          # N -> T checked (0 for skipped N)
        self.examples = examples        # sorted (N, T, r, expected)
        self.total = total
        self.overflow = overflow        # more counterexamples than cex_cap


def mont_verify_sweep(variant: int, log2R: int, alpha: int, N_lo: int, N_hi: int,
                      claimed: MontBounds | None = None, flags: int = 0,
                      cex_cap: int = 1 << 16, stream=None) -> SweepResult:
    """Run the exhaustive sweep on the device (synchronous); see montgb.h."""
    first = N_lo if N_lo % 2 else N_lo + 1
    moduli = list(range(first, N_hi + 1, 2))
    n = max(len(moduli), 1)
    counts = (ctypes.c_uint64 * n)()
    checked = (ctypes.c_uint64 * n)()
    cex = (MontCex * max(cex_cap, 1))()
    total = ctypes.c_size_t()
    st = lib().mont_verify_sweep(variant, log2R, alpha, N_lo, N_hi,
                                 ctypes.byref(claimed) if claimed is not None else None, flags,
                                 counts, checked, cex, cex_cap, ctypes.byref(total),
                                 _stream(stream))
    if st not in (MONT_OK, MONT_EOVERFLOW):
        raise MontError(st, "mont_verify_sweep")
    nrec = min(total.value, cex_cap)
    ex = [(int(c.N), int(c.T), int(c.r), int(c.expected)) for c in cex[:nrec]]
    return SweepResult(moduli, {N: int(counts[i]) for i, N in enumerate(moduli)},
                       {N: int(checked[i]) for i, N in enumerate(moduli)}, ex, total.value,
                       st == MONT_EOVERFLOW)


def mont_tune_set(width_bits: int, variant: int, mode: int, shape: dict | None) -> None:
    """Set (or clear, with shape=None) one launch-shape table entry."""
    ptr = None
    if shape is not None:
        ptr = ctypes.byref(MontLaunchShape(**{k: int(v) for k, v in shape.items()}))
    _check(lib().mont_tune_set(width_bits, variant, mode, ptr), "mont_tune_set")


def mont_tune_get(width_bits: int, variant: int, mode: int) -> dict:
    sh = MontLaunchShape()
    _check(lib().mont_tune_get(width_bits, variant, mode, ctypes.byref(sh)), "mont_tune_get")
    return {k: getattr(sh, k) for k, _ in MontLaunchShape._fields_}


def mont_autotune(ctx: Ctx, n: int, flags: int = MONT_TUNE_ELEMENTWISE, stream=None) -> None:
    _check(lib().mont_autotune(ctx, n, flags, _stream(stream)), "mont_autotune")


def mont_tune_save(path: str) -> None:
    _check(lib().mont_tune_save(path.encode()), "mont_tune_save")


def mont_tune_load(path: str) -> None:
    _check(lib().mont_tune_load(path.encode()), "mont_tune_load")


MONT_SWEEP_NOALLOC_MAX_MODULI = 8192
MONT_SWEEP_NOALLOC_MAX_CEX = 4096


def mont_verify_sweep_noalloc(variant: int, log2R: int, alpha: int, N_lo: int, N_hi: int,
                              claimed: MontBounds | None = None, flags: int = 0,
                              cex_cap: int = MONT_SWEEP_NOALLOC_MAX_CEX,
                              stream=None) -> SweepResult:
    """The sweep through the entry point that allocates nothing (fixed
    device scratch; bounded sizes); see montgb.h.  The result buffers are
    created here, in Python, before the call."""
    first = N_lo if N_lo % 2 else N_lo + 1
    moduli = list(range(first, N_hi + 1, 2))
    n = max(len(moduli), 1)
    counts = (ctypes.c_uint64 * n)()
    checked = (ctypes.c_uint64 * n)()
    cex = (MontCex * max(cex_cap, 1))()
    total = ctypes.c_size_t()
    st = lib().mont_verify_sweep_noalloc(variant, log2R, alpha, N_lo, N_hi,
                                         ctypes.byref(claimed) if claimed is not None else None,
                                         flags, counts, checked, cex, cex_cap,
                                         ctypes.byref(total), _stream(stream))
    if st not in (MONT_OK, MONT_EOVERFLOW):
        raise MontError(st, "mont_verify_sweep_noalloc")
    nrec = min(total.value, cex_cap)
    ex = [(int(c.N), int(c.T), int(c.r), int(c.expected)) for c in cex[:nrec]]
    return SweepResult(moduli, {N: int(counts[i]) for i, N in enumerate(moduli)},
                       {N: int(checked[i]) for i, N in enumerate(moduli)}, ex, total.value,
                       st == MONT_EOVERFLOW)


def _host_ptr(x):
    """Address of host memory: a CPU torch tensor or a numpy array (contiguous)."""
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if x.is_cuda or not x.is_contiguous():
            raise ValueError("expected a contiguous CPU tensor (host pointer argument)")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a contiguous array")
        return x.ctypes.data
    raise TypeError(f"cannot take a host pointer of {type(x).__name__}")


class Server:
    """A mont_server_t: continuous batching of modmul and sweep jobs.

    The host buffers of a job are kept referenced until the job is retrieved
    by wait(), and, for a job that timed out, until the server reports that
    its device work no longer uses them (job_busy)."""

    def __init__(self, mem_budget_bytes: int, slots: int = 4, job_timeout_ms: int = 60000):
        h = ctypes.c_void_p()
        _check(lib().mont_server_create(ctypes.byref(h), mem_budget_bytes, slots,
                                        job_timeout_ms), "mont_server_create")
        self.handle = h.value
        self._keep = {}
        self._busy = {}   # timed-out jobs whose buffers the device may still use

    def submit_modmul(self, ctx: Ctx, a, b, out, n: int | None = None,
                      timeout_ms: int = 0) -> int:
        """Queue out = a b R^{-1} (host buffers) and return the job id."""
        if n is None:
            n = _nbytes(out) // ctx.elem_bytes if hasattr(out, "numel") else out.nbytes // ctx.elem_bytes
        job = MontJob(kind=MONT_JOB_MODMUL, ctx=ctx.handle, a=_host_ptr(a), b=_host_ptr(b),
                      out=_host_ptr(out), n=n, timeout_ms=timeout_ms)
        jid = ctypes.c_uint64()
        _check(lib().mont_server_submit(self.handle, ctypes.byref(job), ctypes.byref(jid)),
               "mont_server_submit")
        self._keep[jid.value] = (ctx, a, b, out)
        return jid.value

    def submit_sweep(self, variant, log2R, alpha, N_lo, N_hi, claimed=None, flags=0,
                     cex_cap=1024, timeout_ms: int = 0) -> int:
        first = N_lo if N_lo % 2 else N_lo + 1
        moduli = list(range(first, N_hi + 1, 2))
        n = max(len(moduli), 1)
        counts = (ctypes.c_uint64 * n)()
        checked = (ctypes.c_uint64 * n)()
        cex = (MontCex * max(cex_cap, 1))()
        total = ctypes.c_size_t()
        job = MontJob(kind=MONT_JOB_SWEEP, variant=variant, log2R=log2R, alpha=alpha, N_lo=N_lo,
                      N_hi=N_hi, claimed=ctypes.pointer(claimed) if claimed is not None else None,
                      flags=flags, per_N_counts=counts, per_N_checked=checked, cex=cex,
                      cex_cap=cex_cap, n_cex_total=ctypes.pointer(total), timeout_ms=timeout_ms)
        jid = ctypes.c_uint64()
        _check(lib().mont_server_submit(self.handle, ctypes.byref(job), ctypes.byref(jid)),
               "mont_server_submit")
        self._keep[jid.value] = (moduli, counts, checked, cex, total, cex_cap)
        return jid.value

    def wait(self, jid: int, timeout_ms: int = -1) -> dict:
        """Wait for a job; returns its status and times (plus sweep results)."""
        res = MontJobResult()
        _check(lib().mont_server_wait(self.handle, jid, timeout_ms, ctypes.byref(res)),
               "mont_server_wait")
        out = {"status": res.status, "t_submit": res.t_submit, "t_admit": res.t_admit,
               "t_done": res.t_done}
        keep = self._keep.pop(jid, None)
        if res.status == MONT_ETIMEOUT and keep is not None:
            self._busy[jid] = keep
        elif keep is not None and len(keep) == 6 and res.status == MONT_OK:
            moduli, counts, checked, cex, total, cap = keep
            nrec = min(total.value, cap)
            out["sweep"] = SweepResult(
                moduli, {N: int(counts[i]) for i, N in enumerate(moduli)},
                {N: int(checked[i]) for i, N in enumerate(moduli)},
                [(int(c.N), int(c.T), int(c.r), int(c.expected)) for c in cex[:nrec]],
                total.value, total.value > cap)
        return out

    def job_busy(self, jid: int) -> bool:
        """True while a timed-out job's device work may still use its buffers."""
        b = ctypes.c_int()
        _check(lib().mont_server_job_busy(self.handle, jid, ctypes.byref(b)),
               "mont_server_job_busy")
        if not b.value:
            self._busy.pop(jid, None)
        return bool(b.value)

    def query(self) -> dict:
        q, r, f, t = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_double()
        _check(lib().mont_server_query(self.handle, ctypes.byref(q), ctypes.byref(r),
                                       ctypes.byref(f), ctypes.byref(t)), "mont_server_query")
        return {"queued": q.value, "running": r.value, "arena_free": f.value, "now": t.value}

    def close(self) -> int:
        """Destroy the server; returns its status (MONT_ETIMEOUT: the device work
        of timed-out jobs did not end, and their buffers stay referenced)."""
        st = MONT_OK
        if self.handle:
            st = lib().mont_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()
            if st == MONT_OK:
                self._busy.clear()
        return st

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mont_server_create(mem_budget_bytes: int, slots: int = 4, job_timeout_ms: int = 60000):
    return Server(mem_budget_bytes, slots, job_timeout_ms)


def mont_server_destroy(server: Server) -> None:
    server.close()


class Pipe:
    """A mont_pipe_t: element-wise operations on vectors in host memory.

    ``ops`` is a sequence of ``(ctx, op, a, b, out)`` or ``(ctx, op, a, b, out, n)``
    tuples: ``op`` a ``MONT_OP_*`` code, ``a``/``b``/``out`` CPU tensors, numpy
    arrays or host addresses (``b`` None unless ``op`` is ``MONT_OP_MUL``), ``n``
    defaulting to the elements ``out`` holds.  The buffers must stay alive and
    the inputs unchanged until the stream passes the run.
    """

    def __init__(self, staging_bytes: int = 256 << 20):
        h = ctypes.c_void_p()
        _check(lib().mont_pipe_create(ctypes.byref(h), staging_bytes), "mont_pipe_create")
        self.handle = h.value

    @staticmethod
    def _ops(ops):
        arr = (MontHostOp * max(len(ops), 1))()
        for i, o in enumerate(ops):
            ctx, code, a, b, out = o[:5]
            if len(o) > 5:
                n = o[5]
            elif out is None:
                n = 0
            else:
                nb = _nbytes(out) if hasattr(out, "numel") else out.nbytes
                n = nb // ctx.elem_bytes
            hp = [None if x is None else _host_ptr(x) for x in (a, b, out)]
            arr[i] = MontHostOp(ctx=ctx.handle, op=code, a=hp[0], b=hp[1], out=hp[2], n=n)
        return arr

    def run(self, ops, stream=None) -> None:
        _check(lib().mont_pipe_run(self.handle, self._ops(ops), len(ops), _stream(stream)),
               "mont_pipe_run")

    def plan(self, ops) -> tuple[int, int]:
        """(chunk in elements, distinct inputs) a run of ``ops`` would use."""
        chunk, distinct = ctypes.c_size_t(), ctypes.c_int()
        _check(lib().mont_pipe_plan(self.handle, self._ops(ops), len(ops), ctypes.byref(chunk),
                                    ctypes.byref(distinct)), "mont_pipe_plan")
        return chunk.value, distinct.value

    def close(self):
        if self.handle:
            lib().mont_pipe_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mont_pipe_create(staging_bytes: int = 256 << 20) -> Pipe:
    return Pipe(staging_bytes)


def mont_pipe_run(pipe: Pipe, ops, stream=None) -> None:
    pipe.run(ops, stream)


def mont_pipe_plan(pipe: Pipe, ops) -> tuple[int, int]:
    return pipe.plan(ops)


def mont_pipe_destroy(pipe: Pipe) -> None:
    pipe.close()


def mont_probe_int_rate(kind: int, iters: int = 4096, stream=None) -> float:
    """Measured thread-instructions per second for an integer mix (see montgb.h)."""
    r = ctypes.c_double()
    _check(lib().mont_probe_int_rate(kind, iters, _stream(stream), ctypes.byref(r)),
           "mont_probe_int_rate")
    return r.value


def mont_const_prepare(ctx: Ctx, b, b_pre, n: int | None = None, stream=None) -> None:
    """b_pre[i] = b[i] N^{-1} mod R (Plantard family; see montgb.h)."""
    _check(lib().mont_const_prepare(ctx, _ptr(b), _ptr(b_pre), _count(ctx, b, n),
                                    _stream(stream)), "mont_const_prepare")


def mont_mul_pre(ctx: Ctx, a, b_pre, out, n: int | None = None, stream=None) -> None:
    """out[i] = reduce(a[i] b[i]) from the prepared multipliers b_pre."""
    _check(lib().mont_mul_pre(ctx, _ptr(a), _ptr(b_pre), _ptr(out), _count(ctx, out, n),
                              _stream(stream)), "mont_mul_pre")


class Ntt:
    """A mont_ntt_t plan: batched negacyclic NTTs of length 2^log2n."""

    def __init__(self, ctx: Ctx, log2n: int, psi: int):
        h = ctypes.c_void_p()
        _check(lib().mont_ntt_create(ctypes.byref(h), ctx, log2n, _limbs(psi, ctx.n_limbs)),
               "mont_ntt_create")
        self.handle = h.value
        self.n = 1 << log2n
        self.elem_bytes = ctx.elem_bytes

    def _batch(self, x, batch):
        if batch is not None:
            return int(batch)
        return _nbytes(x) // (self.elem_bytes * self.n)

    def forward(self, x, out, batch: int | None = None, stream=None) -> None:
        _check(lib().mont_ntt_forward(self.handle, _ptr(x), _ptr(out), self._batch(x, batch),
                                      _stream(stream)), "mont_ntt_forward")

    def inverse(self, x, out, batch: int | None = None, stream=None) -> None:
        _check(lib().mont_ntt_inverse(self.handle, _ptr(x), _ptr(out), self._batch(x, batch),
                                      _stream(stream)), "mont_ntt_inverse")

    def close(self):
        if self.handle:
            lib().mont_ntt_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mont_ntt_create(ctx: Ctx, log2n: int, psi: int) -> Ntt:
    return Ntt(ctx, log2n, psi)


def mont_dot_lazy(ctx: Ctx, a, b, out, k: int, rows: int | None = None, stream=None) -> None:
    """out[j] = Algorithm 4 applied once to a row dot product (see montgb.h)."""
    if rows is None:
        rows = _count(ctx, out, None)
    _check(lib().mont_dot_lazy(ctx, _ptr(a), _ptr(b), _ptr(out), rows, k, _stream(stream)),
           "mont_dot_lazy")


class Rns:
    """A mont_rns_t: conversions between big integers and residues."""

    def __init__(self, moduli):
        arr = (ctypes.c_uint64 * len(moduli))(*[int(p) for p in moduli])
        h = ctypes.c_void_p()
        _check(lib().mont_rns_create(ctypes.byref(h), arr, len(moduli)), "mont_rns_create")
        self.handle = h.value
        c, k = ctypes.c_int(), ctypes.c_int()
        _check(lib().mont_rns_query(self.handle, ctypes.byref(c), ctypes.byref(k)), "mont_rns_query")
        self.count, self.limbs = c.value, k.value

    def to_residues(self, X, residues, n: int, stream=None) -> None:
        _check(lib().mont_rns_to_residues(self.handle, _ptr(X), _ptr(residues), n, _stream(stream)),
               "mont_rns_to_residues")

    def from_residues(self, residues, X, n: int, stream=None) -> None:
        _check(lib().mont_rns_from_residues(self.handle, _ptr(residues), _ptr(X), n,
                                            _stream(stream)), "mont_rns_from_residues")

    def close(self):
        if self.handle:
            lib().mont_rns_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mont_rns_create(moduli) -> Rns:
    return Rns(moduli)


def mont_sync(stream=None) -> None:
    _check(lib().mont_sync(_stream(stream)), "mont_sync")


def mont_strerror(status: int) -> str:
    return lib().mont_strerror(status).decode()


def mont_last_cuda_error() -> int:
    return lib().mont_last_cuda_error()


def mont_version() -> int:
    return lib().mont_version()
