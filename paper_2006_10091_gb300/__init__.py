"""Python binding of libhegb300.so, the sm_103a library for the encrypted
logistic-regression worker step of Li & Huang (KDD'20).

Argument marshalling only: every residue operation runs in the library's
CUDA kernels.  The functions keep the C ABI's names (include/he_gb300.h).
PyTorch provides device memory (ciphertext buffers are int64 CUDA tensors
holding uint64 residues) and the stream.  Importing the package does not
touch the GPU; the first call that needs the library loads it and raises
if it is missing -- there is no other implementation to fall back to.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhegb300.so")

HE_OK, HE_EINVAL, HE_ELEVEL, HE_ESCALE, HE_ENOKEY, HE_ENOMEM, HE_ECUDA, HE_ETIMEOUT = range(8)


class HeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class he_params(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_uint32), ("n_limbs", ctypes.c_uint32),
                ("limb_bits", ctypes.c_uint32), ("n_special", ctypes.c_uint32),
                ("special_bits", ctypes.c_uint32), ("dnum", ctypes.c_uint32),
                ("scale", ctypes.c_double), ("sigma", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class he_ct(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("level", ctypes.c_uint32),
                ("cap", ctypes.c_uint32), ("scale", ctypes.c_double)]


class he_lr_shard(ctypes.Structure):
    _fields_ = [("Z", ctypes.c_void_p), ("nZ", ctypes.c_size_t), ("W", ctypes.c_void_p),
                ("W_out", ctypes.c_void_p), ("S_out", ctypes.c_void_p), ("refresh_cid", ctypes.c_uint32),
                ("min_level", ctypes.c_uint32)]


HE_LR_GRAPH = 1
HE_REQ_GRADIENT, HE_REQ_INFERENCE = 0, 1


class he_lr_config(ctypes.Structure):
    _fields_ = [("coeffs", ctypes.c_double * 4), ("lr", ctypes.c_double),
                ("g", ctypes.c_uint32), ("pad", ctypes.c_uint32), ("mask_scale", ctypes.c_double),
                ("l2", ctypes.c_double)]


class he_server_config(ctypes.Structure):
    _fields_ = [("ctxs", ctypes.c_void_p), ("n_ctx", ctypes.c_size_t), ("hbm_budget", ctypes.c_size_t),
                ("max_inflight", ctypes.c_uint32), ("max_wave", ctypes.c_uint32),
                ("max_running", ctypes.c_uint32)]


class he_request(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_uint32), ("kind", ctypes.c_uint32), ("nZ", ctypes.c_uint32),
                ("z_level", ctypes.c_uint32), ("w_level", ctypes.c_uint32), ("refresh_cid", ctypes.c_uint32),
                ("min_w_level", ctypes.c_uint32),
                ("z_scale", ctypes.c_double), ("w_scale", ctypes.c_double), ("Z", ctypes.c_void_p),
                ("W", ctypes.c_void_p), ("cfg", he_lr_config), ("out", ctypes.c_void_p),
                ("out_words", ctypes.c_size_t)]


class he_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("level", ctypes.c_uint32),
                ("scale", ctypes.c_double), ("latency_ms", ctypes.c_double)]


_lib = None
VP = ctypes.c_void_p
CTP = ctypes.POINTER(he_ct)


def load():
    """Load libhegb300.so (build it first with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2006_10091_gb300.build.build() "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    lib.he_last_error.restype = ctypes.c_char_p
    sig = {
        "he_ctx_create": [ctypes.POINTER(he_params), VP, ctypes.c_size_t, VP, ctypes.POINTER(VP)],
        "he_ctx_destroy": [VP],
        "he_set_stream": [VP, VP],
        "he_sync": [VP],
        "he_ctx_info": [VP, VP, VP, VP, VP, VP],
        "he_encode": [VP, VP, ctypes.c_size_t, ctypes.c_double, VP],
        "he_encrypt_poly": [VP, VP, ctypes.c_double, ctypes.c_uint32, ctypes.c_int, ctypes.c_uint32, CTP],
        "he_encode_encrypt": [VP, VP, ctypes.c_size_t, ctypes.c_double, ctypes.c_uint32, ctypes.c_int,
                              ctypes.c_uint32, CTP],
        "he_decrypt_poly": [VP, CTP, VP],
        "he_decrypt_decode": [VP, CTP, VP, ctypes.c_size_t],
        "he_ct_export": [VP, CTP, VP, ctypes.c_size_t],
        "he_ct_import": [VP, VP, ctypes.c_uint32, ctypes.c_double, CTP],
        "he_add": [VP, CTP, CTP, CTP],
        "he_sub": [VP, CTP, CTP, CTP],
        "he_drop_level": [VP, CTP, ctypes.c_uint32, CTP],
        "he_mul_const": [VP, CTP, ctypes.c_double, ctypes.c_double, CTP],
        "he_add_const": [VP, CTP, ctypes.c_double, CTP],
        "he_mul_plain": [VP, CTP, VP, ctypes.c_double, CTP],
        "he_rescale": [VP, CTP, CTP],
        "he_mul_relin_rescale": [VP, CTP, CTP, CTP],
        "he_mul_relin": [VP, CTP, CTP, CTP],
        "he_rotate": [VP, CTP, ctypes.c_int32, CTP],
        "he_mul_relin_rescale_batch": [VP, CTP, CTP, CTP, ctypes.c_size_t],
        "he_rotate_batch": [VP, CTP, ctypes.c_int32, CTP, ctypes.c_size_t],
        "he_rotate_sum": [VP, CTP, VP, ctypes.c_uint32, CTP],
        "he_rotate_sum_batch": [VP, CTP, VP, ctypes.c_uint32, CTP, ctypes.c_size_t],
        "he_lr_gradient_step": [VP, CTP, ctypes.c_size_t, CTP, ctypes.POINTER(he_lr_config), CTP],
        "he_refresh": [VP, CTP, ctypes.c_uint32, ctypes.c_double, ctypes.c_uint32, CTP],
        "he_ntt": [VP, VP, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int],
        "he_keyswitch": [VP, VP, ctypes.c_uint32, ctypes.c_uint64, VP, VP],
        "he_moddown": [VP, VP, ctypes.c_uint32, CTP, CTP],
        "he_ct_import_batch": [VP, VP, ctypes.c_uint32, ctypes.c_double, CTP, ctypes.c_size_t],
        "he_ct_export_batch": [VP, CTP, ctypes.c_size_t, VP, ctypes.c_size_t],
        "he_profile_enable": [VP, ctypes.c_int],
        "he_profile_read": [VP, ctypes.c_char_p, VP, VP, VP, VP],
        "he_profile_names": [VP, ctypes.c_char_p, ctypes.c_size_t],
        "he_profile_read_kinds": [VP, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double)],
        "he_set_tuning": [VP, ctypes.c_char_p, ctypes.c_double],
        "he_lr_train": [VP, VP, ctypes.c_size_t, ctypes.POINTER(he_lr_config), ctypes.c_uint32, ctypes.c_uint32,
                        ctypes.c_uint32, ctypes.c_uint32, CTP],
        "he_lr_gradient_step_host": [VP, VP, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_double, VP, ctypes.c_uint32,
                                     ctypes.c_double, ctypes.POINTER(he_lr_config), VP, ctypes.c_size_t,
                                     ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_double)],
        "he_get_tuning": [VP, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double)],
        "he_probe_alu": [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
        "he_fit_poly": [VP, VP, ctypes.c_size_t, ctypes.c_uint32, VP],
        "he_autotune": [VP, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double)],
        "he_rescale_noalloc": [VP, CTP, CTP],
        "he_sum": [VP, VP, ctypes.c_size_t, CTP],
        "he_ct_alloc": [VP, ctypes.c_uint32, ctypes.POINTER(CTP)],
        "he_ct_free": [CTP],
        "he_ctx_workspace": [VP, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_uint64)],
        "he_lr_gradient_step_workers": [VP, VP, ctypes.c_size_t, ctypes.POINTER(he_lr_config),
                                        ctypes.c_uint32, ctypes.c_int],
        "he_lr_inference_workers": [VP, VP, ctypes.c_size_t, ctypes.POINTER(he_lr_config),
                                    ctypes.c_uint32, ctypes.c_int],
        "he_server_create": [ctypes.POINTER(he_server_config), ctypes.POINTER(VP)],
        "he_server_submit": [VP, ctypes.POINTER(he_request), ctypes.POINTER(ctypes.c_uint64)],
        "he_server_poll": [VP, VP, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)],
        "he_server_drain": [VP, ctypes.c_double],
        "he_server_stats": [VP, VP, VP, VP, VP],
        "he_server_last_error": [VP, ctypes.c_char_p, ctypes.c_size_t],
        "he_server_destroy": [VP],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc: int):
    if rc != HE_OK:
        raise HeError(rc, load().he_last_error().decode())


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _torch():
    import torch
    return torch


def current_stream_handle():
    torch = _torch()
    return torch.cuda.current_stream().cuda_stream


# ---------------------------------------------------------------------------
# Handles
# ---------------------------------------------------------------------------

class Context:
    """An he_ctx*: parameters, primes and keys resident on the device."""

    def __init__(self, log_n: int, n_limbs: int, limb_bits: int, n_special: int, special_bits: int,
                 scale: float, sigma: float = 3.2, seed: int = 0, rot_steps=(), dnum: int = 0,
                 stream=None):
        lib = load()
        p = he_params(log_n, n_limbs, limb_bits, n_special, special_bits, dnum, float(scale),
                      float(sigma), seed)
        rots = (ctypes.c_int32 * max(1, len(rot_steps)))(*rot_steps)
        self.stream = current_stream_handle() if stream is None else stream
        h = ctypes.c_void_p()
        _check(lib.he_ctx_create(ctypes.byref(p), rots, len(rot_steps), ctypes.c_void_p(self.stream),
                                 ctypes.byref(h)))
        self.ptr = h
        self.log_n, self.n, self.L, self.alpha = log_n, 1 << log_n, n_limbs, n_special
        self.scale = float(scale)
        n = ctypes.c_uint32()
        beta = ctypes.c_uint32()
        primes = np.zeros(n_limbs + n_special, dtype=np.uint64)
        _check(lib.he_ctx_info(h, ctypes.byref(n), None, None, ctypes.byref(beta), _ptr(primes)))
        self.beta = beta.value
        self.primes = [int(x) for x in primes]

    def close(self):
        if getattr(self, "ptr", None):
            load().he_ctx_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def new_ct(self, cap: int, count: int | None = None):
        """Ciphertext buffers of `cap` limbs: one, or `count` of them laid out
        back to back in a single allocation (a uniform batch)."""
        torch = _torch()
        shape = (count if count is not None else 1, 2, cap, self.n)
        buf = torch.empty(shape, dtype=torch.int64, device="cuda")
        cts = [Ciphertext(buf[i], cap) for i in range(shape[0])]
        return cts if count is not None else cts[0]


class Ciphertext:
    """A ciphertext buffer (int64 CUDA tensor [2][cap][N]) plus level and scale."""

    def __init__(self, tensor, cap: int, level: int = 0, scale: float = 0.0):
        self.tensor = tensor
        self.cap = cap
        self.level = level
        self.scale = scale

    def c(self) -> he_ct:
        return he_ct(self.tensor.data_ptr(), self.level, self.cap, self.scale)

    def update(self, s: he_ct):
        self.level, self.scale = s.level, s.scale

    def residues(self) -> np.ndarray:
        """[2][level][N] uint64 on the host (synchronises)."""
        return self.tensor[:, : self.level].cpu().numpy().view(np.uint64)


def _run(fn, ctx, outs, *args):
    """Call fn(ctx.ptr, *args) where args may contain Ciphertexts; outputs
    listed in outs get their level/scale back."""
    structs = {}
    cargs = []
    for a in args:
        if isinstance(a, Ciphertext):
            s = a.c()
            structs[id(a)] = (a, s)
            cargs.append(ctypes.byref(s))
        elif isinstance(a, Handle):  # the library's own he_ct: level and scale live in it
            cargs.append(a.ptr)
        else:
            cargs.append(a)
    _check(fn(ctx.ptr, *cargs))
    for o in outs:
        if id(o) in structs:
            a, s = structs[id(o)]
            a.update(s)


def _batch(cts):
    arr = (he_ct * len(cts))(*[c.c() for c in cts])
    return arr


def _same_len(name: str, first: list, *others: list) -> None:
    # the C entry points take one count for all their arrays
    if any(len(o) != len(first) for o in others):
        raise ValueError(f"{name}: the batches must have the same length")


# ---------------------------------------------------------------------------
# Entry points (names of the C ABI)
# ---------------------------------------------------------------------------

def he_set_stream(ctx: Context, stream):
    ctx.stream = stream
    _check(load().he_set_stream(ctx.ptr, ctypes.c_void_p(stream)))


def he_set_tuning(ctx: Context, key: str, value: float):
    _check(load().he_set_tuning(ctx.ptr, key.encode(), float(value)))


def he_get_tuning(ctx: Context, key: str) -> float:
    v = ctypes.c_double()
    _check(load().he_get_tuning(ctx.ptr, key.encode(), ctypes.byref(v)))
    return v.value


def he_probe_alu(kind: int) -> dict:
    """Register-resident integer throughput: kind 0 IMAD, 1 Shoup product, 2 lazy butterfly,
    3 64 x 64 -> 128-bit multiply-accumulate."""
    pc, ps = ctypes.c_double(), ctypes.c_double()
    _check(load().he_probe_alu(kind, ctypes.byref(pc), ctypes.byref(ps)))
    return {"per_clock_per_sm": pc.value, "per_second": ps.value}


def he_autotune(ctx: Context, level: int, count: int) -> dict:
    """Time the kernel knobs on a key switch of `count` polynomials at `level`
    and keep the fastest; returns the chosen knobs and the time (ms)."""
    ms = ctypes.c_double()
    _check(load().he_autotune(ctx.ptr, level, count, ctypes.byref(ms)))
    out = {k: he_get_tuning(ctx, k) for k in ("ntt_shape", "ntt_pb_max")}
    out["ms_per_keyswitch"] = ms.value
    return out


def he_sync(ctx: Context):
    _check(load().he_sync(ctx.ptr))


def he_encode(ctx: Context, slots, scale: float) -> np.ndarray:
    z = np.ascontiguousarray(slots, dtype=np.float64)
    out = np.zeros(ctx.n, dtype=np.int64)
    _check(load().he_encode(ctx.ptr, _ptr(z), len(z), float(scale), _ptr(out)))
    return out


def he_encrypt_poly(ctx: Context, coeffs, scale: float, level: int, out: Ciphertext,
                    use_sk: bool = False, cid: int = 0):
    m = np.ascontiguousarray(coeffs, dtype=np.int64)
    _run(load().he_encrypt_poly, ctx, [out], _ptr(m), float(scale), level, int(use_sk), cid, out)
    return out


def he_encode_encrypt(ctx: Context, slots, scale: float, level: int, out: Ciphertext,
                      use_sk: bool = False, cid: int = 0):
    z = np.ascontiguousarray(slots, dtype=np.float64)
    _run(load().he_encode_encrypt, ctx, [out], _ptr(z), len(z), float(scale), level, int(use_sk), cid,
         out)
    return out


def he_decrypt_poly(ctx: Context, ct: Ciphertext) -> np.ndarray:
    out = np.zeros(ctx.n, dtype=np.float64)
    _run(load().he_decrypt_poly, ctx, [], ct, _ptr(out))
    return out


def he_decrypt_decode(ctx: Context, ct: Ciphertext, n_slots: int | None = None) -> np.ndarray:
    n_slots = ctx.n // 2 if n_slots is None else n_slots
    out = np.zeros(n_slots, dtype=np.float64)
    _run(load().he_decrypt_decode, ctx, [], ct, _ptr(out), n_slots)
    return out


def he_ct_export(ctx: Context, ct: Ciphertext) -> np.ndarray:
    out = np.zeros((2, ct.level, ctx.n), dtype=np.uint64)
    _run(load().he_ct_export, ctx, [], ct, _ptr(out), out.size)
    return out


def he_ct_import(ctx: Context, residues, level: int, scale: float, out: Ciphertext):
    r = np.ascontiguousarray(residues, dtype=np.uint64)
    _run(load().he_ct_import, ctx, [out], _ptr(r), level, float(scale), out)
    return out


def he_add(ctx, a, b, out):
    _run(load().he_add, ctx, [out], a, b, out)
    return out


def he_sub(ctx, a, b, out):
    _run(load().he_sub, ctx, [out], a, b, out)
    return out


def he_drop_level(ctx, a, level: int, out):
    _run(load().he_drop_level, ctx, [out], a, level, out)
    return out


def he_mul_const(ctx, a, value: float, value_scale: float, out):
    _run(load().he_mul_const, ctx, [out], a, float(value), float(value_scale), out)
    return out


def he_add_const(ctx, a, value: float, out):
    _run(load().he_add_const, ctx, [out], a, float(value), out)
    return out


def he_mul_plain(ctx, a, coeffs, pt_scale: float, out):
    m = np.ascontiguousarray(coeffs, dtype=np.int64)
    _run(load().he_mul_plain, ctx, [out], a, _ptr(m), float(pt_scale), out)
    return out


def he_rescale(ctx, a, out):
    _run(load().he_rescale, ctx, [out], a, out)
    return out


def he_sum(ctx, cts: list, out):
    """out = sum of the ciphertexts (modular addition of residues, one scale)."""
    arr = _batch(cts)
    s = out.c()
    _check(load().he_sum(ctx.ptr, arr, len(cts), ctypes.byref(s)))
    out.update(s)
    return out


class Handle:
    """A library-owned ciphertext (he_ct_alloc): .ptr is the he_ct*; freed by
    close() or on collection."""

    def __init__(self, ctx, cap: int):
        p = CTP()
        _check(load().he_ct_alloc(ctx.ptr, cap, ctypes.byref(p)))
        self.ptr = p

    @property
    def level(self) -> int:
        return self.ptr.contents.level

    @property
    def scale(self) -> float:
        return self.ptr.contents.scale

    def close(self):
        if getattr(self, "ptr", None):
            _check(load().he_ct_free(self.ptr))
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def he_ct_alloc(ctx, cap: int) -> Handle:
    return Handle(ctx, cap)


def he_ctx_workspace(ctx) -> dict:
    """The context's workspace: bytes held now and scratch requests so far."""
    b, r = ctypes.c_size_t(), ctypes.c_uint64()
    _check(load().he_ctx_workspace(ctx.ptr, ctypes.byref(b), ctypes.byref(r)))
    return {"bytes": b.value, "requests": r.value}


def he_rescale_noalloc(ctx, a, out):
    """he_rescale with its scratch in the library's static device array (no
    allocation; for callers with a fixed device-memory budget)."""
    _run(load().he_rescale_noalloc, ctx, [out], a, out)
    return out


def he_mul_relin_rescale(ctx, a, b, out):
    _run(load().he_mul_relin_rescale, ctx, [out], a, b, out)
    return out


def he_mul_relin(ctx, a, b, out):
    _run(load().he_mul_relin, ctx, [out], a, b, out)
    return out


def he_rotate(ctx, a, steps: int, out):
    _run(load().he_rotate, ctx, [out], a, steps, out)
    return out


def he_rotate_sum(ctx, a, steps, out):
    """out = a + sum of rotate(a, s) over steps (1 to 16 steps), one shared
    decomposition; out may be a."""
    st = (ctypes.c_int32 * len(steps))(*steps)
    _run(load().he_rotate_sum, ctx, [out], a, st, len(steps), out)
    return out


def he_rotate_sum_batch(ctx, a: list, steps, out: list):
    _same_len("he_rotate_sum_batch", a, out)
    st = (ctypes.c_int32 * len(steps))(*steps)
    A, O = _batch(a), _batch(out)
    _check(load().he_rotate_sum_batch(ctx.ptr, A, st, len(steps), O, len(a)))
    for o, s in zip(out, O):
        o.update(s)
    return out


def he_mul_relin_rescale_batch(ctx, a: list, b: list, out: list):
    _same_len("he_mul_relin_rescale_batch", a, b, out)
    A, B, O = _batch(a), _batch(b), _batch(out)
    _check(load().he_mul_relin_rescale_batch(ctx.ptr, A, B, O, len(a)))
    for o, s in zip(out, O):
        o.update(s)
    return out


def he_rotate_batch(ctx, a: list, steps: int, out: list):
    _same_len("he_rotate_batch", a, out)
    A, O = _batch(a), _batch(out)
    _check(load().he_rotate_batch(ctx.ptr, A, steps, O, len(a)))
    for o, s in zip(out, O):
        o.update(s)
    return out


def he_fit_poly(x, y, degree: int) -> np.ndarray:
    """Least-squares polynomial coefficients c_0 .. c_degree of samples
    (x_i, y_i) (Eq. 3); host computation."""
    xs = np.ascontiguousarray(x, dtype=np.float64)
    ys = np.ascontiguousarray(y, dtype=np.float64)
    if xs.shape != ys.shape or xs.ndim != 1:
        raise ValueError("x and y must be 1-D arrays of one length")
    c = np.zeros(degree + 1, dtype=np.float64)
    _check(load().he_fit_poly(ctypes.c_void_p(xs.ctypes.data), ctypes.c_void_p(ys.ctypes.data), len(xs), degree,
                              ctypes.c_void_p(c.ctypes.data)))
    return c


def fit_gradient_polynomial(f, a: float, degree: int = 3, n: int = 200001, seed=None) -> np.ndarray:
    """Eq. 3: fit f by least squares on n samples of [-a, a]: random samples
    uniform in the interval with a seed, or (seed None) n evenly spaced
    points, the limit of many random samples.  With f(x) = 1/(1+e^x) (the
    negated logistic-loss derivative), a = 16 and degree 3 the latter gives
    Table 2's binomial row to its printed digits."""
    if seed is None:
        x = np.linspace(-a, a, n)
    else:
        from . import workloads
        x = workloads.uniform_slots(seed, n, -a, a)
    return he_fit_poly(x, f(x), degree)


def rotsum_stage_sizes(count: int) -> list:
    """Doublings per stage of a rotate-and-sum over 2^count offsets: stages of
    three (radix 8, seven rotations), the first of four (radix 16) when count
    = 1 mod 3 and a last one of two (radix 4) when count = 2 mod 3.  Every
    stage pays one ModUp and one ModDown and each of its rotations one inner
    product, so stages of three doublings are the cheapest split."""
    if count <= 0:
        return []
    r = count % 3
    sizes = [3] * (count // 3)
    if r == 1:
        sizes = [4] + sizes[1:] if sizes else [1]
    elif r == 2:
        sizes = sizes + [2]
    return sizes


def rotsum_stages(step: int, count: int) -> list:
    """The stages in which a rotate-and-sum over the 2^count offsets 0, step,
    2 step, ... is evaluated: one he_rotate_sum per stage of k doublings
    (rotsum_stage_sizes), with rotations by s, 2s, ..., (2^k - 1) s, then
    s <- 2^k s."""
    out, s = [], step
    for k in rotsum_stage_sizes(count):
        out.append([s * m for m in range(1, 1 << k)])
        s <<= k
    return out


def lr_rot_steps(n_slots: int, g: int) -> list:
    """Rotation steps whose Galois keys the gradient step and inference need
    for g samples per ciphertext: the feature sum (stages of step g over
    n_slots / g positions), the sample sum (step 1) and the replication
    (step -1), each over g positions."""
    log_f, log_g = (n_slots // g).bit_length() - 1, g.bit_length() - 1
    steps = []
    for st in rotsum_stages(g, log_f) + rotsum_stages(1, log_g) + rotsum_stages(-1, log_g):
        steps += [r for r in st if r not in steps]
    return steps


def lr_config(coeffs, lr: float, g: int, mask_scale: float, l2: float = 0.0) -> he_lr_config:
    """Step configuration; l2 > 0 adds the L2 regulariser's gradient l2 * w (Eq. 4, 6)."""
    return he_lr_config((ctypes.c_double * 4)(*coeffs), float(lr), g, 0, float(mask_scale), float(l2))


def he_lr_gradient_step(ctx, Z: list, W: Ciphertext, cfg: he_lr_config, W_out: Ciphertext):
    Zs = _batch(Z)
    Ws, Os = W.c(), W_out.c()
    _check(load().he_lr_gradient_step(ctx.ptr, Zs, len(Z), ctypes.byref(Ws), ctypes.byref(cfg),
                                      ctypes.byref(Os)))
    W_out.update(Os)
    return W_out


def _shards(shards, infer):
    keep, arr = [], (he_lr_shard * len(shards))()
    for k, sh in enumerate(shards):
        Z, W, out = sh[0], sh[1], sh[2]
        cid = sh[3] if len(sh) > 3 else 0x40000000 + k
        zs, w = _batch(Z), W.c()
        if infer:
            _same_len("inference shard", Z, out)
            so = _batch(out)
            keep.append((zs, w, so))
            arr[k] = he_lr_shard(ctypes.cast(zs, ctypes.c_void_p), len(Z), ctypes.addressof(w), None,
                                 ctypes.cast(so, ctypes.c_void_p), cid, 0)
        else:
            wo = out.c()
            keep.append((zs, w, wo))
            arr[k] = he_lr_shard(ctypes.cast(zs, ctypes.c_void_p), len(Z), ctypes.addressof(w),
                                 ctypes.addressof(wo), None, cid, 0)
    return arr, keep


def he_lr_train(ctx, workers: list, cfg: he_lr_config, iterations: int, refresh_every: int, top_level: int,
                W_final, cid0: int = 1 << 20):
    """workers: list of (Z list, W at top_level).  Returns W_final (the last
    averaged weights, re-encrypted at top_level)."""
    shards = [(Z, W, W) for Z, W in workers]  # W_out is not used by the loop
    arr, keep = _shards(shards, False)
    f = W_final.c()
    _check(load().he_lr_train(ctx.ptr, arr, len(workers), ctypes.byref(cfg), iterations, refresh_every, top_level,
                              cid0, ctypes.byref(f)))
    W_final.update(f)
    return W_final


def he_lr_gradient_step_host(ctx, Z_host, z_level: int, z_scale: float, W_host, w_level: int, w_scale: float,
                             cfg: he_lr_config, out_host):
    """The step on host buffers (numpy uint64 arrays or pinned CPU torch tensors):
    Z_host [nZ][2][z_level][N], W_host [2][w_level][N], out_host >= [2][w_level-5][N].
    Returns (level, scale) of the result."""
    if (_nwords(Z_host) < Z_host.shape[0] * 2 * z_level * ctx.n or _nwords(W_host) < 2 * w_level * ctx.n):
        raise ValueError("he_lr_gradient_step_host: host arrays smaller than their ciphertexts")
    lv, sc = ctypes.c_uint32(), ctypes.c_double()
    _check(load().he_lr_gradient_step_host(ctx.ptr, ctypes.c_void_p(_addr(Z_host)), Z_host.shape[0], z_level,
                                           float(z_scale), ctypes.c_void_p(_addr(W_host)), w_level, float(w_scale),
                                           ctypes.byref(cfg), ctypes.c_void_p(_addr(out_host)), _nwords(out_host),
                                           ctypes.byref(lv), ctypes.byref(sc)))
    return lv.value, sc.value


def he_lr_gradient_step_workers(ctx, shards: list, cfg: he_lr_config, refresh_level: int = 0,
                                graph: bool = False):
    """shards: list of (Z list, W, W_out[, refresh_cid]) per worker."""
    arr, keep = _shards(shards, False)
    _check(load().he_lr_gradient_step_workers(ctx.ptr, arr, len(shards), ctypes.byref(cfg), refresh_level,
                                              HE_LR_GRAPH if graph else 0))
    for sh, (_, _, wo) in zip(shards, keep):
        sh[2].update(wo)
    return [s[2] for s in shards]


def he_lr_inference_workers(ctx, shards: list, cfg: he_lr_config, refresh_level: int = 0,
                            graph: bool = False):
    """shards: list of (Z list, W, S_out list[, refresh_cid]) per worker."""
    arr, keep = _shards(shards, True)
    _check(load().he_lr_inference_workers(ctx.ptr, arr, len(shards), ctypes.byref(cfg), refresh_level,
                                          HE_LR_GRAPH if graph else 0))
    for sh, (_, _, so) in zip(shards, keep):
        for o, s in zip(sh[2], so):
            o.update(s)
    return [s[2] for s in shards]


def he_refresh(ctx, a, level: int, out_scale: float, cid: int, out):
    _run(load().he_refresh, ctx, [out], a, level, float(out_scale), cid, out)
    return out


def he_ntt(ctx, tensor, npolys: int, poly_stride: int, nl: int, prime0: int, inverse: bool):
    """In-place NTT of limbs of device polynomials held by an int64 tensor."""
    _check(load().he_ntt(ctx.ptr, ctypes.c_void_p(tensor.data_ptr()), npolys, poly_stride, nl, prime0,
                         int(inverse)))
    return tensor


def he_keyswitch(ctx, d, level: int, galois: int, out0, out1):
    _check(load().he_keyswitch(ctx.ptr, ctypes.c_void_p(d.data_ptr()), level, galois,
                               ctypes.c_void_p(out0.data_ptr()), ctypes.c_void_p(out1.data_ptr())))
    return out0, out1


def he_moddown(ctx, acc, level: int, out, d01=None):
    """ModDown of a device accumulator acc ([2][level + alpha][N] residues in
    an int64 tensor): round(acc / P) into out at `level`, or with d01 the
    merged form round((P d01 + acc) / (P q_{level-1})) at level - 1."""
    if acc.numel() < 2 * (level + ctx.alpha) * ctx.n:
        raise ValueError("he_moddown: accumulator smaller than [2][level + alpha][N]")
    if d01 is None:
        _run(load().he_moddown, ctx, [out], ctypes.c_void_p(acc.data_ptr()), level, None, out)
    else:
        _run(load().he_moddown, ctx, [out], ctypes.c_void_p(acc.data_ptr()), level, d01, out)
    return out


def he_ct_import_batch(ctx, host, level: int, scale: float, out: list):
    """host: uint64 array [count][2][level][N] (pinned memory copies fastest)."""
    if _nwords(host) < len(out) * 2 * level * ctx.n:
        raise ValueError("he_ct_import_batch: host array smaller than the ciphertexts")
    O = _batch(out)
    _check(load().he_ct_import_batch(ctx.ptr, ctypes.c_void_p(_addr(host)), level, float(scale), O, len(out)))
    for o, s in zip(out, O):
        o.update(s)
    return out


def he_ct_export_batch(ctx, cts: list, host):
    A = _batch(cts)
    _check(load().he_ct_export_batch(ctx.ptr, A, len(cts), ctypes.c_void_p(_addr(host)), _nwords(host)))
    return host


def _addr(x) -> int:
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()  # a host torch tensor (e.g. pinned)


def _nwords(x) -> int:
    if isinstance(x, np.ndarray):
        return x.size * x.itemsize // 8
    return x.numel() * x.element_size() // 8


def he_profile_enable(ctx, enable: bool):
    _check(load().he_profile_enable(ctx.ptr, int(enable)))


def he_profile_read(ctx, kernel_class: str) -> dict:
    n = ctypes.c_uint64()
    ms, work, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().he_profile_read(ctx.ptr, kernel_class.encode(), ctypes.byref(n), ctypes.byref(ms),
                                  ctypes.byref(work), ctypes.byref(by)))
    bfly, mac, mac3 = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().he_profile_read_kinds(ctx.ptr, kernel_class.encode(), ctypes.byref(bfly), ctypes.byref(mac),
                                        ctypes.byref(mac3)))
    return {"launches": n.value, "ms": ms.value, "work": work.value, "bytes": by.value, "mac": mac.value,
            "mac3": mac3.value, "bfly": bfly.value}


def he_profile_names(ctx) -> list:
    buf = ctypes.create_string_buffer(4096)
    _check(load().he_profile_names(ctx.ptr, buf, 4096))
    v = buf.value.decode()
    return v.split(",") if v else []


def galois_elt(log_n: int, r: int) -> int:
    """5^(r mod N/2) mod 2N, the Galois element of a left rotation by r."""
    slots = 1 << (log_n - 1)
    return pow(5, r % slots, 2 << log_n)


class Server:
    """he_server: a continuous-batching request loop over several contexts."""

    def __init__(self, ctxs: list, hbm_budget: int, max_inflight: int = 4, max_wave: int = 16,
                 max_running: int = 0):
        self._ctxs = ctxs
        self._arr = (ctypes.c_void_p * len(ctxs))(*[c.ptr.value for c in ctxs])
        cfg = he_server_config(ctypes.cast(self._arr, ctypes.c_void_p), len(ctxs), int(hbm_budget),
                               max_inflight, max_wave, max_running)
        h = ctypes.c_void_p()
        _check(load().he_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.ptr = h
        self._keep = {}

    def submit(self, ctx_index: int, kind: int, Z_host, z_level: int, z_scale: float, W_host, w_level: int,
               w_scale: float, cfg: he_lr_config, out_host, refresh_cid: int = 0, min_w_level: int = 0) -> int:
        """Z_host, W_host, out_host: host arrays or (pinned) CPU torch tensors of uint64 residues."""
        nZ = Z_host.shape[0]
        r = he_request(ctx_index, kind, nZ, z_level, w_level, refresh_cid, min_w_level, float(z_scale), float(w_scale),
                       _addr(Z_host), _addr(W_host), cfg, _addr(out_host), _nwords(out_host))
        rid = ctypes.c_uint64()
        _check(load().he_server_submit(self.ptr, ctypes.byref(r), ctypes.byref(rid)))
        self._keep[rid.value] = (Z_host, W_host, out_host)
        return rid.value

    def poll(self, cap: int = 1024) -> list:
        res = (he_result * cap)()
        n = ctypes.c_size_t()
        _check(load().he_server_poll(self.ptr, res, cap, ctypes.byref(n)))
        out = []
        for i in range(n.value):
            r = res[i]
            self._keep.pop(r.id, None)
            out.append({"id": r.id, "status": r.status, "level": r.level, "scale": r.scale,
                        "latency_ms": r.latency_ms})
        return out

    def drain(self, timeout_s: float = 600.0):
        _check(load().he_server_drain(self.ptr, float(timeout_s)))

    def last_error(self) -> str:
        buf = ctypes.create_string_buffer(512)
        _check(load().he_server_last_error(self.ptr, buf, 512))
        return buf.value.decode()

    def stats(self) -> dict:
        v = [ctypes.c_size_t() for _ in range(4)]
        _check(load().he_server_stats(self.ptr, *[ctypes.byref(x) for x in v]))
        return dict(zip(("used", "peak_used", "waves", "peak_running"), [x.value for x in v]))

    def close(self):
        if getattr(self, "ptr", None):
            load().he_server_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
